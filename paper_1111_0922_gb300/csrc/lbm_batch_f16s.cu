// Batch step kernels instantiated for one storage precision (f16s); the
// templates live in lbm_batch.cuh.
#define LBM_BATCH_KERNELS
#include "lbm_batch.cuh"

namespace lbmk {
template cudaError_t launch_batch_t<CodecF16S>(int, int, int, bool, const BatchParams &, int, int, unsigned *, int *, uint64_t,
                                       int, cudaStream_t);
}  // namespace lbmk
