// Swap kernels instantiated for one storage precision (f16s); the templates
// live in lbm_swap.cuh.
#include "lbm_swap.cuh"

namespace lbmk {
template void swap_pass_t<CodecF16S>(const StepParams &, const SwapPass &, const KernelKey &, size_t, cudaStream_t);
template int swap_pass_tma_t<CodecF16S>(const StepParams &, const SwapPass &, const KernelKey &, const CUtensorMap *,
                                     int, int, cudaStream_t);
template void swap_pass_pair_t<CodecPair<CodecF16S>>(const StepParams &, const SwapPass &, const KernelKey &, size_t,
                                                     cudaStream_t);
}  // namespace lbmk
