// State kernels instantiated for one storage precision (f64); the
// templates live in lbm_state.cuh.
#include "lbm_state.cuh"

namespace lbmk {
template void state_op_t<CodecF64>(int, const StateDesc &, const double *, double *, const double *, double *,
                              const double *, double *, double *, int, cudaStream_t);
}  // namespace lbmk
