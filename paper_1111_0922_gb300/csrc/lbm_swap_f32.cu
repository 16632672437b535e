// Swap kernels instantiated for one storage precision (f32); the templates
// live in lbm_swap.cuh.
#include "lbm_swap.cuh"

namespace lbmk {
template void swap_pass_t<CodecF32>(const StepParams &, const SwapPass &, const KernelKey &, size_t, cudaStream_t);
template int swap_pass_tma_t<CodecF32>(const StepParams &, const SwapPass &, const KernelKey &, const CUtensorMap *,
                                     int, int, cudaStream_t);
template void swap_pass_pair_t<CodecPair<CodecF32>>(const StepParams &, const SwapPass &, const KernelKey &, size_t,
                                                    cudaStream_t);
}  // namespace lbmk
