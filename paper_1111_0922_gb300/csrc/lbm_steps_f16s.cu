// Step kernels instantiated for one storage precision (f16s); the
// templates live in lbm_steps.cuh.
#include "lbm_steps.cuh"

namespace lbmk {
template void launch_step_kernel_t<CodecF16S>(int, int, const StepParams &, const KernelKey &, const LaunchShape &);
}  // namespace lbmk
