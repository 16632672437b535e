// Step kernels instantiated for one storage precision (f32); the
// templates live in lbm_steps.cuh.
#include "lbm_steps.cuh"

namespace lbmk {
template void launch_step_kernel_t<CodecF32>(int, int, const StepParams &, const KernelKey &, const LaunchShape &);
}  // namespace lbmk
