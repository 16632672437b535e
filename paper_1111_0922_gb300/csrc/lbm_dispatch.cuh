// Runtime -> compile-time dispatch for the kernel templates:
// precision x layout x addressing x force x fused reduction.
#pragma once

#include "lbm_core.cuh"

namespace lbmk {

// Chained launches (programmatic dependent launch) for the step kernels:
// the next kernel (the next step, or the next swap colour pass, compressed-
// grid slab or two-step kernel of the same step) may be scheduled while the
// previous one drains, so its blocks are resident when it finishes instead
// of after a launch gap (measured on 256^3: compressed grid +3 to +4 %,
// swap +2 to +3 %, two-step +1 %).  Every kernel launched this
// way starts with chain_wait(): griddepcontrol.wait returns once the
// previous kernel in the stream has completed and its stores are visible;
// launch_dependents then lets the following kernel be scheduled.
__device__ __forceinline__ void chain_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline void launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                           Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// L<C, AOS, IND, FORCE, RED>::run(args...) is called with the template
// arguments matching the runtime flags.
template <template <class, int, bool, bool, bool> class L, class C, int AOS, bool IND, bool FORCE, class... A>
inline void dispatch_red(bool red, A &&...a) {
  if (red)
    L<C, AOS, IND, FORCE, true>::run(a...);
  else
    L<C, AOS, IND, FORCE, false>::run(a...);
}
template <template <class, int, bool, bool, bool> class L, class C, int AOS, bool IND, class... A>
inline void dispatch_force(bool force, bool red, A &&...a) {
  if (force)
    dispatch_red<L, C, AOS, IND, true>(red, a...);
  else
    dispatch_red<L, C, AOS, IND, false>(red, a...);
}
template <template <class, int, bool, bool, bool> class L, class C, int AOS, class... A>
inline void dispatch_ind(bool ind, bool force, bool red, A &&...a) {
  if (ind)
    dispatch_force<L, C, AOS, true>(force, red, a...);
  else
    dispatch_force<L, C, AOS, false>(force, red, a...);
}
template <template <class, int, bool, bool, bool> class L, class C, class... A>
inline void dispatch_layout(int aos, bool ind, bool force, bool red, A &&...a) {
  if (aos)
    dispatch_ind<L, C, 1>(ind, force, red, a...);
  else
    dispatch_ind<L, C, 0>(ind, force, red, a...);
}
// precision: 0 = F64, 1 = F32, 2 = F16S
template <template <class, int, bool, bool, bool> class L, class... A>
inline void dispatch(int precision, int aos, bool ind, bool force, bool red, A &&...a) {
  if (precision == 0)
    dispatch_layout<L, CodecF64>(aos, ind, force, red, a...);
  else if (precision == 1)
    dispatch_layout<L, CodecF32>(aos, ind, force, red, a...);
  else
    dispatch_layout<L, CodecF16S>(aos, ind, force, red, a...);
}

}  // namespace lbmk
