// Fused collide-and-propagate kernels for the order-free propagation schemes:
// two-step (Sec. 2), one-step push and pull (Sec. 3), AA pattern (Sec. 6) and
// esoteric twist (Sec. 7).  One thread updates one node per loop iteration
// (grid-stride loop, so a launch may give each thread several nodes).  All
// kernels load the 19 PDFs of a node, run the collision in registers and
// store 19 PDFs: q loads + q stores per update, no read-for-ownership on the
// GPU (full-sector stores allocate in L2 without a DRAM read).
#pragma once

#include "lbm_dispatch.cuh"
#include "lbm_internal.h"

namespace lbmk {

template <class C, int AOS>
__device__ __forceinline__ Lattice<C, AOS> lattice_of(void *p, const StepParams &P) {
  Lattice<C, AOS> L;
  L.p = static_cast<typename C::S *>(p);
  L.npad = P.npad;
  L.scale = P.scale;
  L.inv_scale = P.inv_scale;
  return L;
}

template <typename T, bool FORCE>
__device__ __forceinline__ void run_collision(T (&d)[Q], const StepParams &p, double &m, double &j) {
  T drho, rjx;
  collide<T, FORCE>(d, T(p.omega), T(p.gx), T(p.gy), T(p.gz), drho, rjx);
  m += 1.0 + (double)drho;
  j += (double)rjx;
}

#define LBM_GRID_LOOP(n) \
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < p.nnodes; n += (int64_t)gridDim.x * blockDim.x)

// ---------------------------------------------------------------------------
// Two-step, kernel 1 (Tab. 1, collision): A -> B at the same slot.
template <class C, int AOS, class Node, bool FORCE, bool RED>
__global__ void __launch_bounds__(512) k_ts_collide(StepParams p) {
  using T = typename C::T;
  const auto A = lattice_of<C, AOS>(p.A, p);
  const auto B = lattice_of<C, AOS>(p.B, p);
  double m = 0.0, j = 0.0;
  LBM_GRID_LOOP(n) {
    Node nd;
    if (!nd.init(p, n)) continue;
    T d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = A.ld(i, nd.s);
    run_collision<T, FORCE>(d, p, m, j);
#pragma unroll
    for (int i = 0; i < Q; ++i) B.st(i, nd.s, d[i]);
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

// Two-step, kernel 2 (Tab. 1, propagation), pull form: A_i(x) = B_i(x - c_i),
// or B_opp(i)(x) across a solid/wall link.  Raw copies: bit-exact.
template <class C, int AOS, class Node>
__global__ void __launch_bounds__(512) k_ts_stream(StepParams p) {
  const auto A = lattice_of<C, AOS>(p.A, p);
  const auto B = lattice_of<C, AOS>(p.B, p);
  LBM_GRID_LOOP(n) {
    Node nd;
    if (!nd.init(p, n)) continue;
    *A.at(0, nd.s) = *B.at(0, nd.s);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int src = nd.nb(p, OPP(i));
      *A.at(i, nd.s) = src >= 0 ? *B.at(i, src) : *B.at(OPP(i), nd.s);
    }
  }
}

// One-step push (Fig. 1a,b): read A at the node, write B at the neighbours.
template <class C, int AOS, class Node, bool FORCE, bool RED>
__global__ void __launch_bounds__(512) k_os_push(StepParams p) {
  using T = typename C::T;
  const auto A = lattice_of<C, AOS>(p.A, p);
  const auto B = lattice_of<C, AOS>(p.B, p);
  double m = 0.0, j = 0.0;
  LBM_GRID_LOOP(n) {
    Node nd;
    if (!nd.init(p, n)) continue;
    T d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = A.ld(i, nd.s);
    run_collision<T, FORCE>(d, p, m, j);
    B.st(0, nd.s, d[0]);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int dst = nd.nb(p, i);
      if (dst >= 0)
        B.st(i, dst, d[i]);
      else
        B.st(OPP(i), nd.s, d[i]);
    }
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

// One-step pull (Fig. 1c,d): gather from the neighbours in A, write B at the
// node.  The stored state is post-collision.
template <class C, int AOS, class Node, bool FORCE, bool RED>
__global__ void __launch_bounds__(512) k_os_pull(StepParams p) {
  using T = typename C::T;
  const auto A = lattice_of<C, AOS>(p.A, p);
  const auto B = lattice_of<C, AOS>(p.B, p);
  double m = 0.0, j = 0.0;
  LBM_GRID_LOOP(n) {
    Node nd;
    if (!nd.init(p, n)) continue;
    T d[Q];
    d[0] = A.ld(0, nd.s);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int src = nd.nb(p, OPP(i));
      d[i] = src >= 0 ? A.ld(i, src) : A.ld(OPP(i), nd.s);
    }
    run_collision<T, FORCE>(d, p, m, j);
#pragma unroll
    for (int i = 0; i < Q; ++i) B.st(i, nd.s, d[i]);
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

// AA pattern, even step (Fig. 5a,b): node-local; the post-collision PDF of
// direction i goes to the node's slot of the opposite direction.
template <class C, int AOS, class Node, bool FORCE, bool RED>
__global__ void __launch_bounds__(512) k_aa_even(StepParams p) {
  using T = typename C::T;
  const auto A = lattice_of<C, AOS>(p.A, p);
  double m = 0.0, j = 0.0;
  LBM_GRID_LOOP(n) {
    Node nd;
    if (!nd.init(p, n)) continue;
    T d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = A.ld(i, nd.s);
    run_collision<T, FORCE>(d, p, m, j);
#pragma unroll
    for (int i = 0; i < Q; ++i) A.st(OPP(i), nd.s, d[i]);
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

// AA pattern, odd step (Fig. 5c,d): f_i comes from the opposite slot of the
// node at x - c_i (own slot i across a solid link); the result goes to slot i
// of x + c_i (own opposite slot across a solid link).  Every slot written was
// read by the same thread.
template <class C, int AOS, class Node, bool FORCE, bool RED>
__global__ void __launch_bounds__(512) k_aa_odd(StepParams p) {
  using T = typename C::T;
  const auto A = lattice_of<C, AOS>(p.A, p);
  double m = 0.0, j = 0.0;
  LBM_GRID_LOOP(n) {
    Node nd;
    if (!nd.init(p, n)) continue;
    int nb[Q];
#pragma unroll
    for (int i = 1; i < Q; ++i) nb[i] = nd.nb(p, i);
    T d[Q];
    d[0] = A.ld(0, nd.s);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int src = nb[OPP(i)];
      d[i] = src >= 0 ? A.ld(OPP(i), src) : A.ld(i, nd.s);
    }
    run_collision<T, FORCE>(d, p, m, j);
    A.st(0, nd.s, d[0]);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int dst = nb[i];
      if (dst >= 0)
        A.st(i, dst, d[i]);
      else
        A.st(OPP(i), nd.s, d[i]);
    }
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

// Esoteric twist (Fig. 6): PDF f_i of node x lives in array map[i] at x for
// the rest and odd directions, and at x + c_{i-1} for even i (the neighbour
// along the odd direction i-1).  Post-collision f_i goes to array map[opp i]
// at x + s(opp i); across a solid link to array map[i] at the same slot.  The
// host then exchanges map[i] and map[opp i].
//   direct:   positions and solid tests from coordinates; beyond a wall the
//             position is a halo slot
//   indirect: word k of the packed index (k = 0..8, direction 2k+1) holds the
//             slot of x + c_{2k+1} in bits 0..30 (a ghost slot >= nfluid when
//             that cell is solid) and in bit 31 whether x + c_{2k+2} is solid.
template <class C, int AOS, bool IND, bool FORCE, bool RED>
__global__ void __launch_bounds__(512) k_et(StepParams p) {
  using T = typename C::T;
  const auto A = lattice_of<C, AOS>(p.A, p);
  double m = 0.0, j = 0.0;
  LBM_GRID_LOOP(n) {
    int s;
    int pos[10];
    bool lp[10], lm[10];
    if (IND) {
      s = (int)n;
#pragma unroll
      for (int k = 1; k <= 9; ++k) {
        const uint32_t w = (uint32_t)__ldg(p.idx + (int64_t)(k - 1) * p.ipad + n);
        pos[k] = (int)(w & 0x7fffffffu);
        lp[k] = pos[k] < p.nfluid;
        lm[k] = (w >> 31) == 0u;
      }
    } else {
      DirectNode nd;
      if (!nd.init(p, n)) continue;
      s = nd.s;
#pragma unroll
      for (int k = 1; k <= 9; ++k) {
        const int i = 2 * k - 1;
        pos[k] = (int)grid_position(p.g, nd.x, nd.y, nd.z, CX(i), CY(i), CZ(i));
        lp[k] = nd.nb(p, i) >= 0;
        lm[k] = nd.nb(p, i + 1) >= 0;
      }
    }
    T d[Q];
    d[0] = A.ld(p.map[0], s);
#pragma unroll
    for (int k = 1; k <= 9; ++k) {
      d[2 * k - 1] = A.ld(p.map[2 * k - 1], s);
      d[2 * k] = A.ld(p.map[2 * k], pos[k]);
    }
    run_collision<T, FORCE>(d, p, m, j);
    A.st(p.map[0], s, d[0]);
#pragma unroll
    for (int k = 1; k <= 9; ++k) {
      // odd direction 2k-1: to x + c_{2k-1}
      A.st(lp[k] ? p.map[2 * k] : p.map[2 * k - 1], pos[k], d[2 * k - 1]);
      // even direction 2k: to x itself
      A.st(lm[k] ? p.map[2 * k - 1] : p.map[2 * k], s, d[2 * k]);
    }
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

// ---------------------------------------------------------------------------
// Launchers.
template <bool IND>
using NodeOf = typename std::conditional<IND, IndirectNode, DirectNode>::type;

template <class C, int AOS, bool IND, bool FORCE, bool RED>
struct LaunchTS {
  static void run(const StepParams &p, int phase, const LaunchShape &L) {
    if (phase == 0)
      k_ts_collide<C, AOS, NodeOf<IND>, FORCE, RED><<<L.grid, L.block, 0, L.stream>>>(p);
    else
      k_ts_stream<C, AOS, NodeOf<IND>><<<L.grid, L.block, 0, L.stream>>>(p);
  }
};
template <class C, int AOS, bool IND, bool FORCE, bool RED>
struct LaunchOS {
  static void run(const StepParams &p, int push, const LaunchShape &L) {
    if (push)
      k_os_push<C, AOS, NodeOf<IND>, FORCE, RED><<<L.grid, L.block, 0, L.stream>>>(p);
    else
      k_os_pull<C, AOS, NodeOf<IND>, FORCE, RED><<<L.grid, L.block, 0, L.stream>>>(p);
  }
};
template <class C, int AOS, bool IND, bool FORCE, bool RED>
struct LaunchAA {
  static void run(const StepParams &p, int odd, const LaunchShape &L) {
    if (odd)
      k_aa_odd<C, AOS, NodeOf<IND>, FORCE, RED><<<L.grid, L.block, 0, L.stream>>>(p);
    else
      k_aa_even<C, AOS, NodeOf<IND>, FORCE, RED><<<L.grid, L.block, 0, L.stream>>>(p);
  }
};
template <class C, int AOS, bool IND, bool FORCE, bool RED>
struct LaunchET {
  static void run(const StepParams &p, int, const LaunchShape &L) {
    k_et<C, AOS, IND, FORCE, RED><<<L.grid, L.block, 0, L.stream>>>(p);
  }
};

template <class C>
void launch_step_kernel_t(int variant, int sub, const StepParams &p, const KernelKey &k, const LaunchShape &L) {
  switch (variant) {
    case VAR_TS:
      dispatch_layout<LaunchTS, C>(k.aos, k.ind, k.force, k.red, p, sub, L);
      break;
    case VAR_OS_PUSH:
      dispatch_layout<LaunchOS, C>(k.aos, k.ind, k.force, k.red, p, 1, L);
      break;
    case VAR_OS_PULL:
      dispatch_layout<LaunchOS, C>(k.aos, k.ind, k.force, k.red, p, 0, L);
      break;
    case VAR_AA:
      dispatch_layout<LaunchAA, C>(k.aos, k.ind, k.force, k.red, p, sub, L);
      break;
    case VAR_ET:
      dispatch_layout<LaunchET, C>(k.aos, k.ind, k.force, k.red, p, 0, L);
      break;
    default:
      break;
  }
}

}  // namespace lbmk
