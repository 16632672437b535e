// Kernels that move a natural state into and out of each scheme's storage,
// and read moments and FP64 mass/flux partials from it.  Instantiated per
// storage precision in lbm_state_*.cu.
#pragma once

#include <algorithm>

#include "lbm_dispatch.cuh"
#include "lbm_internal.h"

namespace lbmk {

static inline unsigned state_grid_for(int64_t n, int threads) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 1 << 20));
}

// ---------------------------------------------------------------------------
// Natural state <-> storage.  For every node: the slot holding f_i(x).
template <class C, int AOS, bool IND>
struct NodeSlots {
  int s;
  bool fluid;
  int x, y, z;
  __device__ __forceinline__ void init(const StepParams &p, int64_t n) {
    if (IND) {
      s = (int)n;
      fluid = true;
    } else {
      DirectNode nd;
      fluid = nd.init(p, n);
      s = fluid ? ((p.g.zpair || p.g.ypair) ? (int)grid_slot(p.g, nd.x, nd.y, nd.z) : nd.s) : -1;
      x = nd.x;
      y = nd.y;
      z = nd.z;
    }
  }
  __device__ __forceinline__ int nb(const StepParams &p, int i) const {
    if (IND) return __ldg(p.idx + (int64_t)(i - 1) * p.ipad + s);
    return (int)grid_neighbour(p.g, x, y, z, CX(i), CY(i), CZ(i));
  }
  // slot (array, position) of f_i(x) under map kind M
  template <int M>
  __device__ __forceinline__ void where(const StepParams &p, int i, int &arr, int &pos) const {
    if (M == MAP_NATURAL || i == 0) {
      arr = (M == MAP_ET) ? p.map[i] : i;
      pos = s;
      return;
    }
    if (M == MAP_PULL) {
      const int src = nb(p, OPP(i));
      if (src >= 0) {
        arr = i;
        pos = src;
      } else {
        arr = OPP(i);
        pos = s;
      }
      return;
    }
    // MAP_ET
    arr = p.map[i];
    if (i & 1) {
      pos = s;
    } else if (IND) {
      pos = (int)((uint32_t)__ldg(p.idx + (int64_t)((i - 2) / 2) * p.ipad + s) & 0x7fffffffu);
    } else {
      pos = (int)grid_position(p.g, x, y, z, CX(i - 1), CY(i - 1), CZ(i - 1));
    }
  }
};

template <class C, int AOS, bool IND, int M>
__global__ void k_put_state(StepParams p, const double *f_nat, const double *rho, const double *u) {
  using T = typename C::T;
  Lattice<C, AOS> L{static_cast<typename C::S *>(p.A), p.npad, p.scale, p.inv_scale};
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < p.nnodes; n += (int64_t)gridDim.x * blockDim.x) {
    NodeSlots<C, AOS, IND> ns;
    ns.init(p, n);
    if (!ns.fluid) continue;
    double f[Q];
    if (f_nat) {
#pragma unroll
      for (int i = 0; i < Q; ++i) f[i] = f_nat[(int64_t)i * p.nnodes + n];
    } else {
      const double r = rho ? rho[n] : 1.0;
      const double ux = u ? u[3 * n] : 0.0, uy = u ? u[3 * n + 1] : 0.0, uz = u ? u[3 * n + 2] : 0.0;
      const double usq = ux * ux + uy * uy + uz * uz;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const double cu = CX(i) * ux + CY(i) * uy + CZ(i) * uz;
        f[i] = WD(i) * r * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
      }
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      int arr, pos;
      ns.template where<M>(p, i, arr, pos);
      L.st_dev(arr, pos, (T)(f[i] - WD(i)));
    }
  }
}

template <class C, int AOS, bool IND, int M>
__device__ __forceinline__ void read_natural(const StepParams &p, const NodeSlots<C, AOS, IND> &ns, double (&f)[Q]) {
  Lattice<C, AOS> L{static_cast<typename C::S *>(p.A), p.npad, p.scale, p.inv_scale};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    int arr, pos;
    ns.template where<M>(p, i, arr, pos);
    f[i] = WD(i) + (double)L.ld_dev(arr, pos);
  }
}

template <class C, int AOS, bool IND, int M>
__global__ void k_get_state(StepParams p, double *f_nat) {
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < p.nnodes; n += (int64_t)gridDim.x * blockDim.x) {
    NodeSlots<C, AOS, IND> ns;
    ns.init(p, n);
    double f[Q];
    if (ns.fluid) {
      read_natural<C, AOS, IND, M>(p, ns, f);
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) f[i] = 0.0;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) f_nat[(int64_t)i * p.nnodes + n] = f[i];
  }
}

__device__ __forceinline__ void moments(const double (&f)[Q], const StepParams &p, double &rho, double &ux, double &uy,
                                        double &uz) {
  rho = 0.0;
  double jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    rho += f[i];
    jx += CX(i) * f[i];
    jy += CY(i) * f[i];
    jz += CZ(i) * f[i];
  }
  ux = (jx + 0.5 * rho * p.gx) / rho;
  uy = (jy + 0.5 * rho * p.gy) / rho;
  uz = (jz + 0.5 * rho * p.gz) / rho;
}

template <class C, int AOS, bool IND, int M>
__global__ void k_macroscopics(StepParams p, double *rho, double *u) {
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < p.nnodes; n += (int64_t)gridDim.x * blockDim.x) {
    NodeSlots<C, AOS, IND> ns;
    ns.init(p, n);
    double r = 0.0, ux = 0.0, uy = 0.0, uz = 0.0;
    if (ns.fluid) {
      double f[Q];
      read_natural<C, AOS, IND, M>(p, ns, f);
      moments(f, p, r, ux, uy, uz);
    }
    if (rho) rho[n] = r;
    if (u) {
      u[3 * n] = ux;
      u[3 * n + 1] = uy;
      u[3 * n + 2] = uz;
    }
  }
}

template <class C, int AOS, bool IND, int M>
__global__ void __launch_bounds__(256) k_flux_partials(StepParams p, double *partials) {
  double m = 0.0, j = 0.0;
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < p.nnodes; n += (int64_t)gridDim.x * blockDim.x) {
    NodeSlots<C, AOS, IND> ns;
    ns.init(p, n);
    if (!ns.fluid) continue;
    double f[Q], r, ux, uy, uz;
    read_natural<C, AOS, IND, M>(p, ns, f);
    moments(f, p, r, ux, uy, uz);
    m += r;
    j += r * ux;
  }
  block_reduce_store(m, j, partials);
}

// ---------------------------------------------------------------------------
// Dispatch of the state kernels over layout x addressing x map.
template <class C, int AOS, bool IND, bool, bool>
struct StateOps {
  template <int M>
  static void put(const StateDesc &d, const double *f, const double *rho, const double *u, cudaStream_t s) {
    k_put_state<C, AOS, IND, M><<<state_grid_for(d.p.nnodes, 256), 256, 0, s>>>(d.p, f, rho, u);
  }
  template <int M>
  static void get(const StateDesc &d, double *f, cudaStream_t s) {
    k_get_state<C, AOS, IND, M><<<state_grid_for(d.p.nnodes, 256), 256, 0, s>>>(d.p, f);
  }
  template <int M>
  static void macro(const StateDesc &d, double *rho, double *u, cudaStream_t s) {
    k_macroscopics<C, AOS, IND, M><<<state_grid_for(d.p.nnodes, 256), 256, 0, s>>>(d.p, rho, u);
  }
  template <int M>
  static void flux(const StateDesc &d, double *partials, int nb, cudaStream_t s) {
    k_flux_partials<C, AOS, IND, M><<<nb, 256, 0, s>>>(d.p, partials);
  }
  static void run(int op, const StateDesc &d, const double *fin, double *fout, const double *rho, double *rout,
                  const double *u, double *uout, double *partials, int nb, cudaStream_t s) {
#define LBM_MAPS(CALL)          \
  switch (d.mapkind) {          \
    case MAP_NATURAL:           \
      CALL(MAP_NATURAL);        \
      break;                    \
    case MAP_PULL:              \
      CALL(MAP_PULL);           \
      break;                    \
    default:                    \
      CALL(MAP_ET);             \
      break;                    \
  }
#define LBM_PUT(M) put<M>(d, fin, rho, u, s)
#define LBM_GET(M) get<M>(d, fout, s)
#define LBM_MAC(M) macro<M>(d, rout, uout, s)
#define LBM_FLX(M) flux<M>(d, partials, nb, s)
    if (op == 0) {
      LBM_MAPS(LBM_PUT)
    } else if (op == 1) {
      LBM_MAPS(LBM_GET)
    } else if (op == 2) {
      LBM_MAPS(LBM_MAC)
    } else {
      LBM_MAPS(LBM_FLX)
    }
#undef LBM_PUT
#undef LBM_GET
#undef LBM_MAC
#undef LBM_FLX
#undef LBM_MAPS
  }
};

template <class C>
void state_op_t(int op, const StateDesc &d, const double *fin, double *fout, const double *rho,
                double *rout, const double *u, double *uout, double *partials, int nb, cudaStream_t s) {
  dispatch_layout<StateOps, C>(d.k.aos, d.k.ind, false, false, op, d, fin, fout, rho, rout, u, uout, partials, nb, s);
}

}  // namespace lbmk
