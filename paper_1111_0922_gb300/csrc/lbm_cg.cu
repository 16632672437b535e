// Compressed grid (Sec. 4, Fig. 2, Tab. 3) on a full grid, pull form.
//
// The paper shifts the whole lattice by one cell per axis between steps and
// sweeps serially, alternating the sweep direction.  A serial sweep cannot
// run in parallel, so the shift here is along z only and by k planes: the
// post-collision state of plane z lives at storage plane z + o, o alternating
// between 0 and k.  A sweep reads at offset o and writes at offset o' (the
// other one).  Writing plane z + o' overwrites the old data of plane z + o' - o,
// whose readers are planes z + o' - o - 1 .. z + o' - o + 1.  Processing planes
// in slabs of k - 1 consecutive planes, descending when o' > o and ascending
// otherwise, puts every reader of an overwritten plane in an earlier slab, so
// each slab is one race-free launch.  On a periodic z axis one ghost plane
// below and above the data holds a copy of the opposite face, refreshed before
// each sweep, so a sweep never wraps.  Storage: nz + k + 2 planes.
#include <algorithm>

#include "lbm_dispatch.cuh"
#include "lbm_internal.h"

namespace lbmk {

template <class C, int AOS, bool IND, bool FORCE, bool RED>
__global__ void __launch_bounds__(512) k_cg_slab(StepParams p) {
  using T = typename C::T;
  Lattice<C, AOS> L{static_cast<typename C::S *>(p.A), p.npad, p.scale, p.inv_scale};
  const Grid &g = p.g;
  const int64_t plane = (int64_t)g.nx * g.ny;
  const int64_t count = plane * (p.z1 - p.z0);
  double m = 0.0, jsum = 0.0;
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < count; n += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(n % g.nx);
    const int y = (int)((n / g.nx) % g.ny);
    const int z = p.z0 + (int)(n / plane);
    if (grid_solid(g, x, y, z)) continue;
    const int64_t own_old = (x + g.hx) + g.sx * (int64_t)(y + g.hy) + g.sxy * ((int64_t)z + g.hz + p.zo_read);
    T d[Q];
    d[0] = L.ld(0, own_old);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      // source x - c_i; z unwrapped (the ghost planes hold the periodic copy)
      int a = x - CX(i), b = y - CY(i), c = z - CZ(i);
      bool ok = wrap_axis(a, g.nx, g.px) && wrap_axis(b, g.ny, g.py);
      int cw = c;
      if (ok) ok = wrap_axis(cw, g.nz, g.pz);
      if (ok) ok = !grid_solid(g, a, b, cw);
      if (ok) {
        const int64_t src = (a + g.hx) + g.sx * (int64_t)(b + g.hy) + g.sxy * ((int64_t)c + g.hz + p.zo_read);
        d[i] = L.ld(i, src);
      } else {
        d[i] = L.ld(OPP(i), own_old);
      }
    }
    T drho, rjx;
    collide<T, FORCE>(d, T(p.omega), T(p.gx), T(p.gy), T(p.gz), drho, rjx);
    m += 1.0 + (double)drho;
    jsum += (double)rjx;
    const int64_t own_new = (x + g.hx) + g.sx * (int64_t)(y + g.hy) + g.sxy * ((int64_t)z + g.hz + p.zo_write);
#pragma unroll
    for (int i = 0; i < Q; ++i) L.st(i, own_new, d[i]);
  }
  if (RED) block_reduce_store(m, jsum, p.partials);
}

// Copy plane nz-1 to ghost plane -1 and plane 0 to ghost plane nz (offset zo),
// raw storage values, all 19 arrays.
template <class S, int AOS>
__global__ void k_cg_ghost(S *A, int64_t npad, Grid g, int zo) {
  const int64_t plane = g.sxy;  // storage slots per plane
  const int64_t total = 2 * plane * Q;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / (2 * plane));
    const int side = (int)((t / plane) & 1);
    const int64_t off = t % plane;
    const int64_t src_plane = side == 0 ? (g.nz - 1) : 0;
    const int64_t dst_plane = side == 0 ? -1 : g.nz;
    const int64_t src = off + g.sxy * (src_plane + g.hz + zo);
    const int64_t dst = off + g.sxy * (dst_plane + g.hz + zo);
    if (AOS)
      A[dst * Q + i] = A[src * Q + i];
    else
      A[(int64_t)i * npad + dst] = A[(int64_t)i * npad + src];
  }
}

template <class C, int AOS, bool IND, bool FORCE, bool RED>
struct LaunchCG {
  static void run(const StepParams &p, const LaunchShape &L) {
    k_cg_slab<C, AOS, false, FORCE, RED><<<L.grid, L.block, 0, L.stream>>>(p);
  }
};

void launch_cg_slab(const StepParams &p, const KernelKey &k, const LaunchShape &L) {
  dispatch<LaunchCG>(k.precision, k.aos, false, k.force, k.red, p, L);
}

void launch_cg_ghost(const StepParams &p, int precision, int aos, int zo, cudaStream_t s) {
  const int64_t plane = p.g.sxy;
  const int64_t total = 2 * plane * Q;
  const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, 1 << 20);
  if (precision == 0) {
    if (aos)
      k_cg_ghost<double, 1><<<grid, 256, 0, s>>>(static_cast<double *>(p.A), p.npad, p.g, zo);
    else
      k_cg_ghost<double, 0><<<grid, 256, 0, s>>>(static_cast<double *>(p.A), p.npad, p.g, zo);
  } else if (precision == 1) {
    if (aos)
      k_cg_ghost<float, 1><<<grid, 256, 0, s>>>(static_cast<float *>(p.A), p.npad, p.g, zo);
    else
      k_cg_ghost<float, 0><<<grid, 256, 0, s>>>(static_cast<float *>(p.A), p.npad, p.g, zo);
  } else {
    if (aos)
      k_cg_ghost<__half, 1><<<grid, 256, 0, s>>>(static_cast<__half *>(p.A), p.npad, p.g, zo);
    else
      k_cg_ghost<__half, 0><<<grid, 256, 0, s>>>(static_cast<__half *>(p.A), p.npad, p.g, zo);
  }
}

}  // namespace lbmk
