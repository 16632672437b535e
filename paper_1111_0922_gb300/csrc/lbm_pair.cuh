// AA pattern on a full grid with two x-adjacent nodes per thread.
//
// Each thread owns the pair (x0, x0 + 1), x0 even, of one row, so every PDF
// array is read and written with one aligned 2-element vector access per
// direction (half2 / float2 / double2): half the memory instructions of the
// one-node kernels and twice the bytes in flight per instruction.  The odd
// step's one-cell x shift is resolved inside the warp: a lane takes the
// element it needs from its neighbour lane's vector with a shuffle, and only
// the first and last active lane of a warp access the element beyond the
// warp's span with a scalar load or store.  Requirements (checked by the
// host): SoA, periodic x, even nx, no solid mask, no x halo.  Walls on y or z
// are allowed: a row beyond a wall is replaced by bounce-back for the whole
// warp.
#pragma once

#include "lbm_core.cuh"

namespace lbmk {

template <class S> struct Vec2;
template <> struct Vec2<double> { using V = double2; };
template <> struct Vec2<float> { using V = float2; };
template <> struct Vec2<__half> { using V = __half2; };

template <class C>
struct PairIO {
  using S = typename C::S;
  using T = typename C::T;
  using V = typename Vec2<S>::V;
  S *p;
  int64_t npad;
  float scale, inv_scale;
  __device__ __forceinline__ void ld2(int k, int64_t s0, T &a, T &b) const {
    const V v = *reinterpret_cast<const V *>(p + (int64_t)k * npad + s0);
    a = C::raw(v.x);
    b = C::raw(v.y);
  }
  __device__ __forceinline__ void st2(int k, int64_t s0, T a, T b) const {
    V v;
    v.x = C::unraw(a);
    v.y = C::unraw(b);
    *reinterpret_cast<V *>(p + (int64_t)k * npad + s0) = v;
  }
  __device__ __forceinline__ T ld1(int k, int64_t s) const { return C::raw(p[(int64_t)k * npad + s]); }
  __device__ __forceinline__ void st1(int k, int64_t s, T a) const { p[(int64_t)k * npad + s] = C::unraw(a); }
};

// Row geometry of one thread's pair.
struct PairRow {
  int x0, y, z;
  int s0;            // slot of (x0, y, z)
  int row0;          // slot of (0, y, z)
  int dy[2], dz[2];  // wrapped deltas to the -1 / +1 row and plane
  unsigned wall;     // bit 0/1: y -/+ face is a wall; bit 2/3: z -/+ face
  bool valid;        // the pair lies inside the box
  bool first, last;  // first / last valid lane of the warp

  // slot offset of the row reached by (ey, ez) in {-1, 0, 1}, or -1 if a wall
  __device__ __forceinline__ bool row_off(const Grid &g, int ey, int ez, int &off) const {
    if ((ey < 0 && (wall & 1u)) || (ey > 0 && (wall & 2u)) || (ez < 0 && (wall & 4u)) || (ez > 0 && (wall & 8u)))
      return false;
    const int yy = ey < 0 ? dy[0] : (ey > 0 ? dy[1] : 0);
    const int zz = ez < 0 ? dz[0] : (ez > 0 ? dz[1] : 0);
    off = (int)g.sx * yy + (int)g.sxy * zz;
    return true;
  }
};

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

template <class C, bool FORCE>
__device__ __forceinline__ void pair_collide(typename C::T (&d0)[Q], typename C::T (&d1)[Q], const StepParams &p,
                                             double &m, double &j) {
  using T = typename C::T;
  T r0, j0, r1, j1;
  collide_stored<C, FORCE>(d0, coll_of<T>(p), p.scale, p.inv_scale, r0, j0);
  collide_stored<C, FORCE>(d1, coll_of<T>(p), p.scale, p.inv_scale, r1, j1);
  m += 2.0 + (double)r0 + (double)r1;
  j += (double)j0 + (double)j1;
}

// Common set-up: returns false when the whole warp has nothing to do.
__device__ __forceinline__ bool pair_row(const StepParams &p, int z, PairRow &r) {
  const Grid &g = p.g;
  const int npairs = g.nx >> 1;
  const int px = blockIdx.x * blockDim.x + threadIdx.x;
  r.y = blockIdx.y * blockDim.y + threadIdx.y;
  r.z = z;
  r.x0 = 2 * px;
  r.valid = px < npairs && r.y < g.ny;
  // the warp shares y and z; its valid lanes are a prefix of the warp
  const unsigned active = __ballot_sync(0xffffffffu, r.valid);
  if (active == 0u) return false;
  const int lane = lane_id();
  r.first = lane == __ffs(active) - 1;
  r.last = lane == 31 - __clz(active);
  const int yy = r.y < g.ny ? r.y : 0;
  r.row0 = (int)g.sx * yy + (int)g.sxy * (z + g.zoff);
  r.s0 = r.row0 + r.x0;
  r.wall = 0;
  r.dy[0] = -1;
  r.dy[1] = 1;
  r.dz[0] = -1;
  r.dz[1] = 1;
  if (yy == 0) { if (g.py) r.dy[0] = g.ny - 1; else r.wall |= 1u; }
  if (yy == g.ny - 1) { if (g.py) r.dy[1] = 1 - g.ny; else r.wall |= 2u; }
  if (z == 0) { if (g.pz) r.dz[0] = g.nz - 1; else r.wall |= 4u; }
  if (z == g.nz - 1) { if (g.pz) r.dz[1] = 1 - g.nz; else r.wall |= 8u; }
  return true;
}

// Even step: node-local, reversed slots (Fig. 5a,b), two nodes per thread.
template <class C, bool FORCE, bool RED>
__global__ void __launch_bounds__(256, C::kMinBlocks) k_aa2_even(StepParams p) {
  using T = typename C::T;
  const PairIO<C> A{static_cast<typename C::S *>(p.A), p.npad, p.scale, p.inv_scale};
  double m = 0.0, j = 0.0;
  for (int z = blockIdx.z; z < p.g.nz; z += gridDim.z) {
    PairRow r;
    if (!pair_row(p, z, r)) continue;
    if (!r.valid) continue;
    T d0[Q], d1[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) A.ld2(i, r.s0, d0[i], d1[i]);
    pair_collide<C, FORCE>(d0, d1, p, m, j);
    const int s0 = launder(r.s0);
#pragma unroll
    for (int i = 0; i < Q; ++i) A.st2(OPP(i), s0, d0[i], d1[i]);
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

// Odd step (Fig. 5c,d), two nodes per thread.  Every lane of a warp with any
// valid pair runs the shuffles; lanes past the row end only pass values.
template <class C, bool FORCE, bool RED>
__global__ void __launch_bounds__(256, C::kMinBlocks) k_aa2_odd(StepParams p) {
  using T = typename C::T;
  const PairIO<C> A{static_cast<typename C::S *>(p.A), p.npad, p.scale, p.inv_scale};
  const int nx = p.g.nx;
  double m = 0.0, j = 0.0;
  for (int z = blockIdx.z; z < p.g.nz; z += gridDim.z) {
    PairRow r;
    if (!pair_row(p, z, r)) continue;
    const int xm = r.x0 == 0 ? nx - 1 : r.x0 - 1;       // x0 - 1, periodic
    const int xp = r.x0 + 2 == nx ? 0 : r.x0 + 2;       // x1 + 1, periodic
    T d0[Q], d1[Q];
    if (r.valid) A.ld2(0, r.s0, d0[0], d1[0]);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      // f_i(x) comes from slot opp(i) of x - c_i
      int off;
      const bool linked = r.row_off(p.g, -CY(i), -CZ(i), off);
      T a = T(0), b = T(0);
      if (!linked) {
        if (r.valid) A.ld2(i, r.s0, a, b);  // bounce-back: own slot i
      } else {
        if (r.valid) A.ld2(OPP(i), r.s0 + off, a, b);
        if (CX(i) == 1) {  // from x - 1: (prev lane's second, own first)
          const T up = __shfl_up_sync(0xffffffffu, b, 1);
          const T own_first = a;
          a = up;
          b = own_first;
          if (r.first && r.valid) a = A.ld1(OPP(i), r.row0 + off + xm);
        } else if (CX(i) == -1) {  // from x + 1: (own second, next lane's first)
          const T down = __shfl_down_sync(0xffffffffu, a, 1);
          a = b;
          b = down;
          if (r.last && r.valid) b = A.ld1(OPP(i), r.row0 + off + xp);
        }
      }
      d0[i] = a;
      d1[i] = b;
    }
    if (r.valid) pair_collide<C, FORCE>(d0, d1, p, m, j);
    const int s0 = launder(r.s0);
    const int row0 = launder(r.row0);
    if (r.valid) A.st2(0, s0, d0[0], d1[0]);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      // g_i(x) goes to slot i of x + c_i
      int off;
      const bool linked = r.row_off(p.g, CY(i), CZ(i), off);
      if (!linked) {
        if (r.valid) A.st2(OPP(i), s0, d0[i], d1[i]);  // bounce-back: own slot opp(i)
        continue;
      }
      if (CX(i) == 0) {
        if (r.valid) A.st2(i, s0 + off, d0[i], d1[i]);
      } else if (CX(i) == 1) {
        // slots (x0, x1) of the target row take (prev lane's g(x1), own g(x0))
        const T up = __shfl_up_sync(0xffffffffu, d1[i], 1);
        if (r.valid) {
          if (!r.first)
            A.st2(i, s0 + off, up, d0[i]);
          else
            A.st1(i, row0 + off + r.x0 + 1, d0[i]);
          if (r.last) A.st1(i, row0 + off + xp, d1[i]);
        }
      } else {
        // slots (x0, x1) take (own g(x1), next lane's g(x0))
        const T down = __shfl_down_sync(0xffffffffu, d0[i], 1);
        if (r.valid) {
          if (!r.last)
            A.st2(i, s0 + off, d1[i], down);
          else
            A.st1(i, row0 + off + r.x0, d1[i]);
          if (r.first) A.st1(i, row0 + off + xm, d0[i]);
        }
      }
    }
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

}  // namespace lbmk
