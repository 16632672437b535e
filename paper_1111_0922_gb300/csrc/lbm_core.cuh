// Device-side core of the D3Q19 step: lattice constants, storage codecs,
// PDF layouts, neighbour rules and the BGK + Guo collision in shifted form.
//
// Paper: Wittmann, Zeiser, Hager, Wellein, "Comparison of different
// Propagation Steps for the Lattice Boltzmann Method" (D3Q19, Sec. 1; SoA and
// AoS layouts, Sec. 1; full-grid and IDX addressing, Sec. 1).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmk {

constexpr int Q = 19;

// Velocity set: 0 rest, 1..6 axes (+x -x +y -y +z -z), 7..18 diagonals in
// opposite pairs.  Odd i and i+1 are opposite.
__host__ __device__ constexpr int CX(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int CY(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int CZ(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int OPP(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr double WD(int i) {
  return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// ---------------------------------------------------------------------------
// Storage codecs.  Every precision stores the deviation d_i = f_i - w_i
// (rho0 = 1).  F16S stores round(d_i * S) with a power-of-two S, so decoding
// is exact and only the final rounding to FP16 loses precision.
struct CodecF64 {
  using S = double;  // stored
  using T = double;  // computed
  __device__ static __forceinline__ T dec(S v, float) { return v; }
  __device__ static __forceinline__ S enc(T v, float) { return v; }
};
struct CodecF32 {
  using S = float;
  using T = float;
  __device__ static __forceinline__ T dec(S v, float) { return v; }
  __device__ static __forceinline__ S enc(T v, float) { return v; }
};
struct CodecF16S {
  using S = __half;
  using T = float;
  __device__ static __forceinline__ T dec(S v, float inv_scale) { return __half2float(v) * inv_scale; }
  __device__ static __forceinline__ S enc(T v, float scale) { return __float2half_rn(v * scale); }
};

// ---------------------------------------------------------------------------
// PDF layouts.  SoA: array k holds slot s at k * npad + s (each array starts
// on a 256-byte boundary).  AoS: the 19 PDFs of slot s are contiguous.
template <class C, int AOS>
struct Lattice {
  typename C::S *p;
  int64_t npad;
  float scale, inv_scale;
  __device__ __forceinline__ typename C::S *at(int k, int64_t s) const {
    return AOS ? p + s * Q + k : p + (int64_t)k * npad + s;
  }
  __device__ __forceinline__ typename C::T ld(int k, int64_t s) const { return C::dec(*at(k, s), inv_scale); }
  __device__ __forceinline__ void st(int k, int64_t s, typename C::T v) const { *at(k, s) = C::enc(v, scale); }
};

// ---------------------------------------------------------------------------
// Geometry of a full grid in storage: cell (x, y, z) lives at storage slot
// (x + hx) + sx * (y + hy) + sxy * (z + hz + zoff); halos (h = 1) give ghost
// slots one cell beyond non-periodic faces, zoff shifts whole planes
// (compressed grid).
struct Grid {
  int nx, ny, nz;
  int px, py, pz;  // periodic flags
  int hx, hy, hz;
  int64_t sx, sxy;
  int64_t zoff;
  const uint8_t *solid;  // per cell, or nullptr when every cell is fluid
};

__device__ __forceinline__ int64_t grid_slot(const Grid &g, int x, int y, int z) {
  return (int64_t)(x + g.hx) + g.sx * (int64_t)(y + g.hy) + g.sxy * ((int64_t)z + g.hz + g.zoff);
}

__device__ __forceinline__ bool grid_solid(const Grid &g, int x, int y, int z) {
  return g.solid != nullptr && g.solid[(int64_t)x + (int64_t)g.nx * ((int64_t)y + (int64_t)g.ny * z)] != 0;
}

// Wrap one coordinate; false if it leaves a non-periodic axis.
__device__ __forceinline__ bool wrap_axis(int &v, int n, int periodic) {
  if (v < 0) {
    if (!periodic) return false;
    v += n;
  } else if (v >= n) {
    if (!periodic) return false;
    v -= n;
  }
  return true;
}

// Storage slot of the fluid neighbour (x,y,z) + (dx,dy,dz), or -1 for a wall
// or solid link.
__device__ __forceinline__ int64_t grid_neighbour(const Grid &g, int x, int y, int z, int dx, int dy, int dz) {
  int a = x + dx, b = y + dy, c = z + dz;
  if (!wrap_axis(a, g.nx, g.px) || !wrap_axis(b, g.ny, g.py) || !wrap_axis(c, g.nz, g.pz)) return -1;
  if (grid_solid(g, a, b, c)) return -1;
  return grid_slot(g, a, b, c);
}

// Storage slot of the position (x,y,z) + (dx,dy,dz) whether fluid or not:
// wrapped on periodic axes, in the halo beyond a wall (the esoteric twist's
// ghost slots).
__device__ __forceinline__ int64_t grid_position(const Grid &g, int x, int y, int z, int dx, int dy, int dz) {
  int a = x + dx, b = y + dy, c = z + dz;
  if (g.px) wrap_axis(a, g.nx, 1);
  if (g.py) wrap_axis(b, g.ny, 1);
  if (g.pz) wrap_axis(c, g.nz, 1);
  return grid_slot(g, a, b, c);
}

// ---------------------------------------------------------------------------
// BGK collision with the Guo forcing term, in shifted variables.
//   d_i = f_i - w_i,  rho = 1 + sum d_i,  j = sum c_i d_i  (sum c_i w_i = 0)
//   u = (j + rho g / 2) / rho
//   d_eq,i = w_i [ (rho - 1) + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u.u) ]
//   F_i    = (1 - omega/2) w_i rho [ 3 (c_i - u).g + 9 (c_i.u)(c_i.g) ]
//   d*_i   = d_i - omega (d_i - d_eq,i) + F_i
// Opposite pairs share c.u up to sign, which the pair loop exploits.
// Returns rho - 1 and rho u_x (for the mass and flux reductions).
template <typename T, bool FORCE>
__device__ __forceinline__ void collide(T (&d)[Q], T omega, T gx, T gy, T gz, T &drho_out, T &rjx_out) {
  T sum[10], dif[10];
#pragma unroll
  for (int k = 1; k <= 9; ++k) {
    sum[k] = d[2 * k - 1] + d[2 * k];
    dif[k] = d[2 * k - 1] - d[2 * k];
  }
  const T drho = d[0] + (((sum[1] + sum[2]) + (sum[3] + sum[4])) + ((sum[5] + sum[6]) + (sum[7] + sum[8])) + sum[9]);
  // pair k = (2k-1, 2k); velocity of the odd member
  T jx = 0, jy = 0, jz = 0;
#pragma unroll
  for (int k = 1; k <= 9; ++k) {
    const int i = 2 * k - 1;
    if (CX(i) == 1) jx += dif[k];
    if (CX(i) == -1) jx -= dif[k];
    if (CY(i) == 1) jy += dif[k];
    if (CY(i) == -1) jy -= dif[k];
    if (CZ(i) == 1) jz += dif[k];
    if (CZ(i) == -1) jz -= dif[k];
  }
  const T rho = T(1) + drho;
  const T inv = T(1) / rho;
  T ux, uy, uz;
  if (FORCE) {
    const T hr = T(0.5) * rho;
    ux = (jx + hr * gx) * inv;
    uy = (jy + hr * gy) * inv;
    uz = (jz + hr * gz) * inv;
  } else {
    ux = jx * inv;
    uy = jy * inv;
    uz = jz * inv;
  }
  drho_out = drho;
  rjx_out = rho * ux;
  const T usq15 = T(1.5) * (ux * ux + uy * uy + uz * uz);
  const T om1 = T(1) - omega;
  const T kf = T(1) - T(0.5) * omega;
  T ug = 0;
  if (FORCE) ug = ux * gx + uy * gy + uz * gz;
  {
    const T w = T(WD(0));
    T deq = w * (drho - rho * usq15);
    T v = om1 * d[0] + omega * deq;
    if (FORCE) v -= kf * w * rho * T(3) * ug;
    d[0] = v;
  }
#pragma unroll
  for (int k = 1; k <= 9; ++k) {
    const int i = 2 * k - 1;
    const T w = T(WD(i));
    T cu = 0, cg = 0;
    if (CX(i)) { cu += T(CX(i)) * ux; if (FORCE) cg += T(CX(i)) * gx; }
    if (CY(i)) { cu += T(CY(i)) * uy; if (FORCE) cg += T(CY(i)) * gy; }
    if (CZ(i)) { cu += T(CZ(i)) * uz; if (FORCE) cg += T(CZ(i)) * gz; }
    const T sym = drho + rho * (T(4.5) * cu * cu - usq15);
    const T asym = T(3) * rho * cu;
    T vp = om1 * d[i] + omega * w * (sym + asym);
    T vm = om1 * d[i + 1] + omega * w * (sym - asym);
    if (FORCE) {
      const T fs = kf * w * rho * (T(9) * cu * cg - T(3) * ug);
      const T fa = kf * w * rho * T(3) * cg;
      vp += fs + fa;
      vm += fs - fa;
    }
    d[i] = vp;
    d[i + 1] = vm;
  }
}

// ---------------------------------------------------------------------------
// Kernel parameters shared by every step kernel (passed by value).  Storage
// slots are int32 (a handle holds fewer than 2^31 slots per PDF array).
struct StepParams {
  void *A;            // lattice read (and, for one-lattice schemes, written)
  void *B;            // second lattice (TS, OS)
  int64_t npad;       // SoA stride in slots
  int64_t nnodes;     // nodes the launch iterates over (direct: cells)
  int64_t nfluid;     // fluid nodes (indirect ghost threshold)
  Grid g;             // direct addressing
  const int32_t *idx; // indirect: IDX (18 x ipad) or the esoteric twist's packed 9 x ipad
  int64_t ipad;
  int map[Q];         // esoteric twist: physical array of direction i
  double omega, gx, gy, gz;
  float scale, inv_scale;
  double *partials;   // fused reduction: 2 doubles per block, or nullptr
  int *err;           // device error word
  int z0, z1;         // compressed grid: planes of this launch
  int zo_read, zo_write;  // compressed grid: plane offsets of the old and new state
};

// Per-thread node context for full-grid addressing.
struct DirectNode {
  int x, y, z;
  int s;
  __device__ __forceinline__ bool init(const StepParams &p, int64_t n) {
    const Grid &g = p.g;
    x = (int)(n % g.nx);
    int64_t r = n / g.nx;
    y = (int)(r % g.ny);
    z = (int)(r / g.ny);
    if (grid_solid(g, x, y, z)) return false;
    s = (int)grid_slot(g, x, y, z);
    return true;
  }
  // slot of the fluid neighbour along c_i, or -1
  __device__ __forceinline__ int nb(const StepParams &p, int i) const {
    return (int)grid_neighbour(p.g, x, y, z, CX(i), CY(i), CZ(i));
  }
};

// Per-thread node context for IDX addressing.
struct IndirectNode {
  int s;
  __device__ __forceinline__ bool init(const StepParams &, int64_t n) {
    s = (int)n;
    return true;
  }
  __device__ __forceinline__ int nb(const StepParams &p, int i) const {
    return __ldg(p.idx + (int64_t)(i - 1) * p.ipad + s);
  }
};

// ---------------------------------------------------------------------------
// Block reduction of (mass, flux) into per-block FP64 partials.
__device__ __forceinline__ void block_reduce_store(double m, double j, double *partials) {
  __shared__ double sm[32], sj[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m += __shfl_xor_sync(0xffffffffu, m, o);
    j += __shfl_xor_sync(0xffffffffu, j, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sm[warp] = m;
    sj[warp] = j;
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    m = lane < nw ? sm[lane] : 0.0;
    j = lane < nw ? sj[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      m += __shfl_xor_sync(0xffffffffu, m, o);
      j += __shfl_xor_sync(0xffffffffu, j, o);
    }
    if (lane == 0) {
      partials[2 * blockIdx.x] = m;
      partials[2 * blockIdx.x + 1] = j;
    }
  }
}

}  // namespace lbmk
