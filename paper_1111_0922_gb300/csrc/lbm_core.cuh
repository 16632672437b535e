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
//   raw / unraw: stored value <-> compute type without the scale; the step
//                kernels work on S * d_i throughout (the collision takes S,
//                so no per-PDF multiply is spent on the scale).
//   dec / enc:   stored value <-> d_i (state upload, read-out, reductions).
// kMinBlocks: resident 256-thread blocks per SM the step kernels are built
// for (a register budget: 2 -> 128, 3 -> 85 registers per thread).
struct CodecF64 {
  using S = double;  // stored
  using T = double;  // computed
  static constexpr int kMinBlocks = 2;
  static constexpr bool kScaled = false;
  __device__ static __forceinline__ T raw(S v) { return v; }
  __device__ static __forceinline__ S unraw(T v) { return v; }
  __device__ static __forceinline__ T dec(S v, float) { return v; }
  __device__ static __forceinline__ S enc(T v, float) { return v; }
};
struct CodecF32 {
  using S = float;
  using T = float;
  static constexpr int kMinBlocks = 3;
  static constexpr bool kScaled = false;
  __device__ static __forceinline__ T raw(S v) { return v; }
  __device__ static __forceinline__ S unraw(T v) { return v; }
  __device__ static __forceinline__ T dec(S v, float) { return v; }
  __device__ static __forceinline__ S enc(T v, float) { return v; }
};
struct CodecF16S {
  using S = __half;
  using T = float;
  static constexpr int kMinBlocks = 3;
  static constexpr bool kScaled = true;
  __device__ static __forceinline__ T raw(S v) { return __half2float(v); }
  __device__ static __forceinline__ S unraw(T v) { return __float2half_rn(v); }
  __device__ static __forceinline__ T dec(S v, float inv_scale) { return __half2float(v) * inv_scale; }
  __device__ static __forceinline__ S enc(T v, float scale) { return __float2half_rn(v * scale); }
};

// ---------------------------------------------------------------------------
// PDF layouts.  SoA: array k holds slot s at k * npad + s (each array starts
// on a 256-byte boundary).  AoS: the 19 PDFs of slot s are contiguous.
// CS: stores use the cache-streaming policy (st.global.cs, evict-first), the
// GPU counterpart of the non-temporal stores of the paper's OS-NT (Sec. 3).
template <class C, int AOS, bool CS = false>
struct Lattice {
  typename C::S *p;
  int64_t npad;
  float scale, inv_scale;
  __device__ __forceinline__ typename C::S *at(int k, int64_t s) const {
    return AOS ? p + s * Q + k : p + (int64_t)k * npad + s;
  }
  // step kernels: values in the collision's units (S * d_i for F16S)
  __device__ __forceinline__ typename C::T ld(int k, int64_t s) const { return C::raw(*at(k, s)); }
  __device__ __forceinline__ void st(int k, int64_t s, typename C::T v) const {
    if constexpr (CS)
      __stcs(at(k, s), C::unraw(v));
    else
      *at(k, s) = C::unraw(v);
  }
  // state upload and read-out: the deviation d_i itself
  __device__ __forceinline__ typename C::T ld_dev(int k, int64_t s) const { return C::dec(*at(k, s), inv_scale); }
  __device__ __forceinline__ void st_dev(int k, int64_t s, typename C::T v) const { *at(k, s) = C::enc(v, scale); }
};

// Word of a cell pair (two cells of a full grid, or two consecutive nodes of
// a node list): both cells' storage in one aligned word (FP16: the lower
// cell in the low half; FP32: in .x).  kMinBlocks: resident 256-thread
// blocks per SM of the pair kernels (FP32 pairs hold both cells' 38 values,
// so they get 128 registers; measured faster than 80 with spills).
template <class C>
struct PairWord;
template <>
struct PairWord<CodecF16S> {
  using W = __half2;
  static constexpr int kMinBlocks = 3;
  __device__ static __forceinline__ float lo(W v) { return CodecF16S::raw(__low2half(v)); }
  __device__ static __forceinline__ float hi(W v) { return CodecF16S::raw(__high2half(v)); }
  __device__ static __forceinline__ W with_lo(W v, float a) { return __halves2half2(CodecF16S::unraw(a), __high2half(v)); }
  __device__ static __forceinline__ W with_hi(W v, float b) { return __halves2half2(__low2half(v), CodecF16S::unraw(b)); }
  __device__ static __forceinline__ W swap(W v) { return __lowhigh2highlow(v); }
  // raw storage elements of the two cells
  __device__ static __forceinline__ W pack(__half a, __half b) { return __halves2half2(a, b); }
  __device__ static __forceinline__ __half lo_s(W v) { return __low2half(v); }
  __device__ static __forceinline__ __half hi_s(W v) { return __high2half(v); }
};
template <>
struct PairWord<CodecF32> {
  using W = float2;
  static constexpr int kMinBlocks = 2;
  __device__ static __forceinline__ float lo(W v) { return v.x; }
  __device__ static __forceinline__ float hi(W v) { return v.y; }
  __device__ static __forceinline__ W with_lo(W v, float a) { return make_float2(a, v.y); }
  __device__ static __forceinline__ W with_hi(W v, float b) { return make_float2(v.x, b); }
  __device__ static __forceinline__ W swap(W v) { return make_float2(v.y, v.x); }
  __device__ static __forceinline__ W pack(float a, float b) { return make_float2(a, b); }
  __device__ static __forceinline__ float lo_s(W v) { return v.x; }
  __device__ static __forceinline__ float hi_s(W v) { return v.y; }
};
template <class C>
constexpr bool kPairable = std::is_same<C, CodecF16S>::value || std::is_same<C, CodecF32>::value;

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
  int zghost;            // periodic z through ghost planes (compressed grid):
                         // z deltas stay +-1, only the solid lookup wraps
  int zpair;             // z pairs (FP16 / FP32 storage, no halo): cells z
                         // and z + nz/2 share word (x, y, z mod nz/2), low
                         // and high half; sx, sxy count words
  int ypair;             // y pairs (compressed grid, FP16 / FP32, no x or y
                         // halo): cells y and y + ny/2 share word
                         // (x, y mod ny/2, z); sx counts words, a plane is
                         // sxy / 2 words
};

__device__ __forceinline__ int64_t grid_slot(const Grid &g, int x, int y, int z) {
  if (g.zpair) {
    const int H = g.nz >> 1, hi = z >= H ? 1 : 0;
    return 2 * ((int64_t)x + g.sx * (int64_t)y + g.sxy * (int64_t)(z - hi * H)) + hi;
  }
  if (g.ypair) {
    const int H = g.ny >> 1, hi = y >= H ? 1 : 0;
    return 2 * ((int64_t)x + g.sx * (int64_t)(y - hi * H) + (g.sxy >> 1) * ((int64_t)z + g.hz + g.zoff)) + hi;
  }
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
// Collision with the Guo forcing term, in shifted variables: two-relaxation-
// time (TRT) with rates lp (symmetric halves, sets the viscosity) and lm
// (antisymmetric halves); lm = lp is BGK.
//   d_i = f_i - w_i,  rho = 1 + sum d_i,  j = sum c_i d_i  (sum c_i w_i = 0)
//   u = (j + rho g / 2) / rho
//   for an opposite pair (i, opp i), with a = (d_i + d_opp)/2, b = (d_i - d_opp)/2:
//     a_eq = w_i [ (rho - 1) + rho (4.5 (c.u)^2 - 1.5 u.u) ],  b_eq = w_i 3 rho c.u
//     F+ = (1 - lp/2) w_i rho (9 (c.u)(c.g) - 3 u.g),  F- = (1 - lm/2) w_i rho 3 c.g
//     a* = a - lp (a - a_eq) + F+,  b* = b - lm (b - b_eq) + F-
//     d*_i = a* + b*,  d*_opp = a* - b*
//   rest: d*_0 = d_0 - lp (d_0 - w_0 [(rho - 1) - 1.5 rho u.u]) - (1 - lp/2) w_0 rho 3 u.g
//
// Evaluated with the terms regrouped so that each opposite pair costs six to
// ten operations, with A = lp (rho - 1) - rho (1.5 lp u.u + 3 (1 - lp/2) u.g):
//   a* = (1 - lp)/2 (d_i + d_opp) + w_i A + rho (c.u) (4.5 lp w_i c.u + 9 (1 - lp/2) w_i c.g)
//   b* = (1 - lm)/2 (d_i - d_opp) + rho (3 lm w_i c.u + 3 (1 - lm/2) w_i c.g)
//   d*_0 = (1 - lp) d_0 + w_0 A
// collide_f32 forms u; collide_f64 never does: with J = rho u and sc = c.J,
// rho u.u = J.J / rho, rho u.g = J.g and rho (c.u)^2 = sc^2 / rho, so one
// reciprocal of rho serves every pair and c.J costs additions alone; its
// moments come from direction-group sums.  For BGK d*_i = (1 - lp) d_i +
// (P +- M) with P +- M formed in one chain per member (below), which keeps
// lp = 0 (no collision) an exact identity.
//
// With SCALED the d_i arrive multiplied by the storage scale s (a power of
// two, S for F16S) and leave multiplied by it; the moments are unscaled
// exactly with inv_s.  Without it s and inv_s are ignored.  Returns rho - 1 and rho u_x (for the mass and flux reductions).
// Rounded arithmetic that the compiler may neither contract nor reorder: a
// node's collision then gives the same bits in every kernel it is inlined
// into (one node per thread or several, any block shape), which keeps a
// geometry's solve bit-identical alone and inside a batch.  Host code (the
// per-launch constants) uses plain operators.
template <typename T>
struct Rn;
template <>
struct Rn<float> {
#ifdef __CUDA_ARCH__
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#else
  static float add(float a, float b) { return a + b; }
  static float sub(float a, float b) { return a - b; }
  static float mul(float a, float b) { return a * b; }
  static float fma(float a, float b, float c) { return a * b + c; }
#endif
};
template <>
struct Rn<double> {
#ifdef __CUDA_ARCH__
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
#else
  static double add(double a, double b) { return a + b; }
  static double sub(double a, double b) { return a - b; }
  static double mul(double a, double b) { return a * b; }
  static double fma(double a, double b, double c) { return a * b + c; }
#endif
};

// Per-launch constants of the collision, uniform over the nodes: filled once
// on the host for a lattice's launches (kernel parameters, read by the node
// arithmetic as constant operands), or per thread for a batch segment.
template <typename T>
struct CollK {
  T lp, om1;         // symmetric rate, 1 - lp
  T al, be;          // TRT: (1 - lp)/2 + (1 - lm)/2, (1 - lp)/2 - (1 - lm)/2
  T q15, q3;         // 1.5 lp, 3 (1 - lp/2)
  T tp[2], tm[2];    // 4.5 lp w, 3 lm w for w = 1/18, 1/36
  T fp[10], fm[10];  // pair k (odd member 2k-1): 9 (1 - lp/2) w c.g, 3 (1 - lm/2) w c.g
  T zp[10], zm[10];  // fp_k + tm_c, fp_k - tm_c (c the weight class of pair k)
  T hg[3], g[3];     // g/2, g
  int bgk;           // lm == lp
  int gx_only;       // g = (gx, 0, 0): the FP64 collision drops the zero force terms
};

template <typename T>
__host__ __device__ inline CollK<T> make_collk(T lp, T lm, T gx, T gy, T gz) {
  using R = Rn<T>;
  CollK<T> K;
  const T kp = R::fma(T(-0.5), lp, T(1)), km = R::fma(T(-0.5), lm, T(1));
  K.lp = lp;
  K.om1 = R::sub(T(1), lp);
  const T hp = R::mul(T(0.5), R::sub(T(1), lp)), hm = R::mul(T(0.5), R::sub(T(1), lm));
  K.al = R::add(hp, hm);
  K.be = R::sub(hp, hm);
  K.q15 = R::mul(T(1.5), lp);
  K.q3 = R::mul(T(3), kp);
  const T w[2] = {T(1) / T(18), T(1) / T(36)};
  for (int c = 0; c < 2; ++c) {
    K.tp[c] = R::mul(R::mul(T(4.5), lp), w[c]);
    K.tm[c] = R::mul(R::mul(T(3), lm), w[c]);
  }
  K.fp[0] = K.fm[0] = K.zp[0] = K.zm[0] = T(0);
  for (int k = 1; k <= 9; ++k) {
    const int i = 2 * k - 1;
    const T cg = R::add(R::add(R::mul(T(CX(i)), gx), R::mul(T(CY(i)), gy)), R::mul(T(CZ(i)), gz));
    const T wi = i <= 6 ? w[0] : w[1];
    K.fp[k] = R::mul(R::mul(R::mul(T(9), kp), wi), cg);
    K.fm[k] = R::mul(R::mul(R::mul(T(3), km), wi), cg);
    K.zp[k] = R::add(K.fp[k], K.tm[i <= 6 ? 0 : 1]);
    K.zm[k] = R::sub(K.fp[k], K.tm[i <= 6 ? 0 : 1]);
  }
  K.g[0] = gx;
  K.g[1] = gy;
  K.g[2] = gz;
  for (int a = 0; a < 3; ++a) K.hg[a] = R::mul(T(0.5), K.g[a]);
  K.bgk = lm == lp;
  K.gx_only = gy == T(0) && gz == T(0);
  return K;
}

template <typename T>
__device__ __forceinline__ T recip(T x);
template <>
__device__ __forceinline__ float recip<float>(float x) {
  return __fdividef(1.0f, x);  // rho is near 1: the fast reciprocal is well within FP32 parity
}
// FP64: Newton-Raphson iteration for 1/x (Newton's method on g(r) = 1/r - x:
// r <- r + r (1 - x r), which squares the relative error of r), started from
// the hardware's approximate reciprocal (rcp.approx.ftz.f64, accurate to
// about 20 bits; two steps take the error below 2^-70 before the final
// rounding, so the result is within one unit in the last place of 1/x).
// Four FMAs instead of the correctly rounded division's longer sequence and
// range checks: the FP64 pipe bounds every FP64 step kernel on GB300.
template <>
__device__ __forceinline__ double recip<double>(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = __fma_rn(-x, r, 1.0);
  r = __fma_rn(r, e, r);
  e = __fma_rn(-x, r, 1.0);
  return __fma_rn(r, e, r);
}

// Sum of the five d_i with i in {a, b, c, e, f}, as a fixed tree.
template <typename T>
__device__ __forceinline__ T sum5(const T (&d)[Q], int a, int b, int c, int e, int f) {
  using R = Rn<T>;
  return R::add(R::add(R::add(d[a], d[b]), R::add(d[c], d[e])), d[f]);
}

template <typename T, bool FORCE, bool SCALED>
__device__ __forceinline__ void collide_f32(T (&d)[Q], const CollK<T> &K, T s, T inv_s, T &drho_out, T &rjx_out) {
  using R = Rn<T>;
  T sum[10], dif[10];
#pragma unroll
  for (int k = 1; k <= 9; ++k) {
    sum[k] = R::add(d[2 * k - 1], d[2 * k]);
    dif[k] = R::sub(d[2 * k - 1], d[2 * k]);
  }
  const T sdrho = R::add(d[0], R::add(R::add(R::add(R::add(sum[1], sum[2]), R::add(sum[3], sum[4])),
                                             R::add(R::add(sum[5], sum[6]), R::add(sum[7], sum[8]))),
                                      sum[9]));
  // j = sum over pairs of c_(2k-1) (d_(2k-1) - d_(2k)), in ascending k
  T jx = 0, jy = 0, jz = 0;
  bool fx = true, fy = true, fz = true;
#pragma unroll
  for (int k = 1; k <= 9; ++k) {
    const int i = 2 * k - 1;
    if (CX(i)) { jx = fx ? (CX(i) > 0 ? dif[k] : -dif[k]) : (CX(i) > 0 ? R::add(jx, dif[k]) : R::sub(jx, dif[k])); fx = false; }
    if (CY(i)) { jy = fy ? (CY(i) > 0 ? dif[k] : -dif[k]) : (CY(i) > 0 ? R::add(jy, dif[k]) : R::sub(jy, dif[k])); fy = false; }
    if (CZ(i)) { jz = fz ? (CZ(i) > 0 ? dif[k] : -dif[k]) : (CZ(i) > 0 ? R::add(jz, dif[k]) : R::sub(jz, dif[k])); fz = false; }
  }
  const T drho = SCALED ? R::mul(sdrho, inv_s) : sdrho;
  if (SCALED) {
    jx = R::mul(jx, inv_s);
    jy = R::mul(jy, inv_s);
    jz = R::mul(jz, inv_s);
  }
  const T rho = R::add(T(1), drho);
  const T inv = recip(rho);
  T ux, uy, uz;
  if (FORCE) {
    ux = R::mul(R::fma(rho, K.hg[0], jx), inv);
    uy = R::mul(R::fma(rho, K.hg[1], jy), inv);
    uz = R::mul(R::fma(rho, K.hg[2], jz), inv);
  } else {
    ux = R::mul(jx, inv);
    uy = R::mul(jy, inv);
    uz = R::mul(jz, inv);
  }
  drho_out = drho;
  rjx_out = R::mul(rho, ux);
  T q = R::mul(K.q15, R::fma(uz, uz, R::fma(uy, uy, R::mul(ux, ux))));
  if (FORCE) q = R::fma(K.q3, R::fma(uz, K.g[2], R::fma(uy, K.g[1], R::mul(ux, K.g[0]))), q);
  const T srho = SCALED ? R::mul(s, rho) : rho;
  const T sA = R::fma(-srho, q, R::mul(K.lp, sdrho));  // s * A
  d[0] = R::fma(K.om1, d[0], R::mul(T(WD(0)), sA));
  const T wsA[2] = {R::mul(T(WD(1)), sA), R::mul(T(WD(7)), sA)};
  // For pair k with P = s (w A + rho (c.u)(tp_c c.u + fp_k)) and
  // M = s rho (tm_c c.u + fm_k), the two sums are formed directly:
  //   P +- M = wsA + s rho [ (c.u) (tp_c c.u + (fp_k +- tm_c)) +- fm_k ]
  // (without a force: wsA + (s rho c.u)(tp_c c.u +- tm_c)).
  auto terms = [&](int k, T &Pp, T &Pm) {
    const int i = 2 * k - 1;
    const int c = i <= 6 ? 0 : 1;
    T cu = 0;
    bool first = true;
    if (CX(i)) { cu = CX(i) > 0 ? ux : -ux; first = false; }
    if (CY(i)) { cu = first ? (CY(i) > 0 ? uy : -uy) : (CY(i) > 0 ? R::add(cu, uy) : R::sub(cu, uy)); first = false; }
    if (CZ(i)) { cu = first ? (CZ(i) > 0 ? uz : -uz) : (CZ(i) > 0 ? R::add(cu, uz) : R::sub(cu, uz)); }
    if (FORCE) {
      const T yp = R::fma(cu, R::fma(K.tp[c], cu, K.zp[k]), K.fm[k]);
      const T ym = R::fma(cu, R::fma(K.tp[c], cu, K.zm[k]), -K.fm[k]);
      Pp = R::fma(srho, yp, wsA[c]);
      Pm = R::fma(srho, ym, wsA[c]);
    } else {
      const T sc = R::mul(srho, cu);
      Pp = R::fma(sc, R::fma(K.tp[c], cu, K.tm[c]), wsA[c]);
      Pm = R::fma(sc, R::fma(K.tp[c], cu, -K.tm[c]), wsA[c]);
    }
  };
  if (K.bgk) {
#pragma unroll
    for (int k = 1; k <= 9; ++k) {
      const int i = 2 * k - 1;
      T Pp, Pm;
      terms(k, Pp, Pm);
      d[i] = R::fma(K.om1, d[i], Pp);
      d[i + 1] = R::fma(K.om1, d[i + 1], Pm);
    }
  } else {
    // a* +- b* with a = (d_i + d_opp)/2, b = (d_i - d_opp)/2 expanded, so
    // that only d_i and d_opp stay live:
    //   d*_i = al d_i + be d_opp + (P + M),  d*_opp = be d_i + al d_opp + (P - M)
#pragma unroll
    for (int k = 1; k <= 9; ++k) {
      const int i = 2 * k - 1;
      T Pp, Pm;
      terms(k, Pp, Pm);
      const T di = d[i], dj = d[i + 1];
      d[i] = R::fma(K.al, di, R::fma(K.be, dj, Pp));
      d[i + 1] = R::fma(K.al, dj, R::fma(K.be, di, Pm));
    }
  }
}

// FM: 0 no force, 1 force along x only (the zero terms of the other axes
// dropped at compile time), 2 any force.
template <typename T, int FM, bool SCALED>
__device__ __forceinline__ void collide_f64_body(T (&d)[Q], const CollK<T> &K, T s, T inv_s, T &drho_out, T &rjx_out) {
  using R = Rn<T>;
  // Moments from direction groups: P_a / M_a sum the d_i with c_ia = +1 / -1,
  // j_a = P_a - M_a, rho - 1 = P_x + M_x + (the nine d_i with c_ix = 0).
  // 37 additions for the four moments.
  const T px = sum5(d, 1, 7, 9, 11, 13), mx = sum5(d, 2, 8, 10, 12, 14);
  const T py = sum5(d, 3, 7, 10, 15, 17), my = sum5(d, 4, 8, 9, 16, 18);
  const T pz = sum5(d, 5, 11, 14, 15, 18), mz = sum5(d, 6, 12, 13, 16, 17);
  const T x0 = R::add(R::add(R::add(R::add(d[3], d[4]), R::add(d[5], d[6])),
                             R::add(R::add(d[15], d[16]), R::add(d[17], d[18]))),
                      d[0]);
  const T sdrho = R::add(R::add(px, mx), x0);
  const T sjx = R::sub(px, mx), sjy = R::sub(py, my), sjz = R::sub(pz, mz);
  const T drho = SCALED ? R::mul(sdrho, inv_s) : sdrho;
  const T rho = R::add(T(1), drho);
  const T srho = SCALED ? R::mul(s, rho) : rho;
  // J = j + rho g / 2 = rho u, kept in the stored units (s J)
  constexpr bool FORCE = FM != 0;
  T sJx = sjx, sJy = sjy, sJz = sjz;
  if (FORCE) sJx = R::fma(srho, K.hg[0], sjx);
  if (FM == 2) {
    sJy = R::fma(srho, K.hg[1], sjy);
    sJz = R::fma(srho, K.hg[2], sjz);
  }
  const T inv = SCALED ? R::mul(recip(rho), inv_s) : recip(rho);  // 1 / (s rho)
  drho_out = drho;
  rjx_out = SCALED ? R::mul(sJx, inv_s) : sJx;
  // The velocity itself is never formed: with u = sJ / (s rho),
  //   s rho u.u = |sJ|^2 inv,  s rho u.g = sJ.g,  s rho (c.u) = c.sJ,
  //   c.u = (c.sJ) inv,
  // so each opposite pair needs c.sJ alone (additions of the momentum sums).
  const T J2 = R::fma(sJz, sJz, R::fma(sJy, sJy, R::mul(sJx, sJx)));
  T sA = R::fma(-R::mul(K.q15, inv), J2, R::mul(K.lp, sdrho));  // s * A
  if (FORCE) {
    const T Jg = FM == 1 ? R::mul(sJx, K.g[0]) : R::fma(sJz, K.g[2], R::fma(sJy, K.g[1], R::mul(sJx, K.g[0])));
    sA = R::fma(-K.q3, Jg, sA);
  }
  d[0] = R::fma(K.om1, d[0], R::mul(T(WD(0)), sA));
  const T wsA[2] = {R::mul(T(WD(1)), sA), R::mul(T(WD(7)), sA)};
  const T tpi[2] = {R::mul(K.tp[0], inv), R::mul(K.tp[1], inv)};  // tp_c / (s rho)
  // c_i . v in the fixed order x, y, z
  auto dot = [&](int i, T vx, T vy, T vz) {
    T r = 0;
    bool first = true;
    if (CX(i)) { r = CX(i) > 0 ? vx : -vx; first = false; }
    if (CY(i)) { r = first ? (CY(i) > 0 ? vy : -vy) : (CY(i) > 0 ? R::add(r, vy) : R::sub(r, vy)); first = false; }
    if (CZ(i)) { r = first ? (CZ(i) > 0 ? vz : -vz) : (CZ(i) > 0 ? R::add(r, vz) : R::sub(r, vz)); }
    return r;
  };
  // For pair k with P = s (w A + rho (c.u)(tp_c c.u + fp_k)) and
  // M = s rho (tm_c c.u + fm_k), the two sums are formed directly from
  // sc = c.sJ = s rho c.u:
  //   P +- M = wsA +- s rho fm_k + sc (tp_c inv sc + (fp_k +- tm_c))
  // (without a force: wsA + sc (tp_c inv sc +- tm_c)).
  auto terms = [&](int k, T &Pp, T &Pm) {
    const int i = 2 * k - 1;
    const int c = i <= 6 ? 0 : 1;
    const T sc = dot(i, sJx, sJy, sJz);
    if (FORCE) {
      // fm_k = 0 when c.g = 0: with g along x, for the pairs with c_x = 0
      T bp = wsA[c], bm = wsA[c];
      if (FM == 2 || CX(i) != 0) {
        bp = R::fma(srho, K.fm[k], wsA[c]);
        bm = R::fma(-srho, K.fm[k], wsA[c]);
      }
      Pp = R::fma(sc, R::fma(tpi[c], sc, K.zp[k]), bp);
      Pm = R::fma(sc, R::fma(tpi[c], sc, K.zm[k]), bm);
    } else {
      Pp = R::fma(sc, R::fma(tpi[c], sc, K.tm[c]), wsA[c]);
      Pm = R::fma(sc, R::fma(tpi[c], sc, -K.tm[c]), wsA[c]);
    }
  };
  if (K.bgk) {
#pragma unroll
    for (int k = 1; k <= 9; ++k) {
      const int i = 2 * k - 1;
      T Pp, Pm;
      terms(k, Pp, Pm);
      d[i] = R::fma(K.om1, d[i], Pp);
      d[i + 1] = R::fma(K.om1, d[i + 1], Pm);
    }
  } else {
    // a* +- b* with a = (d_i + d_opp)/2, b = (d_i - d_opp)/2 expanded, so
    // that only d_i and d_opp stay live:
    //   d*_i = al d_i + be d_opp + (P + M),  d*_opp = be d_i + al d_opp + (P - M)
#pragma unroll
    for (int k = 1; k <= 9; ++k) {
      const int i = 2 * k - 1;
      T Pp, Pm;
      terms(k, Pp, Pm);
      const T di = d[i], dj = d[i + 1];
      d[i] = R::fma(K.al, di, R::fma(K.be, dj, Pp));
      d[i + 1] = R::fma(K.al, dj, R::fma(K.be, di, Pm));
    }
  }
}

template <typename T, bool FORCE, bool SCALED>
__device__ __forceinline__ void collide_f64(T (&d)[Q], const CollK<T> &K, T s, T inv_s, T &drho_out, T &rjx_out) {
  // one uniform branch per node (a kernel parameter or a segment's
  // constants), so the force terms that are zero cost no FP64 instruction
  if (!FORCE)
    collide_f64_body<T, 0, SCALED>(d, K, s, inv_s, drho_out, rjx_out);
  else if (K.gx_only)
    collide_f64_body<T, 1, SCALED>(d, K, s, inv_s, drho_out, rjx_out);
  else
    collide_f64_body<T, 2, SCALED>(d, K, s, inv_s, drho_out, rjx_out);
}

// Two evaluations of the same collision.  FP64 runs on GB300's narrow FP64
// pipe (two thread instructions per SM clock), which bounds every FP64 step
// kernel: collide_f64 minimises FP64 instructions (velocity never formed,
// direction-group moments, a Newton reciprocal; ncu: 114 per update without
// a force).  FP32 arithmetic is cheap, the FP32 and FP16 kernels are bound by
// memory and issue rate within 64-85 registers: collide_f32 keeps fewer
// values live (u instead of J and 1/rho).
template <typename T, bool FORCE, bool SCALED>
__device__ __forceinline__ void collide(T (&d)[Q], const CollK<T> &K, T s, T inv_s, T &drho_out, T &rjx_out) {
  if constexpr (sizeof(T) == 8)
    collide_f64<T, FORCE, SCALED>(d, K, s, inv_s, drho_out, rjx_out);
  else
    collide_f32<T, FORCE, SCALED>(d, K, s, inv_s, drho_out, rjx_out);
}

// The collision in the units a codec's step kernels load: S * d_i for F16S,
// d_i otherwise.
template <class C, bool FORCE>
__device__ __forceinline__ void collide_stored(typename C::T (&d)[Q], const CollK<typename C::T> &K, float scale,
                                               float inv_scale, typename C::T &drho, typename C::T &rjx) {
  using T = typename C::T;
  collide<T, FORCE, C::kScaled>(d, K, T(scale), T(inv_scale), drho, rjx);
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
  void *mapbase[Q];   // esoteric twist, SoA: start of array map[i] (A + map[i] npad)
  double omega, gx, gy, gz;
  double omega_m;     // antisymmetric rate (TRT); equal to omega for BGK
  CollK<float> kf;    // collision constants for FP32 arithmetic (F32, F16S)
  CollK<double> kd;   // ... for FP64
  float scale, inv_scale;
  double *partials;   // fused reduction: 2 doubles per block, or nullptr
  int *err;           // device error word
  int z0, z1;         // compressed grid: planes of this launch
  int zo_read, zo_write;  // compressed grid: plane offsets of the old and new state
  int64_t slab0, slab1;   // compressed grid on a node list: node numbers of this launch
  int idx_folded;         // AA pattern, SoA node list: IDX holds bounce-back slots, no -1
};

template <typename T>
__device__ __forceinline__ const CollK<T> &coll_of(const StepParams &p);
template <>
__device__ __forceinline__ const CollK<float> &coll_of<float>(const StepParams &p) {
  return p.kf;
}
template <>
__device__ __forceinline__ const CollK<double> &coll_of<double>(const StepParams &p) {
  return p.kd;
}

// Hide a value's provenance from the optimiser: addresses derived from the
// result are recomputed instead of kept live from an earlier phase (loads and
// stores of a node touch the same slots, and holding 19 64-bit addresses
// across the collision costs ~40 registers).
__device__ __forceinline__ int launder(int v) {
  asm volatile("" : "+r"(v));
  return v;
}

// Per-thread node context for full-grid addressing.  The wrap-adjusted cell
// deltas to the -1/+1 neighbour along each axis are computed once per node
// (on a wall face the delta points into the halo and a wall bit is set), so
// a neighbour slot costs a few 32-bit adds.  Step kernels map threads to
// cells with a 2D block over (x, y) and grid z over planes; the state
// kernels use a flat cell index.
struct DirectNode {
  int x, y, z;
  int s;      // own storage slot
  int cell;   // own cell (solid mask index)
  int dx[2], dy[2], dz[2];
  int dzc[2];     // z deltas for the solid lookup (wrapped even with ghost planes)
  unsigned wall;  // bit 2a + side: face (axis a, -1 / +1 side) is a wall
  bool fast;      // no wall face and no solid mask: every neighbour is fluid

  __device__ __forceinline__ bool setup(const Grid &g) {
    // the cell index is needed only for solid lookups (a mask exists)
    cell = 0;
    if (g.solid != nullptr) {
      cell = x + g.nx * (y + g.ny * z);
      if (g.solid[cell]) return false;
    }
    // storage slots fit in 31 bits (checked when the geometry is built)
    s = (x + g.hx) + (int)g.sx * (y + g.hy) + (int)g.sxy * (z + g.hz + (int)g.zoff);
    const bool xl = x == 0, xh = x == g.nx - 1, yl = y == 0, yh = y == g.ny - 1, zl = z == 0, zh = z == g.nz - 1;
    // deltas to the -1 / +1 neighbour: wrapped across a periodic face, plain
    // +-1 at a wall face (the halo slot beyond it; the face also sets its
    // wall bit)
    dx[0] = (xl && g.px) ? g.nx - 1 : -1;
    dx[1] = (xh && g.px) ? 1 - g.nx : 1;
    dy[0] = (yl && g.py) ? g.ny - 1 : -1;
    dy[1] = (yh && g.py) ? 1 - g.ny : 1;
    dzc[0] = (zl && g.pz) ? g.nz - 1 : -1;
    dzc[1] = (zh && g.pz) ? 1 - g.nz : 1;
    dz[0] = g.zghost ? -1 : dzc[0];
    dz[1] = g.zghost ? 1 : dzc[1];
    wall = (g.px ? 0u : ((unsigned)xl | (unsigned)xh << 1)) | (g.py ? 0u : ((unsigned)yl << 2 | (unsigned)yh << 3)) |
           (g.pz ? 0u : ((unsigned)zl << 4 | (unsigned)zh << 5));
    fast = wall == 0 && g.solid == nullptr;
    return true;
  }
  // flat cell index (state kernels)
  __device__ __forceinline__ bool init(const StepParams &p, int64_t n) {
    const Grid &g = p.g;
    x = (int)(n % g.nx);
    const int64_t r = n / g.nx;
    y = (int)(r % g.ny);
    z = (int)(r / g.ny);
    return setup(g);
  }
  // step kernels: x, y from the 2D block, z = it
  __device__ static __forceinline__ int64_t it_begin(const StepParams &) { return blockIdx.z; }
  __device__ static __forceinline__ int64_t it_end(const StepParams &p) { return p.g.nz; }
  __device__ static __forceinline__ int64_t it_step(const StepParams &) { return gridDim.z; }
  __device__ __forceinline__ bool init_it(const StepParams &p, int64_t it) {
    x = blockIdx.x * blockDim.x + threadIdx.x;
    y = blockIdx.y * blockDim.y + threadIdx.y;
    z = (int)it;
    if (x >= p.g.nx || y >= p.g.ny) return false;
    return setup(p.g);
  }
  __device__ __forceinline__ void launder_all() {
    s = launder(s);
    cell = launder(cell);
    dx[0] = launder(dx[0]);
    dx[1] = launder(dx[1]);
    dy[0] = launder(dy[0]);
    dy[1] = launder(dy[1]);
    dz[0] = launder(dz[0]);
    dz[1] = launder(dz[1]);
    dzc[0] = launder(dzc[0]);
    dzc[1] = launder(dzc[1]);
    wall = (unsigned)launder((int)wall);
    fast = launder((int)fast) != 0;
  }
  // storage slot of x + c_i whether fluid or not (the halo beyond a wall)
  __device__ __forceinline__ int pos(const StepParams &p, int i) const {
    const int ex = CX(i) < 0 ? dx[0] : (CX(i) > 0 ? dx[1] : 0);
    const int ey = CY(i) < 0 ? dy[0] : (CY(i) > 0 ? dy[1] : 0);
    const int ez = CZ(i) < 0 ? dz[0] : (CZ(i) > 0 ? dz[1] : 0);
    return s + ex + (int)p.g.sx * ey + (int)p.g.sxy * ez;
  }
  // neighbour slot when the node is known to be `fast` (never -1)
  __device__ __forceinline__ int nb_fast(const StepParams &p, int i) const { return pos(p, i); }
  // FAST selects nb_fast at compile time
  template <bool FAST>
  __device__ __forceinline__ int nbf(const StepParams &p, int i) const {
    return FAST ? nb_fast(p, i) : nb(p, i);
  }
  // slot of the fluid neighbour along c_i, or -1 for a wall or solid link
  __device__ __forceinline__ int nb(const StepParams &p, int i) const {
    const unsigned need = (CX(i) < 0 ? 1u : 0u) | (CX(i) > 0 ? 2u : 0u) | (CY(i) < 0 ? 4u : 0u) |
                          (CY(i) > 0 ? 8u : 0u) | (CZ(i) < 0 ? 16u : 0u) | (CZ(i) > 0 ? 32u : 0u);
    if (wall & need) return -1;
    const int ex = CX(i) < 0 ? dx[0] : (CX(i) > 0 ? dx[1] : 0);
    const int ey = CY(i) < 0 ? dy[0] : (CY(i) > 0 ? dy[1] : 0);
    const int ez = CZ(i) < 0 ? dz[0] : (CZ(i) > 0 ? dz[1] : 0);
    const int ec = CZ(i) < 0 ? dzc[0] : (CZ(i) > 0 ? dzc[1] : 0);
    if (p.g.solid && p.g.solid[cell + ex + p.g.nx * (ey + p.g.ny * ec)]) return -1;
    return s + ex + (int)p.g.sx * ey + (int)p.g.sxy * ez;
  }
};

// Per-thread node context for IDX addressing.
struct IndirectNode {
  int s;
  __device__ __forceinline__ bool init(const StepParams &, int64_t n) {
    s = (int)n;
    return true;
  }
  __device__ static __forceinline__ int64_t it_begin(const StepParams &) {
    return (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  }
  __device__ static __forceinline__ int64_t it_end(const StepParams &p) { return p.nnodes; }
  __device__ static __forceinline__ int64_t it_step(const StepParams &) { return (int64_t)gridDim.x * blockDim.x; }
  __device__ __forceinline__ bool init_it(const StepParams &p, int64_t it) { return init(p, it); }
  __device__ __forceinline__ void launder_all() { s = launder(s); }
  static constexpr bool fast = false;
  // FAST: the entry is used as a slot whatever it holds (folded IDX)
  template <bool FAST>
  __device__ __forceinline__ int nbf(const StepParams &p, int i) const { return nb(p, i); }
  __device__ __forceinline__ int nb(const StepParams &p, int i) const {
    return __ldg(p.idx + (int64_t)(i - 1) * p.ipad + s);
  }
};

// ---------------------------------------------------------------------------
// Block reduction of (mass, flux) into FP64 partials[2 index], [2 index + 1]
// (a fixed order: warp trees, then the warps in order).  Ends with a block
// barrier, so a block may call it again (one partial per work chunk).
// Works for 1D, 2D and 3D blocks.
__device__ __forceinline__ void block_reduce_store_at(double m, double j, double *partials, int64_t index) {
  __shared__ double sm[32], sj[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m += __shfl_xor_sync(0xffffffffu, m, o);
    j += __shfl_xor_sync(0xffffffffu, j, o);
  }
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int lane = tid & 31, warp = tid >> 5;
  if (lane == 0) {
    sm[warp] = m;
    sj[warp] = j;
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
    m = lane < nw ? sm[lane] : 0.0;
    j = lane < nw ? sj[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      m += __shfl_xor_sync(0xffffffffu, m, o);
      j += __shfl_xor_sync(0xffffffffu, j, o);
    }
    if (lane == 0) {
      partials[2 * index] = m;
      partials[2 * index + 1] = j;
    }
  }
  __syncthreads();
}

// The same with the block's id in launch order as the index.
__device__ __forceinline__ void block_reduce_store(double m, double j, double *partials) {
  block_reduce_store_at(m, j, partials,
                        blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z));
}

}  // namespace lbmk
