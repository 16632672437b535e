// Swap algorithm (Sec. 5, Fig. 3, Tab. 4) on a full grid, push form, blocked.
//
// The serial swap collides a node into its reversed slots (the post-collision
// PDF along c_i goes to the node's slot of the opposite direction) and then
// completes each link to an already visited neighbour by exchanging the two
// PDFs that travel along it; a link into a wall or solid needs no exchange.
// That gives the natural next state for any visiting order in which a link is
// exchanged after both of its nodes have collided.
//
// Here the order is blocked, as Sec. 5 allows: the box is cut into tiles, one
// CTA per tile, and the tiles are coloured so that no two tiles sharing a link
// have the same colour (per axis: tile index mod 2, a third colour for the
// last tile of an odd periodic axis).  Colours run as consecutive launches.
// Inside a CTA every node collides into shared memory; links inside the tile
// are completed there; a link to a tile of an earlier colour is completed by
// exchanging with global memory (that tile left its end reversed); a link to a
// tile of a later colour is left reversed for that tile to complete.  Which
// neighbour tiles are earlier, and from that the class of every link of
// every cell, comes from per-tile tables built on the host for the geometry
// (lbm_swap.cu); the reversed slots of earlier tiles are fetched with
// asynchronous copies while the tile collides.
//
// Kernels and launch templates; lbm_swap_f64.cu / _f32.cu / _f16s.cu
// instantiate them per storage precision, lbm_swap.cu holds the host side.
#pragma once

#include <cuda.h>

#include <algorithm>

#include "lbm_async.cuh"
#include "lbm_dispatch.cuh"
#include "lbm_internal.h"

namespace lbmk {

struct SwapPass {
  int tx, ty, tz;              // tile extent
  int ntx, nty, ntz;           // tiles per axis
  int cx, cy, cz;              // colours per axis
  int colour;                  // colour of this pass (cx-fastest)
  int start[3], count[3];      // tiles of this pass per axis: start + stride k
  int stride;                  // 2 for a colour of the coloured schedule; 1 for every tile at once
  const uint16_t *tcls;        // per tile: index of its link-class table
  const uint32_t *tables;      // kSwapTableWords words per table
};

// The link-class table of a tile (built on the host): [0] earlier-colour
// neighbour mask, [1] self mask, [2 + 3c ...] the class words of cell class c.
__device__ __forceinline__ const uint32_t *tile_table(const SwapPass &sp, const int tile[3]) {
  const int tl = tile[0] + sp.ntx * (tile[1] + sp.nty * tile[2]);
  return sp.tables + kSwapTableWords * (int)__ldg(sp.tcls + tl);
}

static_assert(kSwapTX % 32 == 0 && kSwapTX * kSwapTY * kSwapTZ <= 256, "tile box");

// Cell pairs (Grid::zpair: cells z and z + nz/2 in one word) as one storage
// element: the swap then runs unchanged on the grid of pair words (nz/2
// planes, z periodic), two collisions per element.  A link across that
// grid's z wrap joins the two halves the other way round (the seam), so the
// word is exchanged with its halves swapped.
template <class C1>
struct CodecPair {
  using Single = C1;
  using S = typename std::conditional<sizeof(typename C1::S) == 2, __half2, float2>::type;
  using T = float2;
  static constexpr int kMinBlocks = 2;
  static constexpr bool kScaled = C1::kScaled;
  __device__ static __forceinline__ T raw(S v) {
    if constexpr (sizeof(typename C1::S) == 2)
      return __half22float2(v);
    else
      return v;
  }
  __device__ static __forceinline__ S unraw(T v) {
    if constexpr (sizeof(typename C1::S) == 2)
      return __floats2half2_rn(v.x, v.y);
    else
      return v;
  }
};
template <class C>
struct IsPairCodec : std::false_type {};
template <class C1>
struct IsPairCodec<CodecPair<C1>> : std::true_type {};

// The pull of slot i from x - c_i crosses the seam (pair codecs; z is the
// pair plane, g.nz the number of pair planes).
__device__ __forceinline__ bool swap_seam(const Grid &g, int z, int i) {
  return (CZ(i) > 0 && z == 0) || (CZ(i) < 0 && z == g.nz - 1);
}
template <class C>
__device__ __forceinline__ typename C::T seam_value(typename C::T v, bool seam) {
  if constexpr (IsPairCodec<C>::value)
    return seam ? make_float2(v.y, v.x) : v;
  else
    return v;
}

// Index of a neighbour-tile offset (ox, oy, oz) in {-1, 0, 1}^3.
__host__ __device__ constexpr int tile_bit(int ox, int oy, int oz) { return (ox + 1) + 3 * ((oy + 1) + 3 * (oz + 1)); }

// FIXED: the tile box is the full kSwapTX x kSwapTY x kSwapTZ (every box of
// at least that size), so shared-memory offsets are compile-time constants.
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
      : "memory");
}

// Word of the remote-prefetch buffer: the stored element, or for 2-byte
// elements the aligned 4-byte word that holds it (asynchronous copies move 4,
// 8 or 16 bytes).
template <class C>
using RemoteWord = typename std::conditional<sizeof(typename C::S) == 2, uint32_t, typename C::S>::type;

template <class C>
__device__ __forceinline__ void prefetch_remote(RemoteWord<C> *dst, const typename C::S *src) {
  if constexpr (sizeof(typename C::S) == 2) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(src) & ~uintptr_t(3);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(a) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "n"(sizeof(typename C::S))
                 : "memory");
  }
}
// the prefetched element (odd slots are the high half of a 2-byte pair)
template <class C>
__device__ __forceinline__ typename C::T fetch_remote(const RemoteWord<C> &w, int slot) {
  if constexpr (sizeof(typename C::S) == 2) {
    const unsigned short h = (unsigned short)((slot & 1) ? (w >> 16) : (w & 0xffffu));
    return C::raw(__ushort_as_half(h));
  } else {
    return C::raw(w);
  }
}

template <class C, int AOS, bool FORCE, bool FIXED>
__device__ __forceinline__ void swap_tile(const StepParams &p, const SwapPass &sp, typename C::T *S,
                                          const typename C::S *stage, RemoteWord<C> *R, const uint32_t *cls,
                                          const int org[3], unsigned em, unsigned sm, double &m, double &jsum) {
  using T = typename C::T;
  Lattice<C, AOS> L{static_cast<typename C::S *>(p.A), p.npad, p.scale, p.inv_scale};
  const Grid &g = p.g;
  const int TX = FIXED ? kSwapTX : sp.tx, TY = FIXED ? kSwapTY : sp.ty, TZ = FIXED ? kSwapTZ : sp.tz;
  const int TN = TX * TY * TZ;
  const int lx = threadIdx.x, ly = threadIdx.y, lz = threadIdx.z;
  const int t = lx + TX * (ly + TY * lz);
  // extent of this tile inside the box (the last tile of an axis may be cut)
  const int ex = min(TX, g.nx - org[0]), ey = min(TY, g.ny - org[1]), ez = min(TZ, g.nz - org[2]);
  DirectNode nd;
  bool active = lx < ex && ly < ey && lz < ez;
  if (active) {
    nd.x = org[0] + lx;
    nd.y = org[1] + ly;
    nd.z = org[2] + lz;
    active = nd.setup(g);
  }
  // Full tile whose nodes all have every neighbour (no solid mask, no wall
  // face touching the tile): the branch structure below is uniform over each
  // warp (a warp covers 32 cells of one row) except on the x faces.
  bool tile_fast = FIXED && g.solid == nullptr && ex == TX && ey == TY && ez == TZ;
  if (FIXED) {
    tile_fast = tile_fast && (g.px || (org[0] > 0 && org[0] + TX < g.nx)) &&
                (g.py || (org[1] > 0 && org[1] + TY < g.ny)) && (g.pz || (org[2] > 0 && org[2] + TZ < g.nz));
  }
  const bool xm = lx == 0, xp = lx == TX - 1, ym = ly == 0, yp = ly == TY - 1, zm = lz == 0, zp = lz == TZ - 1;
  // Links to tiles of earlier colours: start the copies of their reversed
  // slots now, so that the collision below covers the memory latency.
  unsigned omask = 0, rmask = 0, smask = 0;
  if (FIXED && tile_fast && active) {
    const int c = (xm ? 0 : (xp ? 2 : 1)) + 3 * ((ym ? 0 : (yp ? 2 : 1)) + 3 * (zm ? 0 : 1));
    omask = __ldg(cls + 3 * c);
    rmask = __ldg(cls + 3 * c + 1);
    smask = __ldg(cls + 3 * c + 2);
#pragma unroll
    for (int i = 1; i < Q; ++i)
      if (rmask & (1u << i)) prefetch_remote<C>(&R[(i - 1) * TN + t], L.at(OPP(i), nd.nb_fast(p, OPP(i))));
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  if (active) {
    T d[Q];
    if (stage) {
#pragma unroll
      for (int i = 0; i < Q; ++i) d[i] = C::raw(stage[i * TN + t]);
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) d[i] = L.ld(i, nd.s);
    }
    if constexpr (IsPairCodec<C>::value) {
      using C1 = typename C::Single;
      float da[Q], db[Q], ra, ja, rb, jb;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        da[i] = d[i].x;
        db[i] = d[i].y;
      }
      collide_stored<C1, FORCE>(da, coll_of<float>(p), p.scale, p.inv_scale, ra, ja);
      collide_stored<C1, FORCE>(db, coll_of<float>(p), p.scale, p.inv_scale, rb, jb);
      m += 1.0 + (double)ra;
      jsum += (double)ja;
      m += 1.0 + (double)rb;
      jsum += (double)jb;
#pragma unroll
      for (int i = 0; i < Q; ++i) d[i] = make_float2(da[i], db[i]);
    } else {
      T drho, rjx;
      collide_stored<C, FORCE>(d, coll_of<T>(p), p.scale, p.inv_scale, drho, rjx);
      m += 1.0 + (double)drho;
      jsum += (double)rjx;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) S[i * TN + t] = d[i];
  }
  __syncthreads();
  if (FIXED && tile_fast && active) {
    asm volatile("cp.async.wait_group 0;" ::: "memory");  // this thread's prefetches
    // Each slot i takes g_i(x - c_i): from the tile (inside), from the other
    // end of the tile (its own neighbour across a periodic face), the node's
    // own reversed PDF (a later tile completes the link), or the prefetched
    // reversed slot of an earlier tile (whose slot then takes our PDF).
    T v[Q];
    v[0] = S[t];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int cx = CX(i), cy = CY(i), cz = CZ(i);
      const bool ox = cx > 0 ? xm : (cx < 0 ? xp : false);
      const bool oy = cy > 0 ? ym : (cy < 0 ? yp : false);
      const bool oz = cz > 0 ? zm : (cz < 0 ? zp : false);
      const unsigned b = 1u << i;
      int a = !(omask & b) ? i * TN + t - (cx + TX * (cy + TY * cz)) : OPP(i) * TN + t;
      if (smask & b)  // the tile's own far end (one tile along a periodic axis)
        a = i * TN + (ox ? (cx > 0 ? TX - 1 : 0) : lx - cx) +
            TX * ((oy ? (cy > 0 ? TY - 1 : 0) : ly - cy) + TY * (oz ? (cz > 0 ? TZ - 1 : 0) : lz - cz));
      v[i] = S[a];
      if (rmask & b) v[i] = seam_value<C>(fetch_remote<C>(R[(i - 1) * TN + t], nd.nb_fast(p, OPP(i))),
                                          IsPairCodec<C>::value && swap_seam(g, nd.z, i));
    }
    nd.launder_all();
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      L.st(i, nd.s, v[i]);
      if (i > 0 && (rmask & (1u << i)))
        L.st(OPP(i), nd.nb_fast(p, OPP(i)),
             seam_value<C>(S[OPP(i) * TN + t], IsPairCodec<C>::value && swap_seam(g, nd.z, i)));
    }
  } else if (active) {
    // Gather every incoming value first (the loads from earlier tiles are
    // independent and overlap), then write: the remote slots written below
    // belong to earlier tiles and are never read by this pass again.
    T v[Q];
    int remote[Q];
    v[0] = S[t];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      remote[i] = -1;
      // the PDF arriving along c_i comes from x - c_i
      const int dx = -CX(i), dy = -CY(i), dz = -CZ(i);
      const bool in_x = dx == 0 || (dx < 0 ? lx > 0 : lx < ex - 1);
      const bool in_y = dy == 0 || (dy < 0 ? ly > 0 : ly < ey - 1);
      const bool in_z = dz == 0 || (dz < 0 ? lz > 0 : lz < ez - 1);
      // source slot, or -1 across a wall or from a solid cell (a fast node
      // has neither, and needs the slot only for a remote exchange)
      int src = 0;
      if (!nd.fast) {
        src = nd.nb(p, OPP(i));
        if (src < 0) {
          v[i] = S[OPP(i) * TN + t];  // bounce-back: the node's own reversed PDF
          continue;
        }
      }
      if (in_x && in_y && in_z) {
        v[i] = S[i * TN + t + dx + TX * (dy + TY * dz)];  // inside the tile
        continue;
      }
      const int bit = tile_bit(in_x ? 0 : dx, in_y ? 0 : dy, in_z ? 0 : dz);
      if (sm & (1u << bit)) {
        // the tile is its own neighbour across a periodic face
        const int wx = in_x ? lx + dx : (dx < 0 ? ex - 1 : 0);
        const int wy = in_y ? ly + dy : (dy < 0 ? ey - 1 : 0);
        const int wz = in_z ? lz + dz : (dz < 0 ? ez - 1 : 0);
        v[i] = S[i * TN + wx + TX * (wy + TY * wz)];
      } else if (em & (1u << bit)) {
        // earlier tile: its reversed slot holds the PDF for us; ours goes there
        if (nd.fast) src = nd.nb_fast(p, OPP(i));
        remote[i] = src;
        v[i] = seam_value<C>(L.ld(OPP(i), src), IsPairCodec<C>::value && swap_seam(g, nd.z, i));
      } else {
        v[i] = S[OPP(i) * TN + t];  // a later tile completes the link
      }
    }
    nd.launder_all();
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      L.st(i, nd.s, v[i]);
      if (i > 0 && remote[i] >= 0)
        L.st(OPP(i), remote[i], seam_value<C>(S[OPP(i) * TN + t], IsPairCodec<C>::value && swap_seam(g, nd.z, i)));
    }
  }
}

// One pass: the tiles of one colour, one block per tile.  Full tiles with
// 4-byte arithmetic fit four blocks per SM (64 registers; measured faster
// than three, the only spill is a few bytes).  Full tiles of FP16 cell
// pairs fit three (80 registers, no spill; 37.3 against 32.0 GFLUP/s at two
// on 256^3; four spill several hundred bytes); FP32 pairs stay at two (24.2
// against 25.5 at three).
template <class C, bool FIXED>
constexpr int swap_min_blocks() {
  if constexpr (IsPairCodec<C>::value)
    return (FIXED && sizeof(typename C::Single::S) == 2) ? 3 : C::kMinBlocks;
  else
    return (FIXED && sizeof(typename C::T) == 4) ? 4 : C::kMinBlocks;
}

template <class C, int AOS, bool FORCE, bool RED, bool FIXED>
__global__ void __launch_bounds__(256, (swap_min_blocks<C, FIXED>())) k_swap_pass(StepParams p, SwapPass sp) {
  chain_wait();
  using T = typename C::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *S = reinterpret_cast<T *>(smem_raw);
  const int TN = sp.tx * sp.ty * sp.tz;
  RemoteWord<C> *R = reinterpret_cast<RemoteWord<C> *>(smem_raw + ((size_t)Q * TN * sizeof(T) + 15) / 16 * 16);
  const int tile[3] = {sp.start[0] + sp.stride * (int)blockIdx.x, sp.start[1] + sp.stride * (int)blockIdx.y,
                       sp.start[2] + sp.stride * (int)blockIdx.z};
  const int org[3] = {tile[0] * sp.tx, tile[1] * sp.ty, tile[2] * sp.tz};
  const uint32_t *tab = tile_table(sp, tile);
  double m = 0.0, jsum = 0.0;
  swap_tile<C, AOS, FORCE, FIXED>(p, sp, S, nullptr, R, tab + 2, org, __ldg(tab), __ldg(tab + 1), m, jsum);
  if (RED) block_reduce_store(m, jsum, p.partials);
}

// ---------------------------------------------------------------------------
// The same pass with the tiles staged by the tensor memory accelerator: a
// persistent block walks its share of the pass's tiles and, while it works
// on one tile, the tensor copy of its next tile (all 19 arrays of the tile's
// box in one 4D copy: x, y, z, array) is already in flight into the other of
// two shared-memory buffers.  Every wait on a copy is bounded by a time
// limit; on expiry the block records the timeout and stops.
constexpr uint64_t kTmaWaitNs = 1000000000ull;  // 1 s

template <class C, bool FORCE, bool RED, bool FIXED>
__global__ void __launch_bounds__(256, C::kMinBlocks) k_swap_tma(StepParams p, SwapPass sp, const __grid_constant__ CUtensorMap map) {
  chain_wait();
  using T = typename C::T;
  using S = typename C::S;
  constexpr bool kInPlace = sizeof(T) == sizeof(S);  // F32, F64: collide into the staged buffer
  extern __shared__ __align__(128) unsigned char smem_tma[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int tiles[2][3];       // [buffer] tile coordinates, written with the copy's issue
  const int TN = sp.tx * sp.ty * sp.tz;
  const size_t stage_bytes = (size_t)Q * TN * sizeof(S);
  const size_t stage_pad = (stage_bytes + 127) / 128 * 128;
  // tensor-copy destinations on 128-byte boundaries (the launch adds 128
  // bytes of slack for this)
  unsigned char *base = smem_tma + ((128u - (smem_addr(smem_tma) & 127u)) & 127u);
  S *stage[2] = {reinterpret_cast<S *>(base), reinterpret_cast<S *>(base + stage_pad)};
  T *Sx = reinterpret_cast<T *>(base + 2 * stage_pad);  // separate buffer when not in place
  const size_t sx_bytes = kInPlace ? 0 : ((size_t)Q * TN * sizeof(T) + 15) / 16 * 16;
  RemoteWord<C> *R = reinterpret_cast<RemoteWord<C> *>(base + 2 * stage_pad + sx_bytes);
  const int t = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int ntiles = sp.count[0] * sp.count[1] * sp.count[2];
  auto tile_of = [&](int n, int tile[3]) {
    tile[0] = sp.start[0] + sp.stride * (n % sp.count[0]);
    tile[1] = sp.start[1] + sp.stride * ((n / sp.count[0]) % sp.count[1]);
    tile[2] = sp.start[2] + sp.stride * (n / (sp.count[0] * sp.count[1]));
  };
  auto issue = [&](int n, int b) {
    int tile[3];
    tile_of(n, tile);
    tiles[b][0] = tile[0];
    tiles[b][1] = tile[1];
    tiles[b][2] = tile[2];
    mbar_expect_tx(&bar[b], (uint32_t)stage_bytes);
    tma_load_4d(stage[b], &map, tile[0] * sp.tx, tile[1] * sp.ty, tile[2] * sp.tz, 0, &bar[b]);
  };
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  double m = 0.0, jsum = 0.0;
  const int G = gridDim.x;
  if (t == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
  __syncthreads();  // tiles[0]
  int it = 0;
  for (int n = blockIdx.x; n < ntiles; n += G, ++it) {
    const int b = it & 1;
    const int tile[3] = {tiles[b][0], tiles[b][1], tiles[b][2]};
    if (t == 0) {
      // the other buffer was last read in the previous iteration, which
      // ended with a block barrier; order those generic-proxy accesses
      // before the tensor copy overwrites it
      if (n + G < ntiles) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(n + G, b ^ 1);
      }
    }
    const bool ok = mbar_wait(&bar[b], (uint32_t)((it >> 1) & 1), kTmaWaitNs);
    if (__syncthreads_or(!ok)) {
      if (t == 0) {
        atomicExch(p.err + 1, 1);
        // let the copies still in flight land before the block exits
        mbar_wait(&bar[b], (uint32_t)((it >> 1) & 1), kTmaWaitNs);
        if (n + G < ntiles) mbar_wait(&bar[b ^ 1], (uint32_t)(((it + 1) >> 1) & 1), kTmaWaitNs);
      }
      break;
    }
    const int org[3] = {tile[0] * sp.tx, tile[1] * sp.ty, tile[2] * sp.tz};
    T *Sbuf = kInPlace ? reinterpret_cast<T *>(stage[b]) : Sx;
    const uint32_t *tab = tile_table(sp, tile);
    swap_tile<C, 0, FORCE, FIXED>(p, sp, Sbuf, stage[b], R, tab + 2, org, __ldg(tab), __ldg(tab + 1), m, jsum);
    __syncthreads();
  }
  if (RED) block_reduce_store(m, jsum, p.partials);
}

template <class C, int AOS, bool IND, bool FORCE, bool RED>
struct LaunchSwap {
  static void run(const StepParams &p, const SwapPass &sp, size_t smem, dim3 blocks, cudaStream_t s) {
    const bool fixed = sp.tx == kSwapTX && sp.ty == kSwapTY && sp.tz == kSwapTZ;
    auto k = fixed ? k_swap_pass<C, AOS, FORCE, RED, true> : k_swap_pass<C, AOS, FORCE, RED, false>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    launch_chained(k, blocks, dim3(sp.tx, sp.ty, sp.tz), smem, s, p, sp);
  }
};

// Persistent launch: as many blocks as fit on the GPU at once (resident
// blocks per SM for this block shape and shared memory x SMs), at most one
// per tile.  Returns the number of blocks launched.
template <class C, int AOS, bool IND, bool FORCE, bool RED>
struct LaunchSwapTma {
  static void run(const StepParams &p, const SwapPass &sp, const CUtensorMap *map, int nsm, int ntiles,
                  cudaStream_t s, int *launched) {
    *launched = 0;
    if constexpr (AOS == 0 && !IND) {
      const bool fixed = sp.tx == kSwapTX && sp.ty == kSwapTY && sp.tz == kSwapTZ;
      auto k = fixed ? k_swap_tma<C, FORCE, RED, true> : k_swap_tma<C, FORCE, RED, false>;
      const int threads = sp.tx * sp.ty * sp.tz;
      const size_t smem = swap_tma_smem_bytes(threads, sizeof(typename C::S), sizeof(typename C::T));
      static_assert(sizeof(RemoteWord<C>) == (sizeof(typename C::S) < 4 ? 4 : sizeof(typename C::S)), "word");
      if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
      const int grid = std::min(ntiles, per_sm * std::max(nsm, 1));
      launch_chained(k, dim3(grid), dim3(sp.tx, sp.ty, sp.tz), smem, s, p, sp, *map);
      *launched = grid;
    }
  }
};

// Per-precision entry points (instantiated in lbm_swap_<precision>.cu).
template <class C>
void swap_pass_t(const StepParams &p, const SwapPass &sp, const KernelKey &k, size_t smem, cudaStream_t s) {
  const dim3 blocks(sp.count[0], sp.count[1], sp.count[2]);
  dispatch_layout<LaunchSwap, C>(k.aos, false, k.force, k.red, p, sp, smem, blocks, s);
}
// Cell pairs: SoA, full grid only, so only those instantiations.
template <class C>
void swap_pass_pair_t(const StepParams &p, const SwapPass &sp, const KernelKey &k, size_t smem, cudaStream_t s) {
  const dim3 blocks(sp.count[0], sp.count[1], sp.count[2]);
  if (k.force) {
    if (k.red)
      LaunchSwap<C, 0, false, true, true>::run(p, sp, smem, blocks, s);
    else
      LaunchSwap<C, 0, false, true, false>::run(p, sp, smem, blocks, s);
  } else {
    if (k.red)
      LaunchSwap<C, 0, false, false, true>::run(p, sp, smem, blocks, s);
    else
      LaunchSwap<C, 0, false, false, false>::run(p, sp, smem, blocks, s);
  }
}
template <class C>
int swap_pass_tma_t(const StepParams &p, const SwapPass &sp, const KernelKey &k, const CUtensorMap *map, int nsm,
                    int ntiles, cudaStream_t s) {
  int launched = 0;
  dispatch_layout<LaunchSwapTma, C>(0, false, k.force, k.red, p, sp, map, nsm, ntiles, s, &launched);
  return launched;
}

}  // namespace lbmk
