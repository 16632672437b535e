// Batch step kernels (included by the per-precision lbm_batch_*.cu files
// and, for the shared types, by lbm_batch.cu).
//
// Every admitted geometry ("slot") of a batch is a node list (lexicographic
// fluid nodes, Sec. 1) stored as one segment of shared SoA arrays; a step
// updates work chunks of block_size x NPT nodes of one segment each, with
// that segment's omega, force and parity: the AA pattern (Sec. 6) or the
// esoteric twist (Sec. 7) on the node list.
#pragma once

#include "../../include/lbm.h"
#include "lbm_dispatch.cuh"
#include "lbm_internal.h"

namespace lbmk {

constexpr int64_t kAlign = 4096;  // segment alignment in slots

struct BatchSlot {
  double omega, gx, gy, gz;
  double omega_m;   // antisymmetric rate (TRT); equal to omega for BGK
  int64_t start;    // first slot of the segment
  int64_t nodes;    // fluid nodes
  int64_t steps;    // steps done before the current round
  int32_t first_work, nwork;
  int32_t active, pad;
};

struct BatchParams {
  void *A;
  int64_t npad;
  const int32_t *idx;  // AA: 18 x npad; ET: 9 x npad (packed)
  const BatchSlot *slots;
  const int2 *work;    // (slot, first node of the chunk)
  int nwork;
  int t;               // step within the round
  float scale, inv_scale;
  double *partials;    // 2 per work chunk
  int folded;          // AA: IDX holds bounce-back slots instead of -1 (capacity < 2^30)
};

template <class C>
__device__ __forceinline__ Lattice<C, 0> batch_lattice(const BatchParams &p) {
  Lattice<C, 0> L;
  L.p = static_cast<typename C::S *>(p.A);
  L.npad = p.npad;
  L.scale = p.scale;
  L.inv_scale = p.inv_scale;
  return L;
}

// Launch of one round's kernels for one precision (lbm_batch_<prec>.cu):
// mode 0: one step (p.t), reducing when red; mode 1: k steps in one
// persistent cooperative launch (step 0 reduces).
template <class C>
cudaError_t launch_batch_t(int variant, int mode, int npt, bool red, const BatchParams &p, int bs, int k,
                           unsigned *count, int *err, uint64_t limit_ns, int nsm, cudaStream_t s);
extern template cudaError_t launch_batch_t<CodecF64>(int, int, int, bool, const BatchParams &, int, int, unsigned *,
                                                     int *, uint64_t, int, cudaStream_t);
extern template cudaError_t launch_batch_t<CodecF32>(int, int, int, bool, const BatchParams &, int, int, unsigned *,
                                                     int *, uint64_t, int, cudaStream_t);
extern template cudaError_t launch_batch_t<CodecF16S>(int, int, int, bool, const BatchParams &, int, int, unsigned *,
                                                      int *, uint64_t, int, cudaStream_t);

#ifdef LBM_BATCH_KERNELS
// One node s of one step of the AA pattern (`odd`: the step's parity) with
// its segment's collision constants K; accumulates its mass and flux.
template <class C>
__device__ __forceinline__ void batch_node_aa(const BatchParams &p, const Lattice<C, 0> &A,
                                              const CollK<typename C::T> &K, bool odd, int s, double &m, double &j) {
  using T = typename C::T;
  T d[Q];
  T drho, rjx;
  if (!odd) {
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = A.ld(i, s);
    collide_stored<C, true>(d, K, p.scale, p.inv_scale, drho, rjx);
    const int s2 = launder(s);
#pragma unroll
    for (int i = 0; i < Q; ++i) A.st(OPP(i), s2, d[i]);
  } else if (p.folded) {
    // every IDX entry is a slot: a solid link holds the slot its
    // bounce-back uses (see k_batch_rebase)
    d[0] = A.ld(0, s);
#pragma unroll
    for (int i = 1; i < Q; ++i) d[i] = A.ld(OPP(i), __ldg(p.idx + (int64_t)(OPP(i) - 1) * p.npad + s));
    collide_stored<C, true>(d, K, p.scale, p.inv_scale, drho, rjx);
    const int s2 = launder(s);
    A.st(0, s2, d[0]);
#pragma unroll
    for (int i = 1; i < Q; ++i) A.st(i, __ldg(p.idx + (int64_t)(i - 1) * p.npad + s2), d[i]);
  } else {
    d[0] = A.ld(0, s);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int src = __ldg(p.idx + (int64_t)(OPP(i) - 1) * p.npad + s);
      d[i] = src >= 0 ? A.ld(OPP(i), src) : A.ld(i, s);
    }
    collide_stored<C, true>(d, K, p.scale, p.inv_scale, drho, rjx);
    const int s2 = launder(s);
    A.st(0, s2, d[0]);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int dst = __ldg(p.idx + (int64_t)(i - 1) * p.npad + s2);
      if (dst >= 0)
        A.st(i, dst, d[i]);
      else
        A.st(OPP(i), s2, d[i]);
    }
  }
  m += 1.0 + (double)drho;
  j += (double)rjx;
}

// One work chunk (block_size x NPT nodes of one segment) of one step of the
// AA pattern; the block takes its segment's parity, omega and force.
// Accumulates the chunk's mass and flux into m, j.
template <class C, int NPT>
__device__ __forceinline__ void batch_chunk_aa(const BatchParams &p, int chunk, int t, double &m, double &j) {
  using T = typename C::T;
  const auto A = batch_lattice<C>(p);
  const int2 w = p.work[chunk];
  const BatchSlot &sl = p.slots[w.x];
  const int64_t end = sl.start + sl.nodes;
  const bool odd = ((sl.steps + t) & 1) != 0;
  const CollK<T> K = make_collk<T>(T(sl.omega), T(sl.omega_m), T(sl.gx), T(sl.gy), T(sl.gz));
#pragma unroll
  for (int r = 0; r < NPT; ++r) {
    const int64_t n64 = (int64_t)w.y + (int64_t)r * blockDim.x + threadIdx.x;
    if (n64 >= end) continue;
    batch_node_aa<C>(p, A, K, odd, (int)n64, m, j);
  }
}

// The same chunk with FP16 storage in node pairs (as k_aa_even_np /
// k_aa_odd_np): nodes 2q and 2q + 1 of the chunk in one thread, NPT / 2
// pairs per thread, one 4-byte word per array for the even step and one
// 8-byte IDX word per direction for the odd step; the per-node arithmetic
// is batch_node_aa's (bit-identical PDFs).  Chunks start at even slots
// (segments are kAlign-aligned, chunks a multiple of 32 nodes long); the
// last node of an odd segment takes the per-node path.  64 FP16 packs
// (79.9 M nodes), rounds of 100 steps: 46.8 against 41.6 GFLUP/s at 512 x 4
// (per-step launches), 38.6 against 31.1 persistent.
template <class C, int NPT>
__device__ __forceinline__ void batch_chunk_aa_np(const BatchParams &p, int chunk, int t, double &m, double &j) {
  using T = typename C::T;
  using PW = PairWord<C>;
  using W = typename PW::W;
  using S = typename C::S;
  const auto A = batch_lattice<C>(p);
  const int2 w = p.work[chunk];
  const BatchSlot &sl = p.slots[w.x];
  const int64_t end = sl.start + sl.nodes;
  const bool odd = ((sl.steps + t) & 1) != 0;
  const CollK<T> K = make_collk<T>(T(sl.omega), T(sl.omega_m), T(sl.gx), T(sl.gy), T(sl.gz));
  W *Aw = static_cast<W *>(p.A);
  S *E = static_cast<S *>(p.A);
  const int64_t nw = p.npad >> 1;  // words per array; IDX words (two nodes) per direction
  const int2 *I = reinterpret_cast<const int2 *>(p.idx);
  auto collide2 = [&](W(&v)[Q]) {
    T d[Q];
    T drho, rjx;
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = PW::lo(v[i]);
    collide_stored<C, true>(d, K, p.scale, p.inv_scale, drho, rjx);
    m += 1.0 + (double)drho;
    j += (double)rjx;
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i] = PW::with_lo(v[i], d[i]);
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = PW::hi(v[i]);
    collide_stored<C, true>(d, K, p.scale, p.inv_scale, drho, rjx);
    m += 1.0 + (double)drho;
    j += (double)rjx;
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i] = PW::with_hi(v[i], d[i]);
  };
#pragma unroll
  for (int r = 0; r < NPT / 2; ++r) {
    const int64_t n64 = (int64_t)w.y + 2 * ((int64_t)r * blockDim.x + threadIdx.x);
    if (n64 >= end) continue;
    if (n64 + 1 == end) {
      batch_node_aa<C>(p, A, K, odd, (int)n64, m, j);
      continue;
    }
    const int wd = (int)(n64 >> 1);
    W v[Q];
    if (!odd) {
#pragma unroll
      for (int i = 0; i < Q; ++i) v[i] = Aw[i * nw + wd];
      collide2(v);
      const int w2 = launder(wd);
#pragma unroll
      for (int i = 0; i < Q; ++i) Aw[OPP(i) * nw + w2] = v[i];
    } else if (p.folded) {
      v[0] = Aw[wd];
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const int2 src = __ldg(I + (OPP(i) - 1) * nw + wd);
        v[i] = PW::pack(E[OPP(i) * p.npad + src.x], E[OPP(i) * p.npad + src.y]);
      }
      collide2(v);
      const int w2 = launder(wd);
      Aw[w2] = v[0];
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const int2 dst = __ldg(I + (i - 1) * nw + w2);
        E[i * p.npad + dst.x] = PW::lo_s(v[i]);
        E[i * p.npad + dst.y] = PW::hi_s(v[i]);
      }
    } else {
      const int s0 = 2 * wd;
      v[0] = Aw[wd];
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const int2 src = __ldg(I + (OPP(i) - 1) * nw + wd);
        const S a = src.x >= 0 ? E[OPP(i) * p.npad + src.x] : E[i * p.npad + s0];
        const S b = src.y >= 0 ? E[OPP(i) * p.npad + src.y] : E[i * p.npad + s0 + 1];
        v[i] = PW::pack(a, b);
      }
      collide2(v);
      const int w2 = launder(wd), s2 = 2 * w2;
      Aw[w2] = v[0];
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const int2 dst = __ldg(I + (i - 1) * nw + w2);
        E[dst.x >= 0 ? i * p.npad + dst.x : OPP(i) * p.npad + s2] = PW::lo_s(v[i]);
        E[dst.y >= 0 ? i * p.npad + dst.y : OPP(i) * p.npad + s2 + 1] = PW::hi_s(v[i]);
      }
    }
  }
}

// One work chunk of one step of the esoteric twist: the array map is the
// identity after an even step count and swaps opposite directions after an
// odd one.
template <class C, int NPT>
__device__ __forceinline__ void batch_chunk_et(const BatchParams &p, int chunk, int t, double &m, double &j) {
  using T = typename C::T;
  const auto A = batch_lattice<C>(p);
  const int2 w = p.work[chunk];
  const BatchSlot &sl = p.slots[w.x];
  const int64_t end = sl.start + sl.nodes;
  const bool odd = ((sl.steps + t) & 1) != 0;
  const CollK<T> K = make_collk<T>(T(sl.omega), T(sl.omega_m), T(sl.gx), T(sl.gy), T(sl.gz));
#pragma unroll
  for (int r = 0; r < NPT; ++r) {
    const int64_t n64 = (int64_t)w.y + (int64_t)r * blockDim.x + threadIdx.x;
    if (n64 >= end) continue;
    const int s = (int)n64;
    uint32_t wd[10];
#pragma unroll
    for (int k = 1; k <= 9; ++k) wd[k] = (uint32_t)__ldg(p.idx + (int64_t)(k - 1) * p.npad + s);
    // array of direction i: i (even step count) or opp(i) (odd)
    T d[Q];
    d[0] = A.ld(0, s);
#pragma unroll
    for (int k = 1; k <= 9; ++k) {
      const int i = 2 * k - 1;
      const int ai = odd ? i + 1 : i, ai1 = odd ? i : i + 1;
      d[i] = A.ld(ai, s);
      d[i + 1] = A.ld(ai1, (int)(wd[k] & 0x7fffffffu));
    }
    T drho, rjx;
    collide_stored<C, true>(d, K, p.scale, p.inv_scale, drho, rjx);
    const int s2 = launder(s);
#pragma unroll
    for (int k = 1; k <= 9; ++k) wd[k] = (uint32_t)launder((int)wd[k]);
    A.st(0, s2, d[0]);
#pragma unroll
    for (int k = 1; k <= 9; ++k) {
      const int i = 2 * k - 1;
      const int ai = odd ? i + 1 : i, ai1 = odd ? i : i + 1;
      const int pos = (int)(wd[k] & 0x7fffffffu);
      const bool lp = pos < end;
      const bool lm = (wd[k] >> 31) == 0u;
      A.st(lp ? ai1 : ai, pos, d[i]);
      A.st(lm ? ai : ai1, s2, d[i + 1]);
    }
    m += 1.0 + (double)drho;
    j += (double)rjx;
  }
}

template <class C, int V, int NPT>
__device__ __forceinline__ void batch_chunk(const BatchParams &p, int chunk, int t, double &m, double &j) {
  if constexpr (V == LBM_ET)
    batch_chunk_et<C, NPT>(p, chunk, t, m, j);
  else if constexpr (std::is_same<C, CodecF16S>::value && NPT >= 2)
    batch_chunk_aa_np<C, NPT>(p, chunk, t, m, j);
  else
    batch_chunk_aa<C, NPT>(p, chunk, t, m, j);
}

// Resident blocks per SM the batch kernels are built for: the step kernels'
// register budget at 256 threads; at 512 threads one block (FP64, 128
// registers) or two (FP32 / FP16, 64 registers).
template <class C, int MAXT>
constexpr int batch_min_blocks() {
  return MAXT <= 256 ? C::kMinBlocks : (C::kMinBlocks == 2 ? 1 : 2);
}

// One step over every active segment: block b takes work chunk b (a chained
// launch: the next step's blocks may be scheduled while this one drains).
template <class C, int V, bool RED, int NPT, int MAXT>
__global__ void __launch_bounds__(MAXT, (batch_min_blocks<C, MAXT>())) k_batch_step(BatchParams p) {
  chain_wait();
  double m = 0.0, j = 0.0;
  batch_chunk<C, V, NPT>(p, blockIdx.x, p.t, m, j);
  if (RED) block_reduce_store_at(m, j, p.partials, blockIdx.x);
}

// Grid-wide barrier of a cooperative launch.  Thread 0 of every block adds
// one to *count, then waits until it reaches `target` (gridDim.x times the
// number of barriers passed so far), reading it with acquire semantics, for
// at most limit_ns nanoseconds; a block that gives up, or sees another
// block's error flag, sets *err and the barrier returns false in every
// thread of the block.
__device__ __forceinline__ bool grid_barrier(unsigned *count, unsigned target, int *err, uint64_t limit_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(count, 1u);
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    int good = 1;
    for (;;) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
      if (v >= target) break;
      if (*((volatile int *)err) != 0) {
        good = 0;
        break;
      }
      uint64_t t1;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
      if (t1 - t0 > limit_ns) {
        atomicExch(err, 1);
        good = 0;
        break;
      }
      __nanosleep(100);
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// A whole round in one cooperative launch: k steps over every active
// segment, blocks striding over the work chunks, a grid barrier between
// steps.  Step 0 writes the per-chunk reduction partials exactly as the
// per-step kernels do (one partial per chunk, same order), so both round
// modes give the same bits.  The PDF loads of a step read what other blocks
// stored in the previous one: plain loads after the barrier's acquire (the
// read-only path is used only for the index, which no step changes).
template <class C, int V, int NPT, int MAXT>
__global__ void __launch_bounds__(MAXT, (batch_min_blocks<C, MAXT>()))
    k_batch_persistent(BatchParams p, int k, unsigned *count, int *err, uint64_t limit_ns) {
  for (int t = 0; t < k; ++t) {
    for (int c = blockIdx.x; c < p.nwork; c += gridDim.x) {
      double m = 0.0, j = 0.0;
      batch_chunk<C, V, NPT>(p, c, t, m, j);
      if (t == 0) block_reduce_store_at(m, j, p.partials, c);
    }
    if (t + 1 < k && !grid_barrier(count, (unsigned)(t + 1) * gridDim.x, err, limit_ns)) return;
  }
}

// Kernel selection: precision x variant x nodes per thread x block bound.
template <class C, int V, int NPT, int MAXT>
static void launch_step_v(bool red, const BatchParams &p, int bs, cudaStream_t s) {
  if (red)
    launch_chained(k_batch_step<C, V, true, NPT, MAXT>, dim3(p.nwork), dim3(bs), 0, s, p);
  else
    launch_chained(k_batch_step<C, V, false, NPT, MAXT>, dim3(p.nwork), dim3(bs), 0, s, p);
}

// Persistent round: the grid is every resident block (co-resident, as a
// cooperative launch requires), at most one per work chunk.
template <class C, int V, int NPT, int MAXT>
static cudaError_t launch_persistent_v(const BatchParams &p, int bs, int k, unsigned *count, int *err,
                                       uint64_t limit_ns, int nsm, cudaStream_t s) {
  auto kern = k_batch_persistent<C, V, NPT, MAXT>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, bs, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  const int grid = std::max(1, std::min(p.nwork, per_sm * nsm));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)bs);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, p, k, count, err, limit_ns);
}

template <class C, int V, int NPT>
static cudaError_t launch_round_npt(int mode, bool red, const BatchParams &p, int bs, int k, unsigned *count, int *err,
                                    uint64_t limit_ns, int nsm, cudaStream_t s) {
  if (mode == 1)
    return bs > 256 ? launch_persistent_v<C, V, NPT, 512>(p, bs, k, count, err, limit_ns, nsm, s)
                    : launch_persistent_v<C, V, NPT, 256>(p, bs, k, count, err, limit_ns, nsm, s);
  if (bs > 256)
    launch_step_v<C, V, NPT, 512>(red, p, bs, s);
  else
    launch_step_v<C, V, NPT, 256>(red, p, bs, s);
  return cudaGetLastError();
}

template <class C, int V>
static cudaError_t launch_round_v(int mode, int npt, bool red, const BatchParams &p, int bs, int k, unsigned *count,
                                  int *err, uint64_t limit_ns, int nsm, cudaStream_t s) {
  switch (npt) {
    case 1: return launch_round_npt<C, V, 1>(mode, red, p, bs, k, count, err, limit_ns, nsm, s);
    case 2: return launch_round_npt<C, V, 2>(mode, red, p, bs, k, count, err, limit_ns, nsm, s);
    case 4: return launch_round_npt<C, V, 4>(mode, red, p, bs, k, count, err, limit_ns, nsm, s);
    default: return launch_round_npt<C, V, 8>(mode, red, p, bs, k, count, err, limit_ns, nsm, s);
  }
}

template <class C>
static cudaError_t launch_round_c(int variant, int mode, int npt, bool red, const BatchParams &p, int bs, int k,
                                  unsigned *count, int *err, uint64_t limit_ns, int nsm, cudaStream_t s) {
  if (variant == LBM_ET) return launch_round_v<C, LBM_ET>(mode, npt, red, p, bs, k, count, err, limit_ns, nsm, s);
  return launch_round_v<C, LBM_AA>(mode, npt, red, p, bs, k, count, err, limit_ns, nsm, s);
}

template <class C>
cudaError_t launch_batch_t(int variant, int mode, int npt, bool red, const BatchParams &p, int bs, int k,
                           unsigned *count, int *err, uint64_t limit_ns, int nsm, cudaStream_t s) {
  return launch_round_c<C>(variant, mode, npt, red, p, bs, k, count, err, limit_ns, nsm, s);
}
#endif  // LBM_BATCH_KERNELS

}  // namespace lbmk
