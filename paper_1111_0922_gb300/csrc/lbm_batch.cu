// Batched solver: many geometries in one set of arrays, advanced together.
//
// Every admitted geometry ("slot") is a node list (lexicographic fluid nodes,
// Sec. 1) stored as one segment of shared SoA arrays; the segment starts on a
// multiple of kAlign slots and holds the nodes and, for the esoteric twist,
// its ghost slots.  IDX entries are rebased to absolute slot numbers.  A step
// is one launch over the work chunks of all active segments; each block
// updates one chunk of one segment with that segment's omega, force and
// parity, so geometries admitted at different times coexist (continuous
// batching).  A round of K steps is replayed from a captured CUDA graph; its
// first step also reduces each segment's mass and flux (FP64) per chunk, and
// a per-segment pass sums the chunks in order.  The per-node arithmetic and
// the chunking relative to the segment start do not depend on the other
// segments, so a geometry gives bit-identical results alone and in a mix.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

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

// AA pattern over all segments: each block takes the parity of its segment.
template <class C, bool RED, int NPT>
__global__ void __launch_bounds__(256, C::kMinBlocks) k_batch_aa(BatchParams p) {
  using T = typename C::T;
  const auto A = batch_lattice<C>(p);
  const int2 w = p.work[blockIdx.x];
  const BatchSlot &sl = p.slots[w.x];
  const int64_t end = sl.start + sl.nodes;
  const bool odd = ((sl.steps + p.t) & 1) != 0;
  const CollK<T> K = make_collk<T>(T(sl.omega), T(sl.omega_m), T(sl.gx), T(sl.gy), T(sl.gz));
  double m = 0.0, j = 0.0;
#pragma unroll
  for (int r = 0; r < NPT; ++r) {
    const int64_t n64 = (int64_t)w.y + (int64_t)r * blockDim.x + threadIdx.x;
    if (n64 >= end) continue;
    const int s = (int)n64;
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
  if (RED) block_reduce_store(m, j, p.partials);
}

// Esoteric twist over all segments: the array map is the identity after an
// even step count and swaps opposite directions after an odd one.
template <class C, bool RED, int NPT>
__global__ void __launch_bounds__(256, C::kMinBlocks) k_batch_et(BatchParams p) {
  using T = typename C::T;
  const auto A = batch_lattice<C>(p);
  const int2 w = p.work[blockIdx.x];
  const BatchSlot &sl = p.slots[w.x];
  const int64_t end = sl.start + sl.nodes;
  const bool odd = ((sl.steps + p.t) & 1) != 0;
  const CollK<T> K = make_collk<T>(T(sl.omega), T(sl.omega_m), T(sl.gx), T(sl.gy), T(sl.gz));
  double m = 0.0, j = 0.0;
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
  if (RED) block_reduce_store(m, j, p.partials);
}

// Per-segment sums of its chunk partials, in chunk order (one thread each).
__global__ void k_batch_slot_sums(const BatchSlot *slots, int nslots, const double *partials, double *out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nslots) return;
  const BatchSlot &sl = slots[s];
  double m = 0.0, j = 0.0;
  if (sl.active) {
    for (int w = sl.first_work; w < sl.first_work + sl.nwork; ++w) {
      m += partials[2 * w];
      j += partials[2 * w + 1];
    }
  }
  out[2 * s] = m;
  out[2 * s + 1] = j;
}

// Copy a geometry's IDX (18 x ipad, node numbers or -1) or packed ET index
// (9 x ipad) into the batch arrays at `start`, rebased to absolute slots.
// folded (AA, capacity < 2^30): a solid link k of slot s becomes
// s + (opp(k) - k) npad, the slot the odd step's bounce-back reads and writes
// through IDX[k] (as for a single lattice, see k_fold_idx).
__global__ void k_batch_rebase(const int32_t *src, int64_t ipad, int rows, int64_t n, int32_t *dst, int64_t npad,
                               int64_t start, int packed, int folded) {
  const int64_t total = (int64_t)rows * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / n);
    const int64_t k = t % n;
    const int32_t v = src[(int64_t)r * ipad + k];
    int32_t o;
    if (packed)
      o = (int32_t)(((uint32_t)v & 0x80000000u) | (uint32_t)(((uint32_t)v & 0x7fffffffu) + (uint32_t)start));
    else if (v >= 0)
      o = (int32_t)(v + start);
    else if (folded)
      o = (int32_t)(start + k + (int64_t)(OPP(r + 1) - (r + 1)) * npad);
    else
      o = -1;
    dst[(int64_t)r * npad + start + k] = o;
  }
}

template <class C, bool RED, int NPT>
static void launch_batch_step_t(int variant, const BatchParams &p, int bs, cudaStream_t s) {
  if (variant == LBM_ET)
    k_batch_et<C, RED, NPT><<<p.nwork, bs, 0, s>>>(p);
  else
    k_batch_aa<C, RED, NPT><<<p.nwork, bs, 0, s>>>(p);
}

template <class C, bool RED>
static void launch_batch_npt(int variant, int npt, const BatchParams &p, int bs, cudaStream_t s) {
  switch (npt) {
    case 1: launch_batch_step_t<C, RED, 1>(variant, p, bs, s); break;
    case 2: launch_batch_step_t<C, RED, 2>(variant, p, bs, s); break;
    case 4: launch_batch_step_t<C, RED, 4>(variant, p, bs, s); break;
    default: launch_batch_step_t<C, RED, 8>(variant, p, bs, s); break;
  }
}

static void launch_batch_step(int precision, int variant, int npt, bool red, const BatchParams &p, int bs,
                              cudaStream_t s) {
  if (precision == LBM_F64) {
    if (red) launch_batch_npt<CodecF64, true>(variant, npt, p, bs, s);
    else launch_batch_npt<CodecF64, false>(variant, npt, p, bs, s);
  } else if (precision == LBM_F32) {
    if (red) launch_batch_npt<CodecF32, true>(variant, npt, p, bs, s);
    else launch_batch_npt<CodecF32, false>(variant, npt, p, bs, s);
  } else {
    if (red) launch_batch_npt<CodecF16S, true>(variant, npt, p, bs, s);
    else launch_batch_npt<CodecF16S, false>(variant, npt, p, bs, s);
  }
}

// Natural state of one AA-pattern segment (even step count) or ET segment.
template <class C>
__global__ void k_batch_get(BatchParams p, int slot, int variant, double *f_nat) {
  const auto A = batch_lattice<C>(p);
  const BatchSlot &sl = p.slots[slot];
  const bool odd = (sl.steps & 1) != 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < sl.nodes; k += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(sl.start + k);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      int arr = i, pos = s;
      if (variant == LBM_ET && i > 0) {
        arr = odd ? OPP(i) : i;
        if (!(i & 1)) pos = (int)((uint32_t)__ldg(p.idx + (int64_t)((i - 2) / 2) * p.npad + s) & 0x7fffffffu);
      }
      f_nat[(int64_t)i * sl.nodes + k] = WD(i) + (double)A.ld_dev(arr, pos);
    }
  }
}

}  // namespace lbmk

using namespace lbmk;

// ---------------------------------------------------------------------------
struct lbm_batch {
  lbm_batch_config cfg{};
  cudaStream_t stream = nullptr;
  std::string err;
  int64_t capacity = 0;  // slots per array (multiple of kAlign)
  bool folded = false;   // AA: bounce-back slots folded into IDX
  void *d_A = nullptr;
  int32_t *d_idx = nullptr;
  size_t state_bytes = 0, idx_bytes = 0;
  std::vector<std::pair<void *, size_t>> allocs;
  // host slot table and free list of [start, end) ranges
  std::vector<BatchSlot> slots;
  std::vector<int64_t> cells, ghosts;
  std::map<int64_t, int64_t> free_ranges;  // start -> end
  BatchSlot *d_slots = nullptr;
  BatchSlot *h_slots = nullptr;  // pinned mirror
  int slot_capacity = 0;
  int2 *d_work = nullptr;
  int work_capacity = 0;
  int nwork = 0;
  double *d_partials = nullptr;
  double *d_sums = nullptr, *h_sums = nullptr;  // pinned
  bool dirty = true;        // work list must be rebuilt
  cudaGraphExec_t graph = nullptr;
  int graph_k = -1, graph_nwork = -1, graph_bs = -1, graph_npt = -1;
  bool round_pending = false;
  int block_size = 256, npt = 1;
  float scale = 1.0f;
};

static std::string g_batch_error;

static lbm_status bfail(lbm_batch_t *b, lbm_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (b)
    b->err = buf;
  else
    g_batch_error = buf;
  return s;
}

#define BCUDA(b, call)                                                                              \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

static void *balloc(lbm_batch_t *b, size_t bytes, bool keep) {
  if (bytes == 0) bytes = 256;
  void *p = nullptr;
  if (b->cfg.dev_alloc) {
    p = b->cfg.dev_alloc(bytes, b->cfg.alloc_ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p && keep) b->allocs.emplace_back(p, bytes);
  return p;
}

static void bfree(lbm_batch_t *b, void *p, size_t bytes) {
  if (!p) return;
  if (b->cfg.dev_free)
    b->cfg.dev_free(p, bytes, b->cfg.alloc_ctx);
  else
    cudaFree(p);
}

static size_t pdf_bytes(int precision) { return precision == LBM_F64 ? 8 : (precision == LBM_F32 ? 4 : 2); }
static int idx_rows(int variant) { return variant == LBM_ET ? 9 : 18; }

extern "C" {

const char *lbm_batch_last_error(const lbm_batch_t *b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

int64_t lbm_batch_bytes_per_slot(int32_t variant, int32_t precision) {
  return (int64_t)Q * (int64_t)pdf_bytes(precision) + 4 * (int64_t)idx_rows(variant);
}

lbm_status lbm_batch_create(const lbm_batch_config *cfg, lbm_batch_t **out) {
  if (!cfg || !out) return bfail(nullptr, LBM_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (cfg->variant != LBM_AA && cfg->variant != LBM_ET)
    return bfail(nullptr, LBM_ERR_UNSUPPORTED, "batches run the AA pattern or the esoteric twist");
  if (cfg->precision < LBM_F64 || cfg->precision > LBM_F16S) return bfail(nullptr, LBM_ERR_INVALID_ARG, "precision");
  if (cfg->capacity_slots < kAlign || cfg->capacity_slots >= ((int64_t)1 << 31) - kAlign)
    return bfail(nullptr, LBM_ERR_INVALID_ARG, "capacity_slots must be in [4096, 2^31 - 8192)");
  if (cfg->max_geometries < 1 || cfg->max_geometries > 1 << 20)
    return bfail(nullptr, LBM_ERR_INVALID_ARG, "max_geometries");
  if (cfg->precision == LBM_F16S && !(cfg->f16_scale > 0.0))
    return bfail(nullptr, LBM_ERR_INVALID_ARG, "an FP16 batch needs f16_scale > 0 (a power of two)");
  if (cfg->dev_alloc && !cfg->dev_free) return bfail(nullptr, LBM_ERR_INVALID_ARG, "dev_alloc without dev_free");
  lbm_batch_t *b = new lbm_batch_t();
  b->cfg = *cfg;
  b->stream = static_cast<cudaStream_t>(cfg->stream);
  b->capacity = (cfg->capacity_slots + kAlign - 1) / kAlign * kAlign;
  b->folded = cfg->variant == LBM_AA && cfg->keep_idx == 0 && b->capacity < ((int64_t)1 << 30);
  b->scale = cfg->precision == LBM_F16S ? (float)cfg->f16_scale : 1.0f;
  b->block_size = cfg->block_size > 0 ? cfg->block_size : 256;
  b->npt = cfg->nodes_per_thread > 0 ? cfg->nodes_per_thread : 1;
  if (b->block_size % 32 || b->block_size > 256 || kAlign % (b->block_size * b->npt) ||
      (b->npt != 1 && b->npt != 2 && b->npt != 4 && b->npt != 8)) {
    delete b;
    return bfail(nullptr, LBM_ERR_INVALID_ARG, "block_size (<= 256) x nodes_per_thread (1,2,4,8) must divide 4096");
  }
  b->state_bytes = (size_t)Q * b->capacity * pdf_bytes(cfg->precision);
  b->idx_bytes = (size_t)idx_rows(cfg->variant) * b->capacity * 4;
  b->slot_capacity = cfg->max_geometries;
  b->work_capacity = (int)(b->capacity / 32) + cfg->max_geometries;
  b->d_A = balloc(b, b->state_bytes, true);
  b->d_idx = static_cast<int32_t *>(balloc(b, b->idx_bytes, true));
  b->d_slots = static_cast<BatchSlot *>(balloc(b, sizeof(BatchSlot) * b->slot_capacity, true));
  b->d_work = static_cast<int2 *>(balloc(b, sizeof(int2) * b->work_capacity, true));
  b->d_partials = static_cast<double *>(balloc(b, sizeof(double) * 2 * b->work_capacity, true));
  b->d_sums = static_cast<double *>(balloc(b, sizeof(double) * 2 * b->slot_capacity, true));
  bool ok = b->d_A && b->d_idx && b->d_slots && b->d_work && b->d_partials && b->d_sums;
  ok = ok && cudaMallocHost(&b->h_sums, sizeof(double) * 2 * b->slot_capacity) == cudaSuccess;
  ok = ok && cudaMallocHost(&b->h_slots, sizeof(BatchSlot) * b->slot_capacity) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    lbm_batch_destroy(b);
    return bfail(nullptr, LBM_ERR_OOM, "batch of %lld slots", (long long)b->capacity);
  }
  b->free_ranges[0] = b->capacity;
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_destroy(lbm_batch_t *b) {
  if (!b) return LBM_OK;
  cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (auto &a : b->allocs) bfree(b, a.first, a.second);
  if (b->h_sums) cudaFreeHost(b->h_sums);
  if (b->h_slots) cudaFreeHost(b->h_slots);
  delete b;
  return LBM_OK;
}

}  // extern "C"

// First-fit allocation of `len` slots from the free list.
static int64_t take_range(lbm_batch_t *b, int64_t len) {
  for (auto it = b->free_ranges.begin(); it != b->free_ranges.end(); ++it) {
    if (it->second - it->first >= len) {
      const int64_t start = it->first, end = it->second;
      b->free_ranges.erase(it);
      if (start + len < end) b->free_ranges[start + len] = end;
      return start;
    }
  }
  return -1;
}

static void give_range(lbm_batch_t *b, int64_t start, int64_t len) {
  int64_t s = start, e = start + len;
  auto next = b->free_ranges.lower_bound(s);
  if (next != b->free_ranges.end() && next->first == e) {
    e = next->second;
    b->free_ranges.erase(next);
  }
  auto prev = b->free_ranges.lower_bound(s);
  if (prev != b->free_ranges.begin()) {
    --prev;
    if (prev->second == s) {
      s = prev->first;
      b->free_ranges.erase(prev);
    }
  }
  b->free_ranges[s] = e;
}

// Rebuild the chunk list of all active segments and upload it with the table.
static lbm_status rebuild_work(lbm_batch_t *b) {
  std::vector<int2> work;
  const int64_t chunk = (int64_t)b->block_size * b->npt;
  for (size_t s = 0; s < b->slots.size(); ++s) {
    BatchSlot &sl = b->slots[s];
    sl.first_work = (int32_t)work.size();
    sl.nwork = 0;
    if (!sl.active) continue;
    for (int64_t k = 0; k < sl.nodes; k += chunk) {
      work.push_back(make_int2((int)s, (int)(sl.start + k)));
      ++sl.nwork;
    }
  }
  if ((int)work.size() > b->work_capacity) return bfail(b, LBM_ERR_OOM, "work list overflow");
  b->nwork = (int)work.size();
  if (!work.empty())
    BCUDA(b, cudaMemcpyAsync(b->d_work, work.data(), sizeof(int2) * work.size(), cudaMemcpyHostToDevice, b->stream));
  BCUDA(b, cudaStreamSynchronize(b->stream));
  b->dirty = false;
  return LBM_OK;
}

static lbm_status upload_slots(lbm_batch_t *b) {
  if (b->slots.empty()) return LBM_OK;
  memcpy(b->h_slots, b->slots.data(), sizeof(BatchSlot) * b->slots.size());
  BCUDA(b, cudaMemcpyAsync(b->d_slots, b->h_slots, sizeof(BatchSlot) * b->slots.size(), cudaMemcpyHostToDevice,
                           b->stream));
  return LBM_OK;
}

static BatchParams batch_params(const lbm_batch_t *b) {
  BatchParams p;
  p.A = b->d_A;
  p.npad = b->capacity;
  p.idx = b->d_idx;
  p.slots = b->d_slots;
  p.work = b->d_work;
  p.nwork = b->nwork;
  p.t = 0;
  p.scale = b->scale;
  p.inv_scale = 1.0f / b->scale;
  p.partials = b->d_partials;
  p.folded = b->folded ? 1 : 0;
  return p;
}

extern "C" {

lbm_status lbm_batch_admit_spheres(lbm_batch_t *b, const int32_t *dims, const int32_t *periodic, int64_t nsph,
                                   const int64_t *centres, int64_t radius, int64_t unit, double omega,
                                   const double *force, int32_t *slot_out) {
  if (!b || !dims || !periodic || !force || !slot_out) return bfail(b, LBM_ERR_INVALID_ARG, "NULL argument");
  if (b->round_pending) BCUDA(b, cudaStreamSynchronize(b->stream));
  const int nx = dims[0], ny = dims[1], nz = dims[2];
  for (int a = 0; a < 3; ++a)
    if (dims[a] < 1 || (periodic[a] && dims[a] < 2)) return bfail(b, LBM_ERR_INVALID_ARG, "box extents");
  if (!(omega > 0.0 && omega < 2.0)) return bfail(b, LBM_ERR_INVALID_ARG, "omega");
  if (nsph < 0 || (nsph > 0 && !centres) || unit < 1 || radius < 0) return bfail(b, LBM_ERR_INVALID_ARG, "spheres");
  const int64_t ncell = (int64_t)nx * ny * nz;
  if (ncell >= ((int64_t)1 << 30)) return bfail(b, LBM_ERR_INVALID_ARG, "box too large");
  // free slot-table entry
  int slot = -1;
  for (size_t s = 0; s < b->slots.size(); ++s)
    if (!b->slots[s].active) {
      slot = (int)s;
      break;
    }
  if (slot < 0) {
    if ((int)b->slots.size() >= b->slot_capacity) return bfail(b, LBM_ERR_OOM, "all %d geometry slots in use", b->slot_capacity);
    slot = (int)b->slots.size();
    b->slots.push_back(BatchSlot{});
    b->cells.push_back(0);
    b->ghosts.push_back(0);
  }
  // temporaries for the geometry build
  const int64_t ext = (int64_t)(nx + 2) * (ny + 2) * (nz + 2);
  const int64_t sc = scan_scratch_elems(std::max(ncell, ext));
  std::vector<std::pair<void *, size_t>> tmp;
  auto talloc = [&](size_t bytes) {
    void *p = balloc(b, bytes, false);
    if (p) tmp.emplace_back(p, bytes);
    return p;
  };
  auto cleanup = [&]() {
    cudaStreamSynchronize(b->stream);
    for (auto &a : tmp) bfree(b, a.first, a.second);
    tmp.clear();
  };
  uint8_t *solid = static_cast<uint8_t *>(talloc(ncell));
  int32_t *node_of = static_cast<int32_t *>(talloc(4 * ncell));
  int32_t *cells = static_cast<int32_t *>(talloc(4 * ncell));
  int32_t *scratch = static_cast<int32_t *>(talloc(4 * sc));
  int64_t *dcen = nsph > 0 ? static_cast<int64_t *>(talloc(sizeof(int64_t) * 3 * nsph)) : nullptr;
  if (!solid || !node_of || !cells || !scratch || (nsph > 0 && !dcen)) {
    cleanup();
    return bfail(b, LBM_ERR_OOM, "geometry temporaries");
  }
  cudaMemsetAsync(solid, 0, ncell, b->stream);
  if (nsph > 0) {
    cudaMemcpyAsync(dcen, centres, sizeof(int64_t) * 3 * nsph, cudaMemcpyHostToDevice, b->stream);
    launch_sphere_mask(solid, nx, ny, nz, periodic, nsph, dcen, radius, unit, b->stream);
  }
  const int64_t N = build_node_list(solid, ncell, node_of, cells, scratch, sc, b->stream);
  if (N < 0) {
    cleanup();
    return bfail(b, LBM_ERR_CUDA, "node list");
  }
  const int64_t ipad = std::max<int64_t>(64, (N + 63) / 64 * 64);
  const int rows = idx_rows(b->cfg.variant);
  int32_t *idx = static_cast<int32_t *>(talloc(sizeof(int32_t) * 18 * ipad));
  if (!idx) {
    cleanup();
    return bfail(b, LBM_ERR_OOM, "IDX temporaries");
  }
  launch_build_idx(cells, node_of, N, nx, ny, nz, periodic, idx, ipad, b->stream);
  int64_t G = 0;
  int32_t *src_idx = idx;
  if (b->cfg.variant == LBM_ET) {
    int32_t *ghost = static_cast<int32_t *>(talloc(sizeof(int32_t) * ext));
    int32_t *et = static_cast<int32_t *>(talloc(sizeof(int32_t) * 9 * ipad));
    if (!ghost || !et) {
      cleanup();
      return bfail(b, LBM_ERR_OOM, "ET temporaries");
    }
    G = build_et_index(cells, node_of, N, nx, ny, nz, periodic, ghost, et, ipad, scratch, sc, b->stream);
    src_idx = et;
  }
  const int64_t len = std::max<int64_t>(kAlign, (N + G + kAlign - 1) / kAlign * kAlign);
  const int64_t start = take_range(b, len);
  if (start < 0) {
    cleanup();
    return bfail(b, LBM_ERR_OOM, "no free range of %lld slots (geometry of %lld fluid nodes)", (long long)len,
                 (long long)N);
  }
  if (N > 0)
    k_batch_rebase<<<(unsigned)std::min<int64_t>((rows * N + 255) / 256, 1 << 20), 256, 0, b->stream>>>(
        src_idx, ipad, rows, N, b->d_idx, b->capacity, start, b->cfg.variant == LBM_ET, b->folded ? 1 : 0);
  // rest state: every deviation zero, the segment's ghosts included
  const size_t es = pdf_bytes(b->cfg.precision);
  for (int i = 0; i < Q; ++i)
    cudaMemsetAsync(static_cast<char *>(b->d_A) + ((int64_t)i * b->capacity + start) * es, 0, len * es, b->stream);
  cudaError_t e = cudaGetLastError();
  cleanup();
  if (e != cudaSuccess) {
    give_range(b, start, len);
    return bfail(b, LBM_ERR_CUDA, "admission kernels: %s", cudaGetErrorString(e));
  }
  BatchSlot &sl = b->slots[slot];
  memset(&sl, 0, sizeof sl);
  sl.omega = omega;
  sl.omega_m = omega;
  sl.gx = force[0];
  sl.gy = force[1];
  sl.gz = force[2];
  sl.start = start;
  sl.nodes = N;
  sl.steps = 0;
  sl.active = 1;
  b->cells[slot] = ncell;
  b->ghosts[slot] = len;  // reserved length
  b->dirty = true;
  *slot_out = slot;
  return LBM_OK;
}

lbm_status lbm_batch_release(lbm_batch_t *b, int32_t slot) {
  if (!b) return bfail(nullptr, LBM_ERR_INVALID_ARG, "NULL batch");
  if (slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].active)
    return bfail(b, LBM_ERR_INVALID_ARG, "slot %d is not in use", slot);
  if (b->round_pending) BCUDA(b, cudaStreamSynchronize(b->stream));
  give_range(b, b->slots[slot].start, b->ghosts[slot]);
  b->slots[slot].active = 0;
  b->dirty = true;
  return LBM_OK;
}

// Capture K steps (the first reducing) and the per-slot sums into a graph.
static lbm_status capture_round(lbm_batch_t *b, int k) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaStream_t cs;
  BCUDA(b, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    BatchParams p = batch_params(b);
    for (int t = 0; t < k; ++t) {
      p.t = t;
      launch_batch_step(b->cfg.precision, b->cfg.variant, b->npt, t == 0, p, b->block_size, cs);
      if (t == 0)
        k_batch_slot_sums<<<((int)b->slots.size() + 127) / 128, 128, 0, cs>>>(b->d_slots, (int)b->slots.size(),
                                                                                b->d_partials, b->d_sums);
    }
    cudaMemcpyAsync(b->h_sums, b->d_sums, sizeof(double) * 2 * b->slots.size(), cudaMemcpyDeviceToHost, cs);
    e = cudaStreamEndCapture(cs, &g);
  }
  if (e == cudaSuccess) {
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
  }
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "round graph: %s", cudaGetErrorString(e));
  b->graph_k = k;
  b->graph_nwork = b->nwork;
  b->graph_bs = b->block_size;
  b->graph_npt = b->npt;
  return LBM_OK;
}

lbm_status lbm_batch_round(lbm_batch_t *b, int32_t k) {
  if (!b) return bfail(nullptr, LBM_ERR_INVALID_ARG, "NULL batch");
  if (k < 1) return bfail(b, LBM_ERR_INVALID_ARG, "k_steps must be >= 1");
  if (b->round_pending) BCUDA(b, cudaStreamSynchronize(b->stream));
  b->round_pending = false;
  bool rebuilt = false;
  if (b->dirty) {
    lbm_status st = rebuild_work(b);
    if (st != LBM_OK) return st;
    rebuilt = true;
  }
  lbm_status st = upload_slots(b);
  if (st != LBM_OK) return st;
  if (b->nwork == 0) return LBM_OK;
  if (!b->graph || rebuilt || b->graph_k != k || b->graph_nwork != b->nwork || b->graph_bs != b->block_size ||
      b->graph_npt != b->npt) {
    st = capture_round(b, k);
    if (st != LBM_OK) return st;
  }
  BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
  for (auto &sl : b->slots)
    if (sl.active) sl.steps += k;
  b->round_pending = true;
  return LBM_OK;
}

lbm_status lbm_batch_poll(lbm_batch_t *b, int32_t slot, double *mass, double *flux, int64_t *steps) {
  if (!b) return bfail(nullptr, LBM_ERR_INVALID_ARG, "NULL batch");
  if (slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].active)
    return bfail(b, LBM_ERR_INVALID_ARG, "slot %d is not in use", slot);
  if (b->round_pending) {
    BCUDA(b, cudaStreamSynchronize(b->stream));
    b->round_pending = false;
  }
  if (mass) *mass = b->h_sums[2 * slot];
  if (flux) *flux = b->h_sums[2 * slot + 1];
  if (steps) *steps = b->slots[slot].steps;
  return LBM_OK;
}

lbm_status lbm_batch_slot_info(lbm_batch_t *b, int32_t slot, int64_t *nodes, int64_t *cells, int64_t *steps) {
  if (!b) return bfail(nullptr, LBM_ERR_INVALID_ARG, "NULL batch");
  if (slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].active)
    return bfail(b, LBM_ERR_INVALID_ARG, "slot %d is not in use", slot);
  if (nodes) *nodes = b->slots[slot].nodes;
  if (cells) *cells = b->cells[slot];
  if (steps) *steps = b->slots[slot].steps;
  return LBM_OK;
}

lbm_status lbm_batch_get_info(lbm_batch_t *b, lbm_batch_info *info) {
  if (!b || !info) return bfail(b, LBM_ERR_INVALID_ARG, "NULL argument");
  memset(info, 0, sizeof *info);
  info->capacity_slots = b->capacity;
  int64_t free_slots = 0, largest = 0;
  for (auto &r : b->free_ranges) {
    free_slots += r.second - r.first;
    largest = std::max(largest, r.second - r.first);
  }
  info->free_slots = free_slots;
  info->largest_free = largest;
  for (auto &sl : b->slots)
    if (sl.active) {
      info->active_geometries += 1;
      info->active_nodes += sl.nodes;
    }
  info->device_bytes = (int64_t)(b->state_bytes + b->idx_bytes);
  info->block_size = b->block_size;
  info->nodes_per_thread = b->npt;
  info->work_chunks = b->nwork;
  return LBM_OK;
}

lbm_status lbm_batch_get_pdfs(lbm_batch_t *b, int32_t slot, double *f_host) {
  if (!b || !f_host) return bfail(b, LBM_ERR_INVALID_ARG, "NULL argument");
  if (slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].active)
    return bfail(b, LBM_ERR_INVALID_ARG, "slot %d is not in use", slot);
  const BatchSlot sl = b->slots[slot];
  if (b->cfg.variant == LBM_AA && (sl.steps & 1))
    return bfail(b, LBM_ERR_STATE, "AA pattern state is natural only after an even step count");
  if (b->round_pending) BCUDA(b, cudaStreamSynchronize(b->stream));
  b->round_pending = false;
  lbm_status st = upload_slots(b);
  if (st != LBM_OK) return st;
  const size_t bytes = sizeof(double) * Q * std::max<int64_t>(sl.nodes, 1);
  double *tmp = static_cast<double *>(balloc(b, bytes, false));
  if (!tmp) return bfail(b, LBM_ERR_OOM, "read-out buffer");
  BatchParams p = batch_params(b);
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((sl.nodes + 255) / 256, 1 << 20));
  if (b->cfg.precision == LBM_F64)
    k_batch_get<CodecF64><<<grid, 256, 0, b->stream>>>(p, slot, b->cfg.variant, tmp);
  else if (b->cfg.precision == LBM_F32)
    k_batch_get<CodecF32><<<grid, 256, 0, b->stream>>>(p, slot, b->cfg.variant, tmp);
  else
    k_batch_get<CodecF16S><<<grid, 256, 0, b->stream>>>(p, slot, b->cfg.variant, tmp);
  cudaError_t e = cudaMemcpyAsync(f_host, tmp, sizeof(double) * Q * sl.nodes, cudaMemcpyDeviceToHost, b->stream);
  cudaError_t e2 = cudaStreamSynchronize(b->stream);
  bfree(b, tmp, bytes);
  if (e != cudaSuccess || e2 != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "read-out");
  return LBM_OK;
}

// Launch-shape autotuner: time `rounds` rounds of k steps of the current
// batch for each (block size, nodes per thread) candidate with CUDA events,
// keep the fastest.  The state advances by rounds * k steps per candidate.
lbm_status lbm_batch_tune(lbm_batch_t *b, int32_t rounds, int32_t k, int32_t *best_bs, int32_t *best_npt,
                          double *best_mflups) {
  if (!b || rounds < 1 || k < 1) return bfail(b, LBM_ERR_INVALID_ARG, "tune arguments");
  static const int cand[][2] = {{128, 1}, {256, 1}, {128, 2}, {256, 2}, {128, 4}, {256, 4}, {64, 2}, {64, 4}};
  int64_t active = 0;
  for (auto &sl : b->slots)
    if (sl.active) active += sl.nodes;
  if (active == 0) return bfail(b, LBM_ERR_STATE, "no active geometry to tune on");
  double best = -1.0;
  int bb = b->block_size, bn = b->npt;
  cudaEvent_t e0, e1;
  BCUDA(b, cudaEventCreate(&e0));
  BCUDA(b, cudaEventCreate(&e1));
  for (auto &c : cand) {
    b->block_size = c[0];
    b->npt = c[1];
    b->dirty = true;
    lbm_status st = lbm_batch_round(b, k);  // warm-up and graph capture
    if (st != LBM_OK) return st;
    BCUDA(b, cudaStreamSynchronize(b->stream));
    b->round_pending = false;
    cudaEventRecord(e0, b->stream);
    for (int r = 0; r < rounds; ++r) {
      st = lbm_batch_round(b, k);
      if (st != LBM_OK) return st;
    }
    cudaEventRecord(e1, b->stream);
    BCUDA(b, cudaEventSynchronize(e1));
    b->round_pending = false;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double mflups = (double)active * rounds * k / (ms * 1e-3) / 1e6;
    if (mflups > best) {
      best = mflups;
      bb = c[0];
      bn = c[1];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->block_size = bb;
  b->npt = bn;
  b->dirty = true;
  if (best_bs) *best_bs = bb;
  if (best_npt) *best_npt = bn;
  if (best_mflups) *best_mflups = best;
  return LBM_OK;
}

}  // extern "C"
