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

#include "lbm_batch.cuh"

namespace lbmk {

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

// mode 0: one step (p.t), reducing when red; mode 1: k steps in one
// persistent launch (step 0 reduces).
static cudaError_t launch_batch(int precision, int variant, int mode, int npt, bool red, const BatchParams &p, int bs,
                                int k, unsigned *count, int *err, uint64_t limit_ns, int nsm, cudaStream_t s) {
  if (precision == LBM_F64)
    return launch_batch_t<CodecF64>(variant, mode, npt, red, p, bs, k, count, err, limit_ns, nsm, s);
  if (precision == LBM_F32)
    return launch_batch_t<CodecF32>(variant, mode, npt, red, p, bs, k, count, err, limit_ns, nsm, s);
  return launch_batch_t<CodecF16S>(variant, mode, npt, red, p, bs, k, count, err, limit_ns, nsm, s);
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
// Host record of an admitted geometry: its description (kept so that the
// autotuner can rebuild the segment for another variant) and the state of
// its steady-flux test.
struct SlotHost {
  int32_t dims[3] = {0, 0, 0}, periodic[3] = {0, 0, 0};
  std::vector<uint8_t> mask;      // mask admission: nx*ny*nz bytes, nonzero = solid
  std::vector<int64_t> centres;   // sphere admission: nsph x 3
  int64_t radius = 0, unit = 1;
  bool spheres = false;
  int64_t cells = 0;              // nx*ny*nz
  int64_t reserved = 0;           // slots of the segment (nodes, ghosts, alignment)
  double tol = 0.0;               // relative flux change that counts as steady
  int64_t max_steps = 0;          // step cap (<= 0: none)
  double mass = 0.0, flux = 0.0;  // of the state the last settled round started from
  double prev_flux = 0.0;
  bool have_prev = false;
  int32_t done = 0;               // 0 running, 1 converged, 2 stopped at max_steps
  int64_t first_round = 0;        // first round whose results belong to this geometry
};

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
  std::vector<SlotHost> host;              // per slot: geometry, convergence record
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
  int64_t rounds_launched = 0;  // rounds enqueued so far
  int64_t rounds_settled = 0;   // rounds whose results are folded into the records
  cudaStream_t admit_stream = nullptr;  // geometry builds, overlapping a round in flight
  cudaEvent_t admit_done = nullptr;     // the next round waits for the last admission
  bool admit_pending = false;
  int block_size = 256, npt = 1;
  int variant = LBM_AA;  // current variant (the tuner may switch it)
  int round_mode = 0;    // 0 per-step launches, 1 one persistent launch per round
  int graph_mode = -1;
  int nsm = 1;
  unsigned *d_count = nullptr;  // grid barrier of the persistent round
  int *d_err = nullptr, *h_err = nullptr;  // its timeout flag (pinned copy)
  float scale = 1.0f;
};

// A persistent round's grid barrier gives up after this long (a round
// step takes milliseconds; the wait exists to turn a lost block into an
// error instead of a hang).
constexpr uint64_t kBarrierLimitNs = 2000000000ull;

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
  // a batch whose variant may be tuned sizes its index for LBM_AA
  return (int64_t)Q * (int64_t)pdf_bytes(precision) + 4 * (int64_t)idx_rows(variant);
}

lbm_status lbm_batch_create(const lbm_batch_config *cfg, lbm_batch_t **out) {
  if (!cfg || !out) return bfail(nullptr, LBM_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (cfg->variant != LBM_AA && cfg->variant != LBM_ET)
    return bfail(nullptr, LBM_ERR_UNSUPPORTED, "batches run the AA pattern or the esoteric twist");
  if (cfg->round_mode != 0 && cfg->round_mode != 1) return bfail(nullptr, LBM_ERR_INVALID_ARG, "round_mode");
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
  b->variant = cfg->variant;
  b->round_mode = cfg->round_mode;
  b->folded = cfg->variant == LBM_AA && cfg->keep_idx == 0 && b->capacity < ((int64_t)1 << 30);
  b->scale = cfg->precision == LBM_F16S ? (float)cfg->f16_scale : 1.0f;
  b->block_size = cfg->block_size > 0 ? cfg->block_size : 256;
  b->npt = cfg->nodes_per_thread > 0 ? cfg->nodes_per_thread : 1;
  if ((b->block_size != 64 && b->block_size != 128 && b->block_size != 256 && b->block_size != 512) ||
      kAlign % (b->block_size * b->npt) || (b->npt != 1 && b->npt != 2 && b->npt != 4 && b->npt != 8)) {
    delete b;
    return bfail(nullptr, LBM_ERR_INVALID_ARG, "block_size (64..512) x nodes_per_thread (1,2,4,8) must divide 4096");
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  b->state_bytes = (size_t)Q * b->capacity * pdf_bytes(cfg->precision);
  b->idx_bytes = (size_t)(cfg->tune_variant ? 18 : idx_rows(cfg->variant)) * b->capacity * 4;
  b->slot_capacity = cfg->max_geometries;
  b->work_capacity = (int)(b->capacity / 32) + cfg->max_geometries;
  b->d_A = balloc(b, b->state_bytes, true);
  b->d_idx = static_cast<int32_t *>(balloc(b, b->idx_bytes, true));
  b->d_slots = static_cast<BatchSlot *>(balloc(b, sizeof(BatchSlot) * b->slot_capacity, true));
  b->d_work = static_cast<int2 *>(balloc(b, sizeof(int2) * b->work_capacity, true));
  b->d_partials = static_cast<double *>(balloc(b, sizeof(double) * 2 * b->work_capacity, true));
  b->d_sums = static_cast<double *>(balloc(b, sizeof(double) * 2 * b->slot_capacity, true));
  b->d_count = static_cast<unsigned *>(balloc(b, 256, true));
  b->d_err = static_cast<int *>(balloc(b, 256, true));
  bool ok = b->d_A && b->d_idx && b->d_slots && b->d_work && b->d_partials && b->d_sums && b->d_count && b->d_err;
  ok = ok && cudaMemset(b->d_err, 0, sizeof(int)) == cudaSuccess;
  ok = ok && cudaMallocHost(&b->h_err, sizeof(int)) == cudaSuccess;
  if (ok) *b->h_err = 0;
  ok = ok && cudaMallocHost(&b->h_sums, sizeof(double) * 2 * b->slot_capacity) == cudaSuccess;
  ok = ok && cudaMallocHost(&b->h_slots, sizeof(BatchSlot) * b->slot_capacity) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&b->admit_stream, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&b->admit_done, cudaEventDisableTiming) == cudaSuccess;
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
  if (b->admit_stream) cudaStreamSynchronize(b->admit_stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->admit_done) cudaEventDestroy(b->admit_done);
  if (b->admit_stream) cudaStreamDestroy(b->admit_stream);
  for (auto &a : b->allocs) bfree(b, a.first, a.second);
  if (b->h_sums) cudaFreeHost(b->h_sums);
  if (b->h_slots) cudaFreeHost(b->h_slots);
  if (b->h_err) cudaFreeHost(b->h_err);
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

// Fold the results of every completed round into the slot records: the
// relative flux change between consecutive rounds (each round reduces the
// state it starts from) decides convergence, as in the single-lattice solve.
static lbm_status settle(lbm_batch_t *b) {
  if (b->round_pending) {
    BCUDA(b, cudaStreamSynchronize(b->stream));
    b->round_pending = false;
    if (*b->h_err) {
      *b->h_err = 0;
      b->rounds_settled = b->rounds_launched;
      return bfail(b, LBM_ERR_TIMEOUT, "a persistent round's grid barrier gave up; its results are invalid");
    }
  }
  if (b->rounds_settled == b->rounds_launched) return LBM_OK;
  for (size_t s = 0; s < b->slots.size(); ++s) {
    const BatchSlot &sl = b->slots[s];
    SlotHost &h = b->host[s];
    if (!sl.active || h.first_round > b->rounds_launched - 1) continue;
    h.mass = b->h_sums[2 * s];
    h.flux = b->h_sums[2 * s + 1];
    if (h.done) continue;
    const bool steady = h.have_prev && std::fabs(h.flux - h.prev_flux) < h.tol * std::fabs(h.flux);
    h.prev_flux = h.flux;
    h.have_prev = true;
    if (steady)
      h.done = 1;
    else if (h.max_steps > 0 && sl.steps >= h.max_steps)
      h.done = 2;
  }
  b->rounds_settled = b->rounds_launched;
  return LBM_OK;
}

// Darcy permeability k = nu <rho u_x> / g_x, the average over every cell of
// the box (superficial velocity), nu = (1/omega - 1/2) / 3 (lattice units).
static double permeability_of(double flux, int64_t cells, double omega, double gx) {
  const double nu = (1.0 / omega - 0.5) / 3.0;
  return gx != 0.0 && cells > 0 ? nu * (flux / (double)cells) / gx : NAN;
}

// Build geometry `slot` (its host record filled) for the batch's variant:
// solid mask on the device (uploaded or from spheres), node list, IDX or the
// esoteric twist's packed index, a free range, the rebased index and the
// rest state, all on the admission stream (a round in flight touches only
// the ranges of active geometries, so the two overlap).  Fills sl.start,
// sl.nodes and host.reserved.
static lbm_status build_segment(lbm_batch_t *b, int slot) {
  SlotHost &h = b->host[slot];
  BatchSlot &sl = b->slots[slot];
  cudaStream_t st = b->admit_stream;
  const int nx = h.dims[0], ny = h.dims[1], nz = h.dims[2];
  const int64_t ncell = (int64_t)nx * ny * nz;
  const int64_t nsph = h.spheres ? (int64_t)h.centres.size() / 3 : 0;
  const int64_t ext = (int64_t)(nx + 2) * (ny + 2) * (nz + 2);
  const int64_t sc = scan_scratch_elems(std::max(ncell, ext));
  std::vector<std::pair<void *, size_t>> tmp;
  auto talloc = [&](size_t bytes) {
    void *p = balloc(b, bytes, false);
    if (p) tmp.emplace_back(p, bytes);
    return p;
  };
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
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
  if (h.spheres) {
    cudaMemsetAsync(solid, 0, ncell, st);
    if (nsph > 0) {
      cudaMemcpyAsync(dcen, h.centres.data(), sizeof(int64_t) * 3 * nsph, cudaMemcpyHostToDevice, st);
      launch_sphere_mask(solid, nx, ny, nz, h.periodic, nsph, dcen, h.radius, h.unit, st);
    }
  } else {
    cudaMemcpyAsync(solid, h.mask.data(), ncell, cudaMemcpyHostToDevice, st);
  }
  const int64_t N = build_node_list(solid, ncell, node_of, cells, scratch, sc, st);
  if (N < 0) {
    cleanup();
    return bfail(b, LBM_ERR_CUDA, "node list");
  }
  const int64_t ipad = std::max<int64_t>(64, (N + 63) / 64 * 64);
  const int rows = idx_rows(b->variant);
  int32_t *idx = static_cast<int32_t *>(talloc(sizeof(int32_t) * 18 * ipad));
  if (!idx) {
    cleanup();
    return bfail(b, LBM_ERR_OOM, "IDX temporaries");
  }
  launch_build_idx(cells, node_of, N, nx, ny, nz, h.periodic, idx, ipad, st);
  int64_t G = 0;
  int32_t *src_idx = idx;
  if (b->variant == LBM_ET) {
    int32_t *ghost = static_cast<int32_t *>(talloc(sizeof(int32_t) * ext));
    int32_t *et = static_cast<int32_t *>(talloc(sizeof(int32_t) * 9 * ipad));
    if (!ghost || !et) {
      cleanup();
      return bfail(b, LBM_ERR_OOM, "ET temporaries");
    }
    G = build_et_index(cells, node_of, N, nx, ny, nz, h.periodic, ghost, et, ipad, scratch, sc, st);
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
    k_batch_rebase<<<(unsigned)std::min<int64_t>((rows * N + 255) / 256, 1 << 20), 256, 0, st>>>(
        src_idx, ipad, rows, N, b->d_idx, b->capacity, start, b->variant == LBM_ET, b->folded ? 1 : 0);
  // rest state: every deviation zero, the segment's ghosts included
  const size_t es = pdf_bytes(b->cfg.precision);
  for (int i = 0; i < Q; ++i)
    cudaMemsetAsync(static_cast<char *>(b->d_A) + ((int64_t)i * b->capacity + start) * es, 0, len * es, st);
  cudaError_t e = cudaEventRecord(b->admit_done, st);
  if (e == cudaSuccess) e = cudaGetLastError();
  cleanup();
  if (e != cudaSuccess) {
    give_range(b, start, len);
    return bfail(b, LBM_ERR_CUDA, "admission kernels: %s", cudaGetErrorString(e));
  }
  b->admit_pending = true;
  sl.start = start;
  sl.nodes = N;
  h.reserved = len;
  return LBM_OK;
}

// Admission common to masks and sphere packs: validate, take a table entry,
// build the segment, set the slot's parameters (at rest, step 0).
static lbm_status admit(lbm_batch_t *b, SlotHost &&h, double omega, const double *force, int32_t *slot_out) {
  for (int a = 0; a < 3; ++a)
    if (h.dims[a] < 1 || (h.periodic[a] && h.dims[a] < 2)) return bfail(b, LBM_ERR_INVALID_ARG, "box extents");
  if (!(omega > 0.0 && omega < 2.0)) return bfail(b, LBM_ERR_INVALID_ARG, "omega");
  if (!(h.tol >= 0.0)) return bfail(b, LBM_ERR_INVALID_ARG, "tol must be >= 0");
  h.cells = (int64_t)h.dims[0] * h.dims[1] * h.dims[2];
  if (h.cells >= ((int64_t)1 << 30)) return bfail(b, LBM_ERR_INVALID_ARG, "box too large");
  // a release or the previous admission may still be pending on the host side
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
    b->host.push_back(SlotHost{});
  }
  b->host[slot] = std::move(h);
  BatchSlot &sl = b->slots[slot];
  memset(&sl, 0, sizeof sl);
  lbm_status st = build_segment(b, slot);
  if (st != LBM_OK) return st;
  sl.omega = omega;
  sl.omega_m = omega;
  sl.gx = force[0];
  sl.gy = force[1];
  sl.gz = force[2];
  sl.steps = 0;
  sl.active = 1;
  // results of the round in flight (if any) do not belong to this geometry
  b->host[slot].first_round = b->rounds_launched;
  b->dirty = true;
  *slot_out = slot;
  return LBM_OK;
}

extern "C" {

lbm_status lbm_batch_admit(lbm_batch_t *b, const uint8_t *mask, int32_t nx, int32_t ny, int32_t nz,
                           const int32_t *periodic, double omega, const double *force, double tol, int64_t max_steps,
                           int32_t *slot_out) {
  if (!b || !mask || !periodic || !force || !slot_out) return bfail(b, LBM_ERR_INVALID_ARG, "NULL argument");
  if (nx < 1 || ny < 1 || nz < 1 || (int64_t)nx * ny * nz >= ((int64_t)1 << 30))
    return bfail(b, LBM_ERR_INVALID_ARG, "box extents");
  SlotHost h;
  h.dims[0] = nx;
  h.dims[1] = ny;
  h.dims[2] = nz;
  for (int a = 0; a < 3; ++a) h.periodic[a] = periodic[a] ? 1 : 0;
  h.mask.assign(mask, mask + (int64_t)nx * ny * nz);
  h.tol = tol;
  h.max_steps = max_steps;
  return admit(b, std::move(h), omega, force, slot_out);
}

lbm_status lbm_batch_admit_spheres(lbm_batch_t *b, const int32_t *dims, const int32_t *periodic, int64_t nsph,
                                   const int64_t *centres, int64_t radius, int64_t unit, double omega,
                                   const double *force, double tol, int64_t max_steps, int32_t *slot_out) {
  if (!b || !dims || !periodic || !force || !slot_out) return bfail(b, LBM_ERR_INVALID_ARG, "NULL argument");
  if (nsph < 0 || (nsph > 0 && !centres) || unit < 1 || radius < 0) return bfail(b, LBM_ERR_INVALID_ARG, "spheres");
  SlotHost h;
  for (int a = 0; a < 3; ++a) {
    h.dims[a] = dims[a];
    h.periodic[a] = periodic[a] ? 1 : 0;
  }
  h.spheres = true;
  if (nsph > 0) h.centres.assign(centres, centres + 3 * nsph);
  h.radius = radius;
  h.unit = unit;
  h.tol = tol;
  h.max_steps = max_steps;
  return admit(b, std::move(h), omega, force, slot_out);
}

lbm_status lbm_batch_release(lbm_batch_t *b, int32_t slot) {
  if (!b) return bfail(nullptr, LBM_ERR_INVALID_ARG, "NULL batch");
  if (slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].active)
    return bfail(b, LBM_ERR_INVALID_ARG, "slot %d is not in use", slot);
  // the range may be in use by a round in flight: finish it first
  lbm_status st = settle(b);
  if (st != LBM_OK) return st;
  give_range(b, b->slots[slot].start, b->host[slot].reserved);
  b->slots[slot].active = 0;
  b->host[slot] = SlotHost{};
  b->dirty = true;
  return LBM_OK;
}

// Capture a round into a graph: K steps (the first reducing) as K launches
// (round_mode 0) or one persistent cooperative launch (round_mode 1), the
// per-slot sums and their copy (with the barrier's timeout flag) to pinned
// host memory.
static lbm_status capture_round(lbm_batch_t *b, int k) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaStream_t cs;
  BCUDA(b, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g;
  cudaError_t le = cudaSuccess;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    BatchParams p = batch_params(b);
    const int nslots = (int)b->slots.size();
    if (b->round_mode == 1) {
      cudaMemsetAsync(b->d_count, 0, sizeof(unsigned), cs);
      cudaMemsetAsync(b->d_err, 0, sizeof(int), cs);
      le = launch_batch(b->cfg.precision, b->variant, 1, b->npt, true, p, b->block_size, k, b->d_count, b->d_err,
                        kBarrierLimitNs, b->nsm, cs);
      k_batch_slot_sums<<<(nslots + 127) / 128, 128, 0, cs>>>(b->d_slots, nslots, b->d_partials, b->d_sums);
    } else {
      for (int t = 0; t < k && le == cudaSuccess; ++t) {
        p.t = t;
        le = launch_batch(b->cfg.precision, b->variant, 0, b->npt, t == 0, p, b->block_size, 1, nullptr, nullptr, 0,
                          b->nsm, cs);
        if (t == 0)
          k_batch_slot_sums<<<(nslots + 127) / 128, 128, 0, cs>>>(b->d_slots, nslots, b->d_partials, b->d_sums);
      }
    }
    cudaMemcpyAsync(b->h_sums, b->d_sums, sizeof(double) * 2 * nslots, cudaMemcpyDeviceToHost, cs);
    cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, cs);
    e = cudaStreamEndCapture(cs, &g);
    if (le != cudaSuccess && e == cudaSuccess) {
      cudaGraphDestroy(g);
      e = le;
    } else if (e == cudaSuccess) {
      e = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
    }
  }
  cudaStreamDestroy(cs);
  cudaGetLastError();
  if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "round graph (mode %d): %s", b->round_mode, cudaGetErrorString(e));
  b->graph_k = k;
  b->graph_nwork = b->nwork;
  b->graph_bs = b->block_size;
  b->graph_npt = b->npt;
  b->graph_mode = b->round_mode;
  return LBM_OK;
}

lbm_status lbm_batch_round(lbm_batch_t *b, int32_t k) {
  if (!b) return bfail(nullptr, LBM_ERR_INVALID_ARG, "NULL batch");
  if (k < 1) return bfail(b, LBM_ERR_INVALID_ARG, "k_steps must be >= 1");
  lbm_status st0 = settle(b);
  if (st0 != LBM_OK) return st0;
  if (b->admit_pending) {  // segments built on the admission stream
    BCUDA(b, cudaStreamWaitEvent(b->stream, b->admit_done, 0));
    b->admit_pending = false;
  }
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
      b->graph_npt != b->npt || b->graph_mode != b->round_mode) {
    st = capture_round(b, k);
    if (st != LBM_OK) return st;
  }
  BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
  for (auto &sl : b->slots)
    if (sl.active) sl.steps += k;
  b->round_pending = true;
  b->rounds_launched += 1;
  return LBM_OK;
}

lbm_status lbm_batch_flux(lbm_batch_t *b, int32_t slot, double *mass, double *flux, int64_t *steps) {
  if (!b) return bfail(nullptr, LBM_ERR_INVALID_ARG, "NULL batch");
  if (slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].active)
    return bfail(b, LBM_ERR_INVALID_ARG, "slot %d is not in use", slot);
  lbm_status st = settle(b);
  if (st != LBM_OK) return st;
  if (mass) *mass = b->host[slot].mass;
  if (flux) *flux = b->host[slot].flux;
  if (steps) *steps = b->slots[slot].steps;
  return LBM_OK;
}

lbm_status lbm_batch_poll(lbm_batch_t *b, int32_t slot, int32_t *done, double *permeability, int64_t *steps) {
  if (!b) return bfail(nullptr, LBM_ERR_INVALID_ARG, "NULL batch");
  if (slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].active)
    return bfail(b, LBM_ERR_INVALID_ARG, "slot %d is not in use", slot);
  lbm_status st = settle(b);
  if (st != LBM_OK) return st;
  const BatchSlot &sl = b->slots[slot];
  const SlotHost &h = b->host[slot];
  if (done) *done = h.done;
  if (permeability) *permeability = permeability_of(h.flux, h.cells, sl.omega, sl.gx);
  if (steps) *steps = sl.steps;
  return LBM_OK;
}

lbm_status lbm_batch_slot_info(lbm_batch_t *b, int32_t slot, int64_t *nodes, int64_t *cells, int64_t *steps) {
  if (!b) return bfail(nullptr, LBM_ERR_INVALID_ARG, "NULL batch");
  if (slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].active)
    return bfail(b, LBM_ERR_INVALID_ARG, "slot %d is not in use", slot);
  if (nodes) *nodes = b->slots[slot].nodes;
  if (cells) *cells = b->host[slot].cells;
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
  info->variant = b->variant;
  info->round_mode = b->round_mode;
  return LBM_OK;
}

lbm_status lbm_batch_get_pdfs(lbm_batch_t *b, int32_t slot, double *f_host) {
  if (!b || !f_host) return bfail(b, LBM_ERR_INVALID_ARG, "NULL argument");
  if (slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].active)
    return bfail(b, LBM_ERR_INVALID_ARG, "slot %d is not in use", slot);
  const BatchSlot sl = b->slots[slot];
  if (b->variant == LBM_AA && (sl.steps & 1))
    return bfail(b, LBM_ERR_STATE, "AA pattern state is natural only after an even step count");
  lbm_status st = settle(b);
  if (st != LBM_OK) return st;
  if (b->admit_pending) {
    BCUDA(b, cudaStreamWaitEvent(b->stream, b->admit_done, 0));
    b->admit_pending = false;
  }
  st = upload_slots(b);
  if (st != LBM_OK) return st;
  const size_t bytes = sizeof(double) * Q * std::max<int64_t>(sl.nodes, 1);
  double *tmp = static_cast<double *>(balloc(b, bytes, false));
  if (!tmp) return bfail(b, LBM_ERR_OOM, "read-out buffer");
  BatchParams p = batch_params(b);
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((sl.nodes + 255) / 256, 1 << 20));
  if (b->cfg.precision == LBM_F64)
    k_batch_get<CodecF64><<<grid, 256, 0, b->stream>>>(p, slot, b->variant, tmp);
  else if (b->cfg.precision == LBM_F32)
    k_batch_get<CodecF32><<<grid, 256, 0, b->stream>>>(p, slot, b->variant, tmp);
  else
    k_batch_get<CodecF16S><<<grid, 256, 0, b->stream>>>(p, slot, b->variant, tmp);
  cudaError_t e = cudaMemcpyAsync(f_host, tmp, sizeof(double) * Q * sl.nodes, cudaMemcpyDeviceToHost, b->stream);
  cudaError_t e2 = cudaStreamSynchronize(b->stream);
  bfree(b, tmp, bytes);
  if (e != cudaSuccess || e2 != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "read-out");
  return LBM_OK;
}

}  // extern "C"

// Rebuild every active geometry for `variant` (index data and, for the
// esoteric twist, ghost slots), laid out again from the start of the arrays,
// at rest.  On failure the previous variant is restored the same way.
static lbm_status relayout(lbm_batch_t *b, int variant) {
  lbm_status st = settle(b);
  if (st != LBM_OK) return st;
  BCUDA(b, cudaStreamSynchronize(b->admit_stream));
  const int old = b->variant;
  for (int attempt = 0; attempt < 2; ++attempt) {
    const int v = attempt == 0 ? variant : old;
    b->variant = v;
    b->folded = v == LBM_AA && b->cfg.keep_idx == 0 && b->capacity < ((int64_t)1 << 30);
    b->free_ranges.clear();
    b->free_ranges[0] = b->capacity;
    st = LBM_OK;
    for (size_t s = 0; s < b->slots.size() && st == LBM_OK; ++s) {
      if (!b->slots[s].active) continue;
      st = build_segment(b, (int)s);
      BatchSlot &sl = b->slots[s];
      SlotHost &h = b->host[s];
      sl.steps = 0;
      h.have_prev = false;
      h.done = 0;
      h.mass = h.flux = 0.0;
      h.first_round = b->rounds_launched;
    }
    b->dirty = true;
    if (st == LBM_OK) break;
    if (attempt == 1) return bfail(b, LBM_ERR_CUDA, "relayout to the previous variant failed");
  }
  BCUDA(b, cudaStreamSynchronize(b->admit_stream));
  b->admit_pending = false;
  return b->variant == variant ? LBM_OK : bfail(b, LBM_ERR_OOM, "the geometries do not fit in variant %d", variant);
}

extern "C" {

// Autotuner: for each candidate (variant, block size, nodes per thread,
// round mode) one warm-up round (graph capture) and `rounds` rounds of k
// steps timed with CUDA events; the fastest is kept and every geometry
// restarts from rest in it.
lbm_status lbm_batch_tune(lbm_batch_t *b, int32_t rounds, int32_t k, int32_t *best_variant, int32_t *best_bs,
                          int32_t *best_npt, int32_t *best_mode, double *best_mflups) {
  if (!b || rounds < 1 || k < 1) return bfail(b, LBM_ERR_INVALID_ARG, "tune arguments");
  int64_t active = 0;
  for (auto &sl : b->slots)
    if (sl.active) active += sl.nodes;
  if (active == 0) return bfail(b, LBM_ERR_STATE, "no active geometry to tune on");
  std::vector<int> variants{b->variant};
  if (b->cfg.tune_variant) variants = {LBM_AA, LBM_ET};
  static const int sizes[] = {128, 256, 512};
  static const int npts[] = {1, 2, 4, 8};
  double best = -1.0;
  int bv = b->variant, bb = b->block_size, bn = b->npt, bm = b->round_mode;
  cudaEvent_t e0, e1;
  BCUDA(b, cudaEventCreate(&e0));
  BCUDA(b, cudaEventCreate(&e1));
  lbm_status result = LBM_OK;
  for (int v : variants) {
    if (v != b->variant && relayout(b, v) != LBM_OK) continue;  // does not fit: skip the variant
    for (int bs : sizes)
      for (int npt : npts)
        for (int mode = 0; mode < 2; ++mode) {
          if (kAlign % (bs * npt)) continue;
          b->block_size = bs;
          b->npt = npt;
          b->round_mode = mode;
          b->dirty = true;
          lbm_status st = lbm_batch_round(b, k);  // warm-up and graph capture
          if (st == LBM_OK) st = settle(b);
          if (st != LBM_OK) {
            if (mode == 1 && st == LBM_ERR_CUDA) continue;  // no co-resident grid for this shape
            result = st;
            goto done;
          }
          cudaEventRecord(e0, b->stream);
          for (int r = 0; r < rounds && st == LBM_OK; ++r) st = lbm_batch_round(b, k);
          cudaEventRecord(e1, b->stream);
          if (st == LBM_OK) st = settle(b);
          if (st != LBM_OK) {
            result = st;
            goto done;
          }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          const double mflups = (double)active * rounds * k / (ms * 1e-3) / 1e6;
          if (mflups > best) {
            best = mflups;
            bv = v;
            bb = bs;
            bn = npt;
            bm = mode;
          }
        }
  }
done:
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != LBM_OK) return result;
  if (best < 0) return bfail(b, LBM_ERR_CUDA, "no candidate ran");
  b->block_size = bb;
  b->npt = bn;
  b->round_mode = bm;
  lbm_status st = relayout(b, bv);  // every geometry back to rest in the chosen variant
  if (st != LBM_OK) return st;
  if (best_variant) *best_variant = bv;
  if (best_bs) *best_bs = bb;
  if (best_npt) *best_npt = bn;
  if (best_mode) *best_mode = bm;
  if (best_mflups) *best_mflups = best;
  return LBM_OK;
}

}  // extern "C"
