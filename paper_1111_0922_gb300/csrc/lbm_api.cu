// C ABI of liblbm (declared in include/lbm.h): handle life cycle, geometry
// set-up, state in/out, time stepping and reductions.  Host code only; every
// step of the path runs in the kernels of lbm_steps.cu, lbm_cg.cu,
// lbm_swap.cu and lbm_setup.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using namespace lbmk;

struct lbm {
  lbm_config cfg{};
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  std::vector<std::pair<void *, size_t>> geo_allocs;  // freed on re-geometry / destroy
  std::vector<std::pair<void *, size_t>> base_allocs; // freed on destroy
  bool has_geometry = false;
  int64_t cells = 0, nodes = 0, nghost = 0;
  int64_t nn = 0;    // node space of a launch (direct: cells, indirect: fluid nodes)
  int64_t slots = 0; // storage slots per PDF array
  int64_t npad = 0;  // SoA stride
  int64_t ipad = 0;
  uint8_t *d_solid = nullptr;
  bool any_solid = false;
  bool idx_folded = false;  // AA pattern, SoA node list: solid links folded into IDX
  int32_t *d_cells = nullptr, *d_idx = nullptr, *d_etidx = nullptr;
  void *d_A = nullptr, *d_B = nullptr;
  size_t state_bytes = 0;
  int64_t index_bytes = 0;
  double *d_partials = nullptr;
  int partial_blocks = 0;
  double *d_out2 = nullptr;
  double *h_out2 = nullptr;  // pinned
  int *d_err = nullptr;
  Grid grid{};
  int map[Q];
  int64_t steps = 0;
  float scale = 1.0f;
  int cg_k = 0, cg_o = 0;
  // compressed grid on a node list: unwrapped index, plane node counts,
  // shift K (nodes), slab size B, lower ghost room G
  int32_t *d_cidx = nullptr;
  int64_t cg_nfirst = 0, cg_nlast = 0, cg_K = 0, cg_B = 0, cg_G = 0;
  int swap_tile[3] = {0, 0, 0};
  // swap on a full grid: the lattice as a 4D tensor (x, y, z, array) for the
  // tile-staging tensor copies, when the layout allows them
  alignas(64) CUtensorMap swap_map{};
  bool swap_tma = false;
  int nsm = 0;
  // swap on a full grid: per-tile link-class tables of the coloured passes
  uint16_t *d_swap_tcls = nullptr;
  uint32_t *d_swap_tables = nullptr;
};

static std::string g_last_error;

static lbm_status fail(lbm_t *h, lbm_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h)
    h->err = buf;
  else
    g_last_error = buf;
  return s;
}

#define CUDA_TRY(h, call)                                                                          \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(h, LBM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (the library links only the runtime).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

static lbm_status check_launch(lbm_t *h, const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(h, LBM_ERR_CUDA, "%s launch: %s", what, cudaGetErrorString(e));
  return LBM_OK;
}

static void *dalloc(lbm_t *h, size_t bytes, std::vector<std::pair<void *, size_t>> &list) {
  if (bytes == 0) bytes = 256;
  void *p = nullptr;
  if (h->cfg.dev_alloc) {
    p = h->cfg.dev_alloc(bytes, h->cfg.alloc_ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) list.emplace_back(p, bytes);
  return p;
}

static void dfree(lbm_t *h, void *p, size_t bytes) {
  if (!p) return;
  if (h->cfg.dev_free)
    h->cfg.dev_free(p, bytes, h->cfg.alloc_ctx);
  else
    cudaFree(p);
}

static void free_list(lbm_t *h, std::vector<std::pair<void *, size_t>> &list) {
  for (auto &a : list) dfree(h, a.first, a.second);
  list.clear();
}

// temporary device buffer freed at scope exit (after a stream sync)
struct TempBuf {
  lbm_t *h;
  void *p = nullptr;
  size_t n = 0;
  TempBuf(lbm_t *h_, size_t bytes) : h(h_), n(bytes) {
    std::vector<std::pair<void *, size_t>> l;
    p = dalloc(h, bytes, l);
  }
  ~TempBuf() {
    if (p) {
      cudaStreamSynchronize(h->stream);
      dfree(h, p, n);
    }
  }
};

static int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

static size_t store_size(int precision) { return precision == LBM_F64 ? 8 : (precision == LBM_F32 ? 4 : 2); }


static bool two_lattices(int variant) {
  return variant == LBM_TS || variant == LBM_OS_PUSH || variant == LBM_OS_PULL;
}

static int map_kind(const lbm_t *h) {
  switch (h->cfg.variant) {
    case LBM_OS_PULL:
    case LBM_CG:
      return MAP_PULL;
    case LBM_ET:
      return MAP_ET;
    default:
      return MAP_NATURAL;
  }
}

static bool is_natural(const lbm_t *h) { return h->cfg.variant != LBM_AA || (h->steps & 1) == 0; }

static KernelKey key_of(const lbm_t *h, bool red) {
  KernelKey k;
  k.precision = h->cfg.precision;
  k.aos = h->cfg.layout == LBM_AOS;
  k.ind = h->cfg.addressing == LBM_INDIRECT;
  k.force = h->cfg.force[0] != 0.0 || h->cfg.force[1] != 0.0 || h->cfg.force[2] != 0.0;
  k.red = red;
  return k;
}

static size_t store_size(int precision);

// Element offset of the current state in an indirect compressed grid.
static int64_t cg_ind_offset(const lbm_t *h, int64_t o) {
  const int64_t e = o + h->cg_G;
  return h->cfg.layout == LBM_AOS ? e * Q : e;
}

static void *shifted(void *base, int64_t elements, int precision) {
  return static_cast<char *>(base) + elements * (int64_t)store_size(precision);
}

// Antisymmetric relaxation rate: omega for BGK; for TRT the rate that gives
// (1/omega - 1/2)(1/omega_m - 1/2) = trt_magic.
static double omega_minus(const lbm_config &c) {
  if (!(c.trt_magic > 0.0) || c.omega <= 0.0) return c.omega;
  return 1.0 / (0.5 + c.trt_magic / (1.0 / c.omega - 0.5));
}

static StepParams params_of(const lbm_t *h) {
  StepParams p;
  memset(&p, 0, sizeof p);
  p.A = h->d_A;
  if (h->cfg.variant == LBM_CG && h->cfg.addressing == LBM_INDIRECT && h->d_A)
    p.A = shifted(h->d_A, cg_ind_offset(h, h->cg_o), h->cfg.precision);
  p.B = h->d_B;
  p.npad = h->npad;
  p.nnodes = h->nn;
  p.nfluid = h->nodes;
  p.g = h->grid;
  p.idx = h->cfg.variant == LBM_ET ? h->d_etidx : h->d_idx;
  p.ipad = h->ipad;
  for (int i = 0; i < Q; ++i) {
    p.map[i] = h->map[i];
    p.mapbase[i] = h->d_A ? static_cast<char *>(p.A) + (int64_t)h->map[i] * h->npad * (int64_t)store_size(h->cfg.precision)
                          : nullptr;
  }
  p.omega = h->cfg.omega;
  p.omega_m = omega_minus(h->cfg);
  p.gx = h->cfg.force[0];
  p.gy = h->cfg.force[1];
  p.gz = h->cfg.force[2];
  p.kf = make_collk<float>((float)p.omega, (float)p.omega_m, (float)p.gx, (float)p.gy, (float)p.gz);
  p.kd = make_collk<double>(p.omega, p.omega_m, p.gx, p.gy, p.gz);
  p.scale = h->scale;
  p.inv_scale = 1.0f / h->scale;
  p.partials = h->d_partials;
  p.err = h->d_err;
  p.idx_folded = h->idx_folded ? 1 : 0;
  return p;
}

// Launch shape of the step kernels.  Full grid: 2D blocks over (x, y) (x
// extent rounded up to a warp, capped at the block size), grid z over planes,
// nodes_per_thread planes per thread.  Node list: 1D, nodes_per_thread nodes
// per thread.
static LaunchShape shape_of(const lbm_t *h) {
  LaunchShape L;
  // default block: 128 threads; 256 for the AA pattern on a node list
  // (measured +2 % FP32, +8 % FP16 on the 512^3 sphere pack)
  const bool aa_list = h->cfg.variant == LBM_AA && h->cfg.addressing == LBM_INDIRECT;
  const int bs = h->cfg.block_size > 0 ? h->cfg.block_size : (aa_list ? 256 : 128);
  // full grids: two planes per thread by default (measured +2 % FP32, +5 %
  // FP16 on 256^3); node lists: one node per thread
  const int npt = h->cfg.nodes_per_thread > 0 ? h->cfg.nodes_per_thread
                                               : (h->cfg.addressing == LBM_DIRECT ? 2 : 1);
  if (h->cfg.addressing == LBM_DIRECT) {
    const int bx = (int)std::min<int64_t>(bs, round_up(h->cfg.nx, 32));
    const int by = std::max(1, bs / bx);
    const int64_t gx = (h->cfg.nx + bx - 1) / bx, gy = (h->cfg.ny + by - 1) / by;
    const int64_t gz = std::min<int64_t>((h->cfg.nz + npt - 1) / npt, 65535);
    L.grid = dim3((unsigned)gx, (unsigned)gy, (unsigned)gz);
    L.block = dim3((unsigned)bx, (unsigned)by);
  } else {
    int64_t blocks = (h->nn + (int64_t)bs * npt - 1) / ((int64_t)bs * npt);
    if (blocks < 1) blocks = 1;
    L.grid = dim3((unsigned)blocks);
    L.block = dim3((unsigned)bs);
  }
  L.stream = h->stream;
  return L;
}

static int64_t blocks_of(const LaunchShape &L) { return (int64_t)L.grid.x * L.grid.y * L.grid.z; }

// FP16 / FP32 storage in z pairs (Grid::zpair, kernels in lbm_steps.cuh and
// lbm_swap.cuh)?  Two-step, one-step and AA pattern on a full grid without
// solid cells or halos, the esoteric twist on a periodic one, the coloured
// swap with a periodic z axis and nz a multiple of 4 (at least two tiles of
// two pair planes, so that no tile spans the seam), with an even nz;
// any_solid and the halos must be known.
static bool use_zpairs(const lbm_t *h) {
  const lbm_config &c = h->cfg;
  const bool scheme = c.variant == LBM_AA || c.variant == LBM_TS ||
                      ((c.variant == LBM_OS_PUSH || c.variant == LBM_OS_PULL) && c.store_hint == 0) ||
                      (c.variant == LBM_ET && c.periodic[0] && c.periodic[1] && c.periodic[2]) ||
                      (c.variant == LBM_SWAP && c.periodic[2] && c.swap_schedule <= 1 && (c.nz % 4) == 0 &&
                       c.nz >= 8);
  const bool prec = c.precision == LBM_F16S || c.precision == LBM_F32;
  return scheme && prec && c.addressing == LBM_DIRECT && c.layout == LBM_SOA && c.pair_z != 2 &&
         (c.nz % 2) == 0 && !h->any_solid && h->grid.hx == 0 && h->grid.hy == 0 && h->grid.hz == 0;
}

// Compressed grid with FP16 / FP32 storage in y pairs (Grid::ypair, lbm_cg.cu)?
// Full grid without solid cells, no x or y halo, even ny.
static bool use_ypairs(const lbm_t *h) {
  const lbm_config &c = h->cfg;
  return c.variant == LBM_CG && c.addressing == LBM_DIRECT && c.layout == LBM_SOA &&
         (c.precision == LBM_F16S || c.precision == LBM_F32) && c.pair_z != 2 && (c.ny % 2) == 0 && !h->any_solid &&
         h->grid.hx == 0 && h->grid.hy == 0;
}

// AA pattern (IDX folded at geometry time) and esoteric twist on a node list
// in node pairs (k_aa_even_np / k_aa_odd_np / k_et_np in lbm_steps.cuh):
// FP16 storage, SoA, pair_z not 2.
static bool use_npairs(const lbm_t *h) {
  const lbm_config &c = h->cfg;
  return ((c.variant == LBM_AA && h->idx_folded) || c.variant == LBM_ET) && c.addressing == LBM_INDIRECT &&
         c.layout == LBM_SOA && c.precision == LBM_F16S && c.pair_z != 2;
}

// node pairs: one thread per pair of consecutive nodes, nodes_per_thread
// pairs per thread (grid-stride; default 2)
static LaunchShape npair_shape_of(const lbm_t *h) {
  LaunchShape L = shape_of(h);
  const int npt = h->cfg.nodes_per_thread > 0 ? h->cfg.nodes_per_thread : 2;
  const int64_t per = (int64_t)L.block.x * npt;
  L.grid = dim3((unsigned)std::max<int64_t>(1, ((h->nn + 1) / 2 + per - 1) / per));
  return L;
}

// one thread per column (x, y) and pair plane, nodes_per_thread pair planes
// (default 4 with FP16 storage, 2 with FP32; measured on 256^3, FP16 4 vs 2
// planes: AA 80.3 vs 78.7 (its even kernel prefetches the next plane),
// one-step push 77.9 vs 76.2, pull 79.5 vs 77.5, esoteric twist 80.9 vs
// 80.2, two-step equal; FP32 best at 2)
static LaunchShape zpair_shape_of(const lbm_t *h) {
  LaunchShape L = shape_of(h);
  const int npt = h->cfg.nodes_per_thread > 0 ? h->cfg.nodes_per_thread : (h->cfg.precision == LBM_F16S ? 4 : 2);
  L.grid.z = (unsigned)std::min<int64_t>((h->cfg.nz / 2 + npt - 1) / npt, 65535);
  return L;
}

// Swap tiles over the grid (with cell pairs: over the grid of pair words,
// nz/2 planes).
static SwapTiles swap_tiles(const lbm_t *h) {
  SwapTiles t;
  t.pairs = h->grid.zpair;
  const int nz = t.pairs ? h->cfg.nz / 2 : h->cfg.nz;
  t.tx = std::min(kSwapTX, h->cfg.nx);
  t.ty = std::min(kSwapTY, h->cfg.ny);
  t.tz = std::min(kSwapTZ, nz);
  t.ntx = (h->cfg.nx + t.tx - 1) / t.tx;
  t.nty = (h->cfg.ny + t.ty - 1) / t.ty;
  t.ntz = (nz + t.tz - 1) / t.tz;
  t.colour = 0;
  t.ncolours = swap_colours(t, h->cfg.periodic[0], h->cfg.periodic[1], h->cfg.periodic[2]);
  t.tcls = h->d_swap_tcls;
  t.tables = h->d_swap_tables;
  return t;
}

static StateDesc state_desc(const lbm_t *h) {
  StateDesc d;
  d.p = params_of(h);
  d.k = key_of(h, false);
  d.mapkind = map_kind(h);
  d.cells = h->d_cells;
  return d;
}

extern "C" {

const char *lbm_status_string(lbm_status s) {
  switch (s) {
    case LBM_OK: return "ok";
    case LBM_ERR_INVALID_ARG: return "invalid argument";
    case LBM_ERR_OOM: return "out of device memory";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_STATE: return "invalid state";
    case LBM_ERR_BOUNDS: return "bounds check failed";
    case LBM_ERR_TIMEOUT: return "device wait timed out";
    case LBM_ERR_NOT_CONVERGED: return "not converged";
    case LBM_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char *lbm_last_error(const lbm_t *h) { return h ? h->err.c_str() : g_last_error.c_str(); }

lbm_status lbm_config_default(lbm_config *cfg) {
  if (!cfg) return fail(nullptr, LBM_ERR_INVALID_ARG, "cfg is NULL");
  memset(cfg, 0, sizeof *cfg);
  cfg->nx = cfg->ny = cfg->nz = 32;
  cfg->periodic[0] = cfg->periodic[1] = cfg->periodic[2] = 1;
  cfg->variant = LBM_AA;
  cfg->addressing = LBM_DIRECT;
  cfg->layout = LBM_SOA;
  cfg->precision = LBM_F32;
  cfg->omega = 1.0;
  return LBM_OK;
}

lbm_status lbm_create(const lbm_config *cfg, lbm_t **out) {
  if (!cfg || !out) return fail(nullptr, LBM_ERR_INVALID_ARG, "cfg and out must not be NULL");
  *out = nullptr;
  const int n[3] = {cfg->nx, cfg->ny, cfg->nz};
  for (int a = 0; a < 3; ++a) {
    if (n[a] < 1) return fail(nullptr, LBM_ERR_INVALID_ARG, "box extent %d on axis %d", n[a], a);
    if (cfg->periodic[a] && n[a] < 2)
      return fail(nullptr, LBM_ERR_INVALID_ARG, "periodic axis %d needs extent >= 2", a);
  }
  if (cfg->ny > 65535) return fail(nullptr, LBM_ERR_INVALID_ARG, "ny must be <= 65535");
  if ((int64_t)n[0] * n[1] * n[2] >= (int64_t)1 << 30)
    return fail(nullptr, LBM_ERR_INVALID_ARG, "box of %lld cells exceeds 2^30", (long long)n[0] * n[1] * n[2]);
  if (cfg->variant < LBM_TS || cfg->variant > LBM_ET) return fail(nullptr, LBM_ERR_INVALID_ARG, "variant");
  if (cfg->addressing != LBM_DIRECT && cfg->addressing != LBM_INDIRECT)
    return fail(nullptr, LBM_ERR_INVALID_ARG, "addressing");
  if (cfg->layout != LBM_SOA && cfg->layout != LBM_AOS) return fail(nullptr, LBM_ERR_INVALID_ARG, "layout");
  if (cfg->precision < LBM_F64 || cfg->precision > LBM_F16S) return fail(nullptr, LBM_ERR_INVALID_ARG, "precision");
  if (!(cfg->omega >= 0.0 && cfg->omega < 2.0)) return fail(nullptr, LBM_ERR_INVALID_ARG, "omega must be in [0, 2)");
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(cfg->force[a])) return fail(nullptr, LBM_ERR_INVALID_ARG, "force");
  if (cfg->block_size != 0 && (cfg->block_size % 32 != 0 || cfg->block_size < 32 || cfg->block_size > 256))
    return fail(nullptr, LBM_ERR_INVALID_ARG, "block_size must be a multiple of 32 in [32, 256]");
  if (cfg->nodes_per_thread < 0 || cfg->nodes_per_thread > 16)
    return fail(nullptr, LBM_ERR_INVALID_ARG, "nodes_per_thread must be in [0, 16]");
  if (cfg->trt_magic < 0.0 || !std::isfinite(cfg->trt_magic)) return fail(nullptr, LBM_ERR_INVALID_ARG, "trt_magic");
  if (cfg->trt_magic > 0.0 && !(cfg->omega > 0.0)) return fail(nullptr, LBM_ERR_INVALID_ARG, "TRT needs omega > 0");
  if (cfg->f16_scale < 0.0 || !std::isfinite(cfg->f16_scale))
    return fail(nullptr, LBM_ERR_INVALID_ARG, "f16_scale");
  if (cfg->f16_scale > 0.0) {
    int e;
    if (std::frexp(cfg->f16_scale, &e) != 0.5) return fail(nullptr, LBM_ERR_INVALID_ARG, "f16_scale must be 2^k");
  }
  if (cfg->dev_alloc && !cfg->dev_free) return fail(nullptr, LBM_ERR_INVALID_ARG, "dev_alloc without dev_free");
  if (cfg->cg_shift < 0 || (cfg->addressing == LBM_DIRECT && cfg->cg_shift == 1))
    return fail(nullptr, LBM_ERR_INVALID_ARG, "cg_shift: >= 2 planes on a full grid, >= 1 node on a node list");
  if (cfg->pair_z < 0 || cfg->pair_z > 2) return fail(nullptr, LBM_ERR_INVALID_ARG, "pair_z must be 0 .. 2");
  if (cfg->store_hint != 0 && cfg->store_hint != 1) return fail(nullptr, LBM_ERR_INVALID_ARG, "store_hint must be 0 or 1");
  if (cfg->store_hint == 1 && (!(cfg->variant == LBM_OS_PUSH || cfg->variant == LBM_OS_PULL) || cfg->layout != LBM_SOA))
    return fail(nullptr, LBM_ERR_INVALID_ARG, "store_hint = 1 needs LBM_OS_PUSH or LBM_OS_PULL with LBM_SOA");
  if (cfg->swap_schedule < 0 || cfg->swap_schedule > 2)
    return fail(nullptr, LBM_ERR_INVALID_ARG, "swap_schedule must be 0 .. 2");

  lbm_t *h = new lbm_t();
  h->cfg = *cfg;
  h->stream = static_cast<cudaStream_t>(cfg->stream);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) {
    delete h;
    return fail(nullptr, LBM_ERR_CUDA, "device attributes: %s", cudaGetErrorString(e));
  }
  h->d_err = static_cast<int *>(dalloc(h, sizeof(int) * 4, h->base_allocs));
  h->d_out2 = static_cast<double *>(dalloc(h, sizeof(double) * 2, h->base_allocs));
  if (!h->d_err || !h->d_out2) {
    free_list(h, h->base_allocs);
    delete h;
    return fail(nullptr, LBM_ERR_OOM, "small device buffers");
  }
  if (cudaMallocHost(&h->h_out2, sizeof(double) * 2) != cudaSuccess) {
    cudaGetLastError();
    free_list(h, h->base_allocs);
    delete h;
    return fail(nullptr, LBM_ERR_OOM, "pinned host buffer");
  }
  cudaMemsetAsync(h->d_err, 0, sizeof(int) * 4, h->stream);
  for (int i = 0; i < Q; ++i) h->map[i] = i;
  *out = h;
  return LBM_OK;
}

lbm_status lbm_destroy(lbm_t *h) {
  if (!h) return LBM_OK;
  cudaStreamSynchronize(h->stream);
  free_list(h, h->geo_allocs);
  free_list(h, h->base_allocs);
  if (h->h_out2) cudaFreeHost(h->h_out2);
  delete h;
  return LBM_OK;
}

lbm_status lbm_sync(lbm_t *h) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID_ARG, "handle is NULL");
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  int flags[4];
  CUDA_TRY(h, cudaMemcpy(flags, h->d_err, sizeof flags, cudaMemcpyDeviceToHost));
  if (flags[0]) return fail(h, LBM_ERR_BOUNDS, "a kernel bounds check tripped (code %d)", flags[0]);
  if (flags[1]) return fail(h, LBM_ERR_TIMEOUT, "a kernel's bounded wait for a tile copy gave up");
  return LBM_OK;
}

// ---------------------------------------------------------------------------
static lbm_status build_geometry(lbm_t *h) {
  const lbm_config &c = h->cfg;
  const bool ind = c.addressing == LBM_INDIRECT;
  const int64_t ncell = h->cells;
  std::vector<std::pair<void *, size_t>> temps;
  auto cleanup = [&]() {
    cudaStreamSynchronize(h->stream);
    free_list(h, temps);
  };
  if (ind) {
    int32_t *node_of = static_cast<int32_t *>(dalloc(h, sizeof(int32_t) * ncell, temps));
    const int64_t ext = (int64_t)(c.nx + 2) * (c.ny + 2) * (c.nz + 2);
    const int64_t sc = scan_scratch_elems(std::max(ncell, ext));
    int32_t *scratch = static_cast<int32_t *>(dalloc(h, sizeof(int32_t) * sc, temps));
    int32_t *cells_tmp = static_cast<int32_t *>(dalloc(h, sizeof(int32_t) * ncell, temps));
    if (!node_of || !scratch || !cells_tmp) {
      cleanup();
      return fail(h, LBM_ERR_OOM, "node-list scratch for %lld cells", (long long)ncell);
    }
    const int64_t N = build_node_list(h->any_solid ? h->d_solid : nullptr, ncell, node_of, cells_tmp, scratch, sc,
                                      h->stream);
    if (N < 0) {
      cleanup();
      return fail(h, LBM_ERR_CUDA, "node-list build failed");
    }
    h->nodes = N;
    h->nn = N;
    h->ipad = round_up(std::max<int64_t>(N, 1), 64);
    h->d_cells = static_cast<int32_t *>(dalloc(h, sizeof(int32_t) * std::max<int64_t>(N, 1), h->geo_allocs));
    h->d_idx = static_cast<int32_t *>(dalloc(h, sizeof(int32_t) * 18 * h->ipad, h->geo_allocs));
    if (!h->d_cells || !h->d_idx) {
      cleanup();
      return fail(h, LBM_ERR_OOM, "IDX for %lld nodes", (long long)N);
    }
    h->index_bytes = (int64_t)sizeof(int32_t) * (N + 18 * h->ipad);
    CUDA_TRY(h, cudaMemcpyAsync(h->d_cells, cells_tmp, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, h->stream));
    launch_build_idx(h->d_cells, node_of, N, c.nx, c.ny, c.nz, c.periodic, h->d_idx, h->ipad, h->stream);
    lbm_status st = check_launch(h, "build_idx");
    if (st != LBM_OK) {
      cleanup();
      return st;
    }
    h->nghost = 0;
    if (c.variant == LBM_ET) {
      int32_t *ghost = static_cast<int32_t *>(dalloc(h, sizeof(int32_t) * ext, temps));
      h->d_etidx = static_cast<int32_t *>(dalloc(h, sizeof(int32_t) * 9 * h->ipad, h->geo_allocs));
      if (!ghost || !h->d_etidx) {
        cleanup();
        return fail(h, LBM_ERR_OOM, "esoteric-twist index");
      }
      h->index_bytes += (int64_t)sizeof(int32_t) * 9 * h->ipad;
      const int64_t G = build_et_index(h->d_cells, node_of, N, c.nx, c.ny, c.nz, c.periodic, ghost, h->d_etidx,
                                       h->ipad, scratch, sc, h->stream);
      if (G < 0) {
        cleanup();
        return fail(h, LBM_ERR_CUDA, "esoteric-twist index build failed");
      }
      h->nghost = G;
    }
    h->slots = N + h->nghost;
    if (c.variant == LBM_CG) {
      h->d_cidx = static_cast<int32_t *>(dalloc(h, sizeof(int32_t) * 18 * h->ipad, h->geo_allocs));
      int *counters = static_cast<int *>(dalloc(h, sizeof(int) * 4, temps));
      if (!h->d_cidx || !counters) {
        cleanup();
        return fail(h, LBM_ERR_OOM, "compressed-grid index");
      }
      h->index_bytes += (int64_t)sizeof(int32_t) * 18 * h->ipad;
      CUDA_TRY(h, cudaMemsetAsync(counters, 0, sizeof(int) * 4, h->stream));
      launch_cg_ind_prep(h->d_idx, h->ipad, h->d_cells, N, c.nx, c.ny, c.nz, h->d_cidx, counters, h->stream);
      int hc[4];
      CUDA_TRY(h, cudaMemcpyAsync(hc, counters, sizeof hc, cudaMemcpyDeviceToHost, h->stream));
      CUDA_TRY(h, cudaStreamSynchronize(h->stream));
      const int64_t D = hc[0];
      h->cg_nfirst = c.periodic[2] ? hc[1] : 0;
      h->cg_nlast = c.periodic[2] ? hc[2] : 0;
      h->cg_B = c.cg_shift > 0 ? c.cg_shift : std::min<int64_t>(std::max<int64_t>(N, 1), (int64_t)1 << 21);
      h->cg_K = D + h->cg_B;
      h->cg_G = h->cg_nlast;
      h->slots = N + h->cg_nfirst + h->cg_nlast + h->cg_K;
    }
    if (h->slots >= ((int64_t)1 << 31) - 1) {
      cleanup();
      return fail(h, LBM_ERR_INVALID_ARG, "too many storage slots");
    }
    cleanup();
  } else {
    // full grid; halos only where a scheme needs slots beyond a wall
    const bool halo = c.variant == LBM_ET;
    Grid &g = h->grid;
    g.nx = c.nx;
    g.ny = c.ny;
    g.nz = c.nz;
    g.px = c.periodic[0];
    g.py = c.periodic[1];
    g.pz = c.periodic[2];
    g.hx = halo && !g.px;
    g.hy = halo && !g.py;
    g.hz = halo && !g.pz;
    int64_t sz = c.nz + 2 * g.hz;
    if (c.variant == LBM_CG) {
      // plane offsets 0 or k, plus a ghost plane below and above
      int k = c.cg_shift;
      if (k == 0) {
        // slabs of about 2^22 cells: fewer, larger launches against k extra
        // planes of storage (256^3: k = 65, +25 %; measured 41.7 vs 40.0
        // GFLUP/s FP32, 52.1 vs 48.5 FP16 with slabs of 2^21 cells)
        const int64_t plane = (int64_t)c.nx * c.ny;
        int64_t want = (1 << 22) / std::max<int64_t>(plane, 1) + 1;
        if (want < 2) want = 2;
        if (want > c.nz + 1) want = c.nz + 1;
        k = (int)want;
      }
      h->cg_k = k;
      g.hz = 1;
      sz = c.nz + k + 2;
    }
    g.sx = c.nx + 2 * g.hx;
    g.sxy = g.sx * (c.ny + 2 * g.hy);
    g.zoff = 0;
    g.solid = h->any_solid ? h->d_solid : nullptr;
    g.zpair = use_zpairs(h) ? 1 : 0;
    g.ypair = use_ypairs(h) ? 1 : 0;
    h->nn = ncell;
    h->slots = g.sxy * sz;
    if (h->slots >= ((int64_t)1 << 31) - 1) return fail(h, LBM_ERR_INVALID_ARG, "too many storage slots");
    h->index_bytes = h->any_solid ? ncell : 0;
  }
  // PDF storage
  const size_t es = store_size(c.precision);
  h->npad = c.layout == LBM_SOA ? round_up(std::max<int64_t>(h->slots, 1), 128) : h->slots;
  h->state_bytes = es * (size_t)Q * (size_t)std::max<int64_t>(h->npad, 1);
  h->d_A = dalloc(h, h->state_bytes, h->geo_allocs);
  if (two_lattices(c.variant)) h->d_B = dalloc(h, h->state_bytes, h->geo_allocs);
  if (!h->d_A || (two_lattices(c.variant) && !h->d_B))
    return fail(h, LBM_ERR_OOM, "PDF storage of %zu bytes", h->state_bytes);
  CUDA_TRY(h, cudaMemsetAsync(h->d_A, 0, h->state_bytes, h->stream));
  if (h->d_B) CUDA_TRY(h, cudaMemsetAsync(h->d_B, 0, h->state_bytes, h->stream));
  if (c.variant == LBM_AA && c.addressing == LBM_INDIRECT && c.layout == LBM_SOA && h->nodes > 0) {
    launch_fold_idx(h->d_idx, h->ipad, h->nodes, h->npad, h->stream);
    lbm_status st = check_launch(h, "fold_idx");
    if (st != LBM_OK) return st;
    h->idx_folded = true;
  }
  h->swap_tma = false;
  if (c.variant == LBM_SWAP && !ind && c.layout == LBM_SOA &&
      c.swap_schedule == 2) {
    // tensor copies need 16-byte row pitches and inner box extents
    const SwapTiles t = swap_tiles(h);
    const cuuint64_t es = (cuuint64_t)store_size(c.precision);
    EncodeTiledFn enc = encode_tiled();
    if (enc && (h->grid.sx * (int64_t)es) % 16 == 0 && ((int64_t)t.tx * (int64_t)es) % 16 == 0 && h->grid.hx == 0 &&
        h->grid.hy == 0 && h->grid.hz == 0 && h->grid.zoff == 0) {
      const cuuint64_t dims[4] = {(cuuint64_t)c.nx, (cuuint64_t)c.ny, (cuuint64_t)c.nz, (cuuint64_t)Q};
      const cuuint64_t strides[3] = {(cuuint64_t)h->grid.sx * es, (cuuint64_t)h->grid.sxy * es,
                                     (cuuint64_t)h->npad * es};
      const cuuint32_t box[4] = {(cuuint32_t)t.tx, (cuuint32_t)t.ty, (cuuint32_t)t.tz, (cuuint32_t)Q};
      const cuuint32_t estr[4] = {1, 1, 1, 1};
      const CUtensorMapDataType dt = c.precision == LBM_F64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                     : c.precision == LBM_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                              : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
      const CUresult r = enc(&h->swap_map, dt, 4, h->d_A, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      h->swap_tma = r == CUDA_SUCCESS;
    }

  }
  if (c.variant == LBM_SWAP && !ind) {
    const SwapTiles t = swap_tiles(h);
    {
      std::vector<uint16_t> tcls;
      std::vector<uint32_t> tables;
      build_swap_tables(t, c.periodic, tcls, tables);
      uint16_t *dt = static_cast<uint16_t *>(dalloc(h, sizeof(uint16_t) * tcls.size(), h->geo_allocs));
      uint32_t *dtab = static_cast<uint32_t *>(dalloc(h, sizeof(uint32_t) * tables.size(), h->geo_allocs));
      if (!dt || !dtab) return fail(h, LBM_ERR_OOM, "swap link-class tables");
      CUDA_TRY(h, cudaMemcpyAsync(dt, tcls.data(), sizeof(uint16_t) * tcls.size(), cudaMemcpyHostToDevice, h->stream));
      CUDA_TRY(h, cudaMemcpyAsync(dtab, tables.data(), sizeof(uint32_t) * tables.size(), cudaMemcpyHostToDevice,
                                  h->stream));
      CUDA_TRY(h, cudaStreamSynchronize(h->stream));  // the host vectors go out of scope
      h->d_swap_tcls = dt;
      h->d_swap_tables = dtab;
    }
  }
  // reduction partials: enough for a step launch and for the read-out kernel
  const LaunchShape L = shape_of(h);
  int64_t need = std::max<int64_t>(blocks_of(L), reduce_blocks_for(h->nn));
  if (c.variant == LBM_CG && c.addressing == LBM_DIRECT)
    need = std::max<int64_t>(need, (int64_t)L.grid.x * L.grid.y * c.nz);  // slabs, 1 plane per z-block
  if (c.variant == LBM_CG && c.addressing == LBM_INDIRECT)
    need += (h->nodes + h->cg_B - 1) / std::max<int64_t>(h->cg_B, 1) + 1;  // one partial block per slab
  if (c.variant == LBM_SWAP) {
    const SwapTiles t = swap_tiles(h);
    need = std::max<int64_t>(need, (int64_t)t.ntx * t.nty * t.ntz);
  }
  h->partial_blocks = (int)need;
  h->d_partials = static_cast<double *>(dalloc(h, sizeof(double) * 2 * h->partial_blocks, h->geo_allocs));
  if (!h->d_partials) return fail(h, LBM_ERR_OOM, "reduction partials");
  h->has_geometry = true;
  return LBM_OK;
}

static void reset_geometry(lbm_t *h) {
  cudaStreamSynchronize(h->stream);
  free_list(h, h->geo_allocs);
  h->d_solid = nullptr;
  h->d_cells = h->d_idx = h->d_etidx = h->d_cidx = nullptr;
  h->cg_nfirst = h->cg_nlast = h->cg_K = h->cg_B = h->cg_G = 0;
  h->d_A = h->d_B = nullptr;
  h->d_partials = nullptr;
  h->has_geometry = false;
  h->cells = (int64_t)h->cfg.nx * h->cfg.ny * h->cfg.nz;
  h->nodes = h->nghost = h->nn = h->slots = h->npad = h->ipad = 0;
  h->idx_folded = false;
  h->swap_tma = false;
  h->d_swap_tcls = nullptr;
  h->d_swap_tables = nullptr;
  h->steps = 0;
  for (int i = 0; i < Q; ++i) h->map[i] = i;
}

static lbm_status finish_geometry(lbm_t *h) {
  lbm_status st = build_geometry(h);
  if (st != LBM_OK) {
    reset_geometry(h);
    return st;
  }
  st = lbm_init(h, nullptr, nullptr, 0);
  if (st != LBM_OK) return st;
  return lbm_sync(h);
}

lbm_status lbm_set_geometry(lbm_t *h, const uint8_t *mask) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID_ARG, "handle is NULL");
  reset_geometry(h);
  const int64_t ncell = h->cells;
  int64_t fluid = ncell;
  h->any_solid = false;
  if (mask) {
    fluid = 0;
    for (int64_t c = 0; c < ncell; ++c) fluid += mask[c] == 0;
    h->any_solid = fluid != ncell;
  }
  h->d_solid = static_cast<uint8_t *>(dalloc(h, (size_t)ncell, h->geo_allocs));
  if (!h->d_solid) return fail(h, LBM_ERR_OOM, "solid mask of %lld cells", (long long)ncell);
  if (mask) {
    // normalise to 0/1 on the host copy path
    std::vector<uint8_t> m01(mask, mask + ncell);
    for (auto &v : m01) v = v != 0;
    CUDA_TRY(h, cudaMemcpyAsync(h->d_solid, m01.data(), (size_t)ncell, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  } else {
    CUDA_TRY(h, cudaMemsetAsync(h->d_solid, 0, (size_t)ncell, h->stream));
  }
  h->nodes = fluid;
  lbm_status st = finish_geometry(h);
  if (st == LBM_OK && h->cfg.addressing == LBM_DIRECT) h->nodes = fluid;
  return st;
}

lbm_status lbm_set_geometry_spheres(lbm_t *h, int64_t nsph, const int64_t *centres, int64_t radius, int64_t unit) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID_ARG, "handle is NULL");
  if (nsph < 0 || (nsph > 0 && !centres) || radius < 0 || unit < 1)
    return fail(h, LBM_ERR_INVALID_ARG, "sphere arguments");
  reset_geometry(h);
  const int64_t ncell = h->cells;
  h->d_solid = static_cast<uint8_t *>(dalloc(h, (size_t)ncell, h->geo_allocs));
  if (!h->d_solid) return fail(h, LBM_ERR_OOM, "solid mask of %lld cells", (long long)ncell);
  CUDA_TRY(h, cudaMemsetAsync(h->d_solid, 0, (size_t)ncell, h->stream));
  if (nsph > 0) {
    TempBuf cen(h, sizeof(int64_t) * 3 * nsph);
    if (!cen.p) return fail(h, LBM_ERR_OOM, "sphere centres");
    CUDA_TRY(h, cudaMemcpyAsync(cen.p, centres, sizeof(int64_t) * 3 * nsph, cudaMemcpyHostToDevice, h->stream));
    launch_sphere_mask(h->d_solid, h->cfg.nx, h->cfg.ny, h->cfg.nz, h->cfg.periodic, nsph,
                       static_cast<const int64_t *>(cen.p), radius, unit, h->stream);
    lbm_status st = check_launch(h, "sphere_mask");
    if (st != LBM_OK) return st;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  // fluid count for the full-grid case (the node list counts it for IDX)
  {
    std::vector<uint8_t> m((size_t)ncell);
    CUDA_TRY(h, cudaMemcpy(m.data(), h->d_solid, (size_t)ncell, cudaMemcpyDeviceToHost));
    int64_t fluid = 0;
    for (auto v : m) fluid += v == 0;
    h->nodes = fluid;
    h->any_solid = fluid != ncell;
  }
  const int64_t fluid = h->nodes;
  lbm_status st = finish_geometry(h);
  if (st == LBM_OK && h->cfg.addressing == LBM_DIRECT) h->nodes = fluid;
  return st;
}

lbm_status lbm_get_mask(lbm_t *h, uint8_t *mask) {
  if (!h || !mask) return fail(h, LBM_ERR_INVALID_ARG, "NULL argument");
  if (!h->has_geometry) return fail(h, LBM_ERR_STATE, "no geometry");
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  CUDA_TRY(h, cudaMemcpy(mask, h->d_solid, (size_t)h->cells, cudaMemcpyDeviceToHost));
  return LBM_OK;
}

lbm_status lbm_get_nodes(lbm_t *h, int32_t *cells) {
  if (!h || !cells) return fail(h, LBM_ERR_INVALID_ARG, "NULL argument");
  if (!h->has_geometry) return fail(h, LBM_ERR_STATE, "no geometry");
  if (h->cfg.addressing != LBM_INDIRECT) return fail(h, LBM_ERR_INVALID_ARG, "node list exists for indirect addressing");
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  CUDA_TRY(h, cudaMemcpy(cells, h->d_cells, sizeof(int32_t) * h->nodes, cudaMemcpyDeviceToHost));
  return LBM_OK;
}

lbm_status lbm_get_idx(lbm_t *h, int32_t *idx) {
  if (!h || !idx) return fail(h, LBM_ERR_INVALID_ARG, "NULL argument");
  if (!h->has_geometry) return fail(h, LBM_ERR_STATE, "no geometry");
  if (h->cfg.addressing != LBM_INDIRECT) return fail(h, LBM_ERR_INVALID_ARG, "IDX exists for indirect addressing");
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (h->nodes > 0)
    CUDA_TRY(h, cudaMemcpy2D(idx, sizeof(int32_t) * h->nodes, h->d_idx, sizeof(int32_t) * h->ipad,
                             sizeof(int32_t) * h->nodes, 18, cudaMemcpyDeviceToHost));
  if (h->idx_folded) {
    // folded bounce-back slots lie outside [0, nodes): report them as -1
    for (int64_t e = 0; e < 18 * h->nodes; ++e)
      if (idx[e] < 0 || idx[e] >= h->nodes) idx[e] = -1;
  }
  return LBM_OK;
}

static int kernels_per_step(const lbm_t *h) {
  switch (h->cfg.variant) {
    case LBM_TS: return 2;
    case LBM_CG: {
      if (h->cfg.addressing == LBM_INDIRECT)
        return (int)((h->nodes + h->cg_B - 1) / std::max<int64_t>(h->cg_B, 1)) + (h->cfg.periodic[2] ? 1 : 0);
      const int slab = h->cg_k - 1;
      return (h->cfg.nz + slab - 1) / slab + (h->cfg.periodic[2] ? 1 : 0);
    }
    case LBM_SWAP:
      return h->cfg.addressing == LBM_INDIRECT ? 2 : swap_tiles(h).ncolours;
    default: return 1;
  }
}

lbm_status lbm_get_info(const lbm_t *h, lbm_info *info) {
  if (!h || !info) return fail(nullptr, LBM_ERR_INVALID_ARG, "NULL argument");
  memset(info, 0, sizeof *info);
  info->cells = h->cells;
  info->nodes = h->nodes;
  info->storage_nodes = h->slots;
  info->state_bytes = (int64_t)h->state_bytes * (h->d_B ? 2 : 1);
  info->index_bytes = h->index_bytes;
  info->steps = h->steps;
  info->natural = is_natural(h);
  info->kernels_per_step = kernels_per_step(h);
  info->f16_scale = h->scale;
  info->reduce_blocks = h->partial_blocks;
  info->tile_staged = h->swap_tma ? 1 : 0;
  info->pair_z = (h->grid.zpair || h->grid.ypair || use_npairs(h)) ? 1 : 0;
  return LBM_OK;
}

// ---------------------------------------------------------------------------
static float choose_scale(const lbm_t *h, double dev_init) {
  if (h->cfg.precision != LBM_F16S) return 1.0f;
  if (h->cfg.f16_scale > 0.0) return (float)h->cfg.f16_scale;
  // largest deviation expected: the initial state's, or the velocity a body
  // force can drive through the box (channel estimate g L^2 / (8 nu)) times
  // the largest 3 w_i c.u term; map it to about 2^12 so the FP16 values stay
  // normal across many decades below it
  const double nu = h->cfg.omega > 0 ? (1.0 / h->cfg.omega - 0.5) / 3.0 : 1.0;
  const double gmag = std::sqrt(h->cfg.force[0] * h->cfg.force[0] + h->cfg.force[1] * h->cfg.force[1] +
                                h->cfg.force[2] * h->cfg.force[2]);
  const double L = std::max(h->cfg.nx, std::max(h->cfg.ny, h->cfg.nz));
  const double dforce = 3.0 / 18.0 * gmag * L * L / (8.0 * std::max(nu, 1e-6));
  double dmax = std::max(dev_init, dforce);
  if (!(dmax > 1e-12)) dmax = 1e-6;
  return (float)std::ldexp(1.0, (int)std::floor(std::log2(4096.0 / dmax)));
}

lbm_status lbm_init(lbm_t *h, const double *rho, const double *u, int on_device) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID_ARG, "handle is NULL");
  if (!h->has_geometry) return fail(h, LBM_ERR_STATE, "no geometry");
  const int64_t n = h->nn;
  double dev = 0.0;
  const double *drho = rho, *du = u;
  TempBuf trho(h, rho && !on_device ? sizeof(double) * n : 0), tu(h, u && !on_device ? sizeof(double) * 3 * n : 0);
  if (!on_device) {
    const bool f16 = h->cfg.precision == LBM_F16S;
    if (rho) {
      if (f16)
        for (int64_t k = 0; k < n; ++k) dev = std::max(dev, std::fabs(rho[k] - 1.0) / 3.0);
      if (!trho.p) return fail(h, LBM_ERR_OOM, "init buffer");
      CUDA_TRY(h, cudaMemcpyAsync(trho.p, rho, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
      drho = static_cast<const double *>(trho.p);
    }
    if (u) {
      double um = 0.0;
      if (f16)
        for (int64_t k = 0; k < 3 * n; ++k) um = std::max(um, std::fabs(u[k]));
      dev += 3.0 / 18.0 * um * 2.0;
      if (!tu.p) return fail(h, LBM_ERR_OOM, "init buffer");
      CUDA_TRY(h, cudaMemcpyAsync(tu.p, u, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, h->stream));
      du = static_cast<const double *>(tu.p);
    }
  } else if (rho || u) {
    dev = 1e-3;  // device arrays are not inspected; assume a small perturbation
  }
  h->scale = choose_scale(h, dev);
  h->steps = 0;
  h->cg_o = 0;
  for (int i = 0; i < Q; ++i) h->map[i] = i;
  h->grid.zoff = 0;
  StateDesc d = state_desc(h);
  launch_put_state(d, nullptr, drho, du, h->stream);
  lbm_status st = check_launch(h, "put_state");
  if (st != LBM_OK) return st;
  if (!on_device) CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

lbm_status lbm_set_pdfs(lbm_t *h, const double *f, int on_device) {
  if (!h || !f) return fail(h, LBM_ERR_INVALID_ARG, "NULL argument");
  if (!h->has_geometry) return fail(h, LBM_ERR_STATE, "no geometry");
  const int64_t n = h->nn;
  const size_t bytes = sizeof(double) * Q * n;
  TempBuf tmp(h, on_device ? 0 : bytes);
  const double *df = f;
  double dev = 0.0;
  if (!on_device) {
    static const double w[Q] = {1. / 3, 1. / 18, 1. / 18, 1. / 18, 1. / 18, 1. / 18, 1. / 18,
                                1. / 36, 1. / 36, 1. / 36, 1. / 36, 1. / 36, 1. / 36, 1. / 36,
                                1. / 36, 1. / 36, 1. / 36, 1. / 36, 1. / 36};
    if (h->cfg.precision == LBM_F16S)
      for (int i = 0; i < Q; ++i)
        for (int64_t k = 0; k < n; ++k) dev = std::max(dev, std::fabs(f[i * n + k] - w[i]));
    if (!tmp.p) return fail(h, LBM_ERR_OOM, "state buffer");
    CUDA_TRY(h, cudaMemcpyAsync(tmp.p, f, bytes, cudaMemcpyHostToDevice, h->stream));
    df = static_cast<const double *>(tmp.p);
  } else {
    dev = 1e-3;
  }
  h->scale = choose_scale(h, dev);
  h->steps = 0;
  h->cg_o = 0;
  h->grid.zoff = 0;
  for (int i = 0; i < Q; ++i) h->map[i] = i;
  StateDesc d = state_desc(h);
  launch_put_state(d, df, nullptr, nullptr, h->stream);
  lbm_status st = check_launch(h, "put_state");
  if (st != LBM_OK) return st;
  if (!on_device) CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

lbm_status lbm_get_pdfs(lbm_t *h, double *f, int on_device) {
  if (!h || !f) return fail(h, LBM_ERR_INVALID_ARG, "NULL argument");
  if (!h->has_geometry) return fail(h, LBM_ERR_STATE, "no geometry");
  if (!is_natural(h)) return fail(h, LBM_ERR_STATE, "AA pattern state is natural only after an even step count");
  const int64_t n = h->nn;
  const size_t bytes = sizeof(double) * Q * n;
  TempBuf tmp(h, on_device ? 0 : bytes);
  double *df = f;
  if (!on_device) {
    if (!tmp.p) return fail(h, LBM_ERR_OOM, "state buffer");
    df = static_cast<double *>(tmp.p);
  }
  StateDesc d = state_desc(h);
  launch_get_state(d, df, h->stream);
  lbm_status st = check_launch(h, "get_state");
  if (st != LBM_OK) return st;
  if (!on_device) {
    CUDA_TRY(h, cudaMemcpyAsync(f, df, bytes, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  return LBM_OK;
}

lbm_status lbm_macroscopics(lbm_t *h, double *rho, double *u, int on_device) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID_ARG, "handle is NULL");
  if (!h->has_geometry) return fail(h, LBM_ERR_STATE, "no geometry");
  if (!is_natural(h)) return fail(h, LBM_ERR_STATE, "AA pattern state is natural only after an even step count");
  const int64_t n = h->nn;
  TempBuf tr(h, (!on_device && rho) ? sizeof(double) * n : 0), tu(h, (!on_device && u) ? sizeof(double) * 3 * n : 0);
  double *dr = rho, *du = u;
  if (!on_device) {
    if ((rho && !tr.p) || (u && !tu.p)) return fail(h, LBM_ERR_OOM, "moment buffers");
    dr = rho ? static_cast<double *>(tr.p) : nullptr;
    du = u ? static_cast<double *>(tu.p) : nullptr;
  }
  StateDesc d = state_desc(h);
  launch_macroscopics(d, dr, du, h->stream);
  lbm_status st = check_launch(h, "macroscopics");
  if (st != LBM_OK) return st;
  if (!on_device) {
    if (rho) CUDA_TRY(h, cudaMemcpyAsync(rho, dr, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    if (u) CUDA_TRY(h, cudaMemcpyAsync(u, du, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  return LBM_OK;
}

static lbm_status read_out2(lbm_t *h, double *mass, double *jx) {
  CUDA_TRY(h, cudaMemcpyAsync(h->h_out2, h->d_out2, sizeof(double) * 2, cudaMemcpyDeviceToHost, h->stream));
  lbm_status st = lbm_sync(h);
  if (st != LBM_OK) return st;
  if (mass) *mass = h->h_out2[0];
  if (jx) *jx = h->h_out2[1];
  return LBM_OK;
}

lbm_status lbm_flux(lbm_t *h, double *mass, double *jx) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID_ARG, "handle is NULL");
  if (!h->has_geometry) return fail(h, LBM_ERR_STATE, "no geometry");
  if (!is_natural(h)) return fail(h, LBM_ERR_STATE, "AA pattern state is natural only after an even step count");
  const int nb = reduce_blocks_for(h->nn);
  StateDesc d = state_desc(h);
  launch_flux_partials(d, h->d_partials, nb, h->stream);
  launch_final_sum(h->d_partials, nb, h->d_out2, h->stream);
  lbm_status st = check_launch(h, "flux");
  if (st != LBM_OK) return st;
  return read_out2(h, mass, jx);
}

// ---------------------------------------------------------------------------
// Time stepping.

// Compressed grid: ghost planes (periodic z), then slabs of k-1 planes in
// the order that keeps every overwritten plane's readers in earlier slabs.
// Returns the number of reduction partials written when red.
static lbm_status cg_step_indirect(lbm_t *h, bool red, int *red_blocks) {
  const KernelKey k = key_of(h, red);
  StepParams p = params_of(h);
  const int64_t o_old = h->cg_o, o_new = o_old == 0 ? h->cg_K : 0;
  void *A_old = shifted(h->d_A, cg_ind_offset(h, o_old), h->cfg.precision);
  void *A_new = shifted(h->d_A, cg_ind_offset(h, o_new), h->cfg.precision);
  if (h->cfg.periodic[2])
    launch_cg_ind_ghost(A_old, h->npad, h->cfg.precision, h->cfg.layout == LBM_AOS, h->nodes, h->cg_nfirst,
                        h->cg_nlast, h->stream);
  p.A = A_old;
  p.B = A_new;
  p.idx = h->d_cidx;
  const int bs = h->cfg.block_size > 0 ? h->cfg.block_size : 128;
  const int npt = h->cfg.nodes_per_thread > 0 ? h->cfg.nodes_per_thread : 1;
  const int64_t N = h->nodes, B = std::max<int64_t>(h->cg_B, 1);
  const int64_t nslab = (N + B - 1) / B;
  int used = 0;
  for (int64_t sl = 0; sl < nslab; ++sl) {
    int64_t a, b;
    if (o_new > o_old) {  // descending
      b = N - sl * B;
      a = std::max<int64_t>(0, b - B);
    } else {
      a = sl * B;
      b = std::min<int64_t>(N, a + B);
    }
    p.slab0 = a;
    p.slab1 = b;
    LaunchShape L;
    L.grid = dim3((unsigned)std::max<int64_t>(1, (b - a + (int64_t)bs * npt - 1) / ((int64_t)bs * npt)));
    L.block = dim3(bs);
    L.stream = h->stream;
    p.partials = h->d_partials + 2 * used;
    launch_cg_ind_slab(p, k, L);
    used += (int)L.grid.x;
  }
  h->cg_o = (int)o_new;
  if (red_blocks) *red_blocks = used;
  return LBM_OK;
}

static lbm_status cg_step(lbm_t *h, bool red, int *red_blocks) {
  if (h->cfg.addressing == LBM_INDIRECT) return cg_step_indirect(h, red, red_blocks);
  const KernelKey k = key_of(h, red);
  StepParams p = params_of(h);
  const int o_old = h->cg_o, o_new = o_old == 0 ? h->cg_k : 0;
  if (h->cfg.periodic[2]) launch_cg_ghost(p, h->cfg.precision, h->cfg.layout == LBM_AOS, o_old, h->stream);
  const int slab = h->cg_k - 1, nz = h->cfg.nz;
  p.zo_read = o_old;
  p.zo_write = o_new;
  int used = 0;
  const int nslab = (nz + slab - 1) / slab;
  for (int s = 0; s < nslab; ++s) {
    int z0, z1;
    if (o_new > o_old) {  // descending
      z1 = nz - s * slab;
      z0 = std::max(0, z1 - slab);
    } else {
      z0 = s * slab;
      z1 = std::min(nz, z0 + slab);
    }
    p.z0 = z0;
    p.z1 = z1;
    LaunchShape L = shape_of(h);  // its grid z covers nz with the planes per thread; refit to the slab
    const int npt = (h->cfg.nz + (int)L.grid.z - 1) / std::max(1, (int)L.grid.z);
    L.grid.z = (unsigned)std::min<int64_t>((z1 - z0 + npt - 1) / npt, 65535);
    if (h->grid.ypair) L.grid.y = (unsigned)((h->cfg.ny / 2 + (int)L.block.y - 1) / (int)L.block.y);  // word rows
    p.partials = h->d_partials + 2 * used;
    launch_step_kernel_cg(p, k, L);
    used += (int)blocks_of(L);
  }
  h->cg_o = o_new;
  h->grid.zoff = o_new;
  if (red_blocks) *red_blocks = used;
  return LBM_OK;
}

static lbm_status swap_step(lbm_t *h, bool red, int *red_blocks) {
  const KernelKey k = key_of(h, red);
  StepParams p = params_of(h);
  if (h->cfg.addressing == LBM_INDIRECT) {
    // collide into the reversed slots (the AA pattern's even kernel), then
    // exchange the PDFs of every link
    const LaunchShape L = shape_of(h);
    launch_step_kernel(VAR_AA, 0, p, k, L);
    launch_swap_links(p, h->cfg.precision, h->cfg.layout == LBM_AOS, h->stream);
    if (red_blocks) *red_blocks = (int)blocks_of(L);
    return LBM_OK;
  }
  SwapTiles t = swap_tiles(h);
  if (t.pairs) {
    // the swap runs on the grid of pair words: nz/2 planes, npad/2 words
    p.g.nz = h->cfg.nz / 2;
    p.g.zpair = 0;
    p.npad = h->npad / 2;
  }
  int used = 0;
  for (int c = 0; c < t.ncolours; ++c) {
    t.colour = c;
    p.partials = h->d_partials + 2 * used;
    if (h->swap_tma) {
      used += launch_swap_pass_tma(p, t, k, &h->swap_map, h->nsm, h->stream);
    } else {
      launch_swap_pass(p, t, k, h->stream);
      used += swap_blocks(t, h->cfg.periodic[0], h->cfg.periodic[1], h->cfg.periodic[2], c);
    }
  }
  if (red_blocks) *red_blocks = used;
  return LBM_OK;
}

static lbm_status one_step(lbm_t *h, bool red, int *red_blocks = nullptr) {
  if (red_blocks) *red_blocks = (int)blocks_of(shape_of(h));
  const KernelKey k = key_of(h, red);
  const LaunchShape L = shape_of(h);
  const int v = h->cfg.variant;
  switch (v) {
    case LBM_TS: {
      StepParams p = params_of(h);
      if (h->grid.zpair) {
        const LaunchShape L2 = zpair_shape_of(h);
        if (red_blocks) *red_blocks = (int)blocks_of(L2);
        launch_step_kernel(VAR_TS, 2, p, k, L2);
        launch_step_kernel(VAR_TS, 3, p, key_of(h, false), L2);
      } else {
        launch_step_kernel(VAR_TS, 0, p, k, L);
        launch_step_kernel(VAR_TS, 1, p, key_of(h, false), L);
      }
      break;
    }
    case LBM_OS_PUSH:
    case LBM_OS_PULL: {
      StepParams p = params_of(h);
      const int var = v == LBM_OS_PUSH ? VAR_OS_PUSH : VAR_OS_PULL;
      if (h->grid.zpair) {
        const LaunchShape L2 = zpair_shape_of(h);
        if (red_blocks) *red_blocks = (int)blocks_of(L2);
        launch_step_kernel(var, 4, p, k, L2);
      } else {
        launch_step_kernel(var, h->cfg.store_hint ? 2 : 0, p, k, L);
      }
      std::swap(h->d_A, h->d_B);
      break;
    }
    case LBM_AA: {
      StepParams p = params_of(h);
      if (h->grid.zpair) {
        const LaunchShape L2 = zpair_shape_of(h);
        if (red_blocks) *red_blocks = (int)blocks_of(L2);
        launch_step_kernel(VAR_AA, 4 + (int)(h->steps & 1), p, k, L2);
      } else if (use_npairs(h)) {
        const LaunchShape L2 = npair_shape_of(h);
        if (red_blocks) *red_blocks = (int)blocks_of(L2);
        launch_step_kernel(VAR_AA, 6 + (int)(h->steps & 1), p, k, L2);
      } else {
        launch_step_kernel(VAR_AA, (int)(h->steps & 1), p, k, L);
      }
      break;
    }
    case LBM_ET: {
      StepParams p = params_of(h);
      if (h->grid.zpair) {
        const LaunchShape L2 = zpair_shape_of(h);
        if (red_blocks) *red_blocks = (int)blocks_of(L2);
        launch_step_kernel(VAR_ET, 1, p, k, L2);
      } else if (use_npairs(h)) {
        const LaunchShape L2 = npair_shape_of(h);
        if (red_blocks) *red_blocks = (int)blocks_of(L2);
        launch_step_kernel(VAR_ET, 2, p, k, L2);
      } else {
        launch_step_kernel(VAR_ET, 0, p, k, L);
      }
      int nm[Q];
      for (int i = 0; i < Q; ++i) nm[i] = h->map[OPP(i)];
      memcpy(h->map, nm, sizeof nm);
      break;
    }
    case LBM_CG: {
      lbm_status st = cg_step(h, red, red_blocks);
      if (st != LBM_OK) return st;
      break;
    }
    case LBM_SWAP: {
      lbm_status st = swap_step(h, red, red_blocks);
      if (st != LBM_OK) return st;
      break;
    }
  }
  lbm_status st = check_launch(h, "step");
  if (st != LBM_OK) return st;
  ++h->steps;
  return LBM_OK;
}

lbm_status lbm_step(lbm_t *h, int n) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID_ARG, "handle is NULL");
  if (!h->has_geometry) return fail(h, LBM_ERR_STATE, "no geometry");
  if (n < 0) return fail(h, LBM_ERR_INVALID_ARG, "negative step count");
  for (int t = 0; t < n; ++t) {
    lbm_status st = one_step(h, false);
    if (st != LBM_OK) return st;
  }
  return LBM_OK;
}

lbm_status lbm_step_flux(lbm_t *h, int n, double *mass, double *jx) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID_ARG, "handle is NULL");
  if (!h->has_geometry) return fail(h, LBM_ERR_STATE, "no geometry");
  if (n < 1) return fail(h, LBM_ERR_INVALID_ARG, "step count must be >= 1");
  if (!is_natural(h)) return fail(h, LBM_ERR_STATE, "AA pattern state is natural only after an even step count");
  int nred = 0;
  lbm_status st = one_step(h, true, &nred);
  if (st != LBM_OK) return st;
  launch_final_sum(h->d_partials, nred, h->d_out2, h->stream);
  st = check_launch(h, "final_sum");
  if (st != LBM_OK) return st;
  for (int t = 1; t < n; ++t) {
    st = one_step(h, false);
    if (st != LBM_OK) return st;
  }
  return read_out2(h, mass, jx);
}

lbm_status lbm_solve_permeability(lbm_t *h, int32_t check, double tol, int64_t max_steps, double *permeability,
                                  double *mass, double *flux, int64_t *steps) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID_ARG, "handle is NULL");
  if (check < 2 || (check & 1)) return fail(h, LBM_ERR_INVALID_ARG, "check interval must be even and >= 2");
  if (!(tol >= 0.0) || max_steps < check) return fail(h, LBM_ERR_INVALID_ARG, "tol >= 0, max_steps >= check");
  if (!(h->cfg.omega > 0.0)) return fail(h, LBM_ERR_INVALID_ARG, "permeability needs omega > 0");
  const int64_t cells = (int64_t)h->cfg.nx * h->cfg.ny * h->cfg.nz;
  const double nu = (1.0 / h->cfg.omega - 0.5) / 3.0, gx = h->cfg.force[0];
  double m = 0.0, j = 0.0, prev = 0.0;
  bool have_prev = false, steady = false;
  int64_t done = 0;
  while (done + check <= max_steps) {
    // the flux of the state this round starts from
    lbm_status st = lbm_step_flux(h, check, &m, &j);
    if (st != LBM_OK) return st;
    done += check;
    steady = have_prev && std::fabs(j - prev) < tol * std::fabs(j);
    if (steady) break;
    prev = j;
    have_prev = true;
  }
  if (permeability) *permeability = gx != 0.0 ? nu * (j / (double)cells) / gx : NAN;
  if (mass) *mass = m;
  if (flux) *flux = j;
  if (steps) *steps = done;
  if (!steady) return fail(h, LBM_ERR_NOT_CONVERGED, "flux not steady after %lld steps", (long long)done);
  return LBM_OK;
}

}  // extern "C"
