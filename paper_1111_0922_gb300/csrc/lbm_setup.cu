// Set-up and read-out kernels: sphere-pack geometry, fluid-node list and IDX
// (Sec. 1, indirect addressing), the esoteric twist's packed index (Sec. 7),
// moving a natural state into and out of each scheme's storage, moments, and
// the FP64 mass/flux reductions with a fixed summation order.
#include <algorithm>

#include "lbm_dispatch.cuh"
#include "lbm_internal.h"

namespace lbmk {

// ---------------------------------------------------------------------------
// Geometry: a cell is solid iff its centre is within radius of a sphere
// centre (minimum image on periodic axes).  Integer positions in units of
// 1/unit cells make the test exact.  One block per sphere walks the sphere's
// bounding box; concurrent writes all store the same byte.
__device__ __forceinline__ int64_t floor_div(int64_t a, int64_t b) {
  int64_t q = a / b;
  return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

__device__ __forceinline__ int64_t min_image(int64_t d, int64_t len, int periodic) {
  if (!periodic) return d;
  d %= len;
  if (d < 0) d += len;
  if (2 * d > len) d -= len;
  return d;
}

__global__ void k_sphere_mask(uint8_t *solid, int nx, int ny, int nz, int px, int py, int pz, int64_t nsph,
                              const int64_t *centres, int64_t radius, int64_t unit) {
  const int n[3] = {nx, ny, nz};
  const int per[3] = {px, py, pz};
  const int64_t r2 = radius * radius;
  for (int64_t sph = blockIdx.x; sph < nsph; sph += gridDim.x) {
    int64_t c[3], lo[3], ext[3];
    for (int a = 0; a < 3; ++a) {
      c[a] = centres[3 * sph + a];
      lo[a] = -floor_div(-(c[a] - radius), unit);  // ceil
      const int64_t hi = floor_div(c[a] + radius, unit);
      ext[a] = hi - lo[a] + 1;
    }
    const int64_t total = ext[0] * ext[1] * ext[2];
    for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
      int64_t v[3] = {lo[0] + t % ext[0], lo[1] + (t / ext[0]) % ext[1], lo[2] + t / (ext[0] * ext[1])};
      bool inside = true;
      int64_t d2 = 0;
      for (int a = 0; a < 3; ++a) {
        int64_t w = v[a];
        if (w < 0 || w >= n[a]) {
          if (!per[a]) {
            inside = false;
            break;
          }
          w %= n[a];
          if (w < 0) w += n[a];
        }
        v[a] = w;
        const int64_t d = min_image(w * unit - c[a], (int64_t)n[a] * unit, per[a]);
        d2 += d * d;
      }
      if (inside && d2 <= r2) solid[v[0] + (int64_t)nx * (v[1] + (int64_t)ny * v[2])] = 1;
    }
  }
}

void launch_sphere_mask(uint8_t *solid, int nx, int ny, int nz, const int *periodic, int64_t nsph,
                        const int64_t *centres, int64_t radius, int64_t unit, cudaStream_t s) {
  if (nsph <= 0) return;
  const int grid = (int)std::min<int64_t>(nsph, 1 << 20);
  k_sphere_mask<<<grid, 256, 0, s>>>(solid, nx, ny, nz, periodic[0], periodic[1], periodic[2], nsph, centres,
                                     radius, unit);
}

// ---------------------------------------------------------------------------
// Stream compaction: three passes over tiles of SCAN_TILE items (count per
// tile, exclusive scan of the tile counts in one block, then per-tile
// numbering).  Pred decides which items are kept.
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int64_t SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

struct FluidPred {  // keep cells that are not solid
  const uint8_t *solid;
  __device__ __forceinline__ bool operator()(int64_t c) const { return solid == nullptr || solid[c] == 0; }
};
struct FlagPred {  // keep nonzero flags
  const int32_t *flag;
  __device__ __forceinline__ bool operator()(int64_t c) const { return flag[c] != 0; }
};

template <class P>
__global__ void k_scan_count(P pred, int64_t n, int32_t *tile_counts) {
  __shared__ int warp_sum[SCAN_THREADS / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int cnt = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k)
    if (base + k < n && pred(base + k)) ++cnt;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < SCAN_THREADS / 32; ++w) t += warp_sum[w];
    tile_counts[blockIdx.x] = t;
  }
}

// One block: exclusive scan of the tile counts in place, total in counts[ntiles].
__global__ void k_scan_tiles(int32_t *counts, int64_t ntiles) {
  __shared__ int32_t buf[1024];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < ntiles; base += 1024) {
    const int64_t i = base + threadIdx.x;
    const int32_t v = i < ntiles ? counts[i] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // Hillis-Steele inclusive scan
      const int32_t add = threadIdx.x >= (unsigned)o ? buf[threadIdx.x - o] : 0;
      __syncthreads();
      buf[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < ntiles) counts[i] = carry + buf[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += buf[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) counts[ntiles] = carry;
}

template <class P>
__global__ void k_scan_apply(P pred, int64_t n, const int32_t *tile_offsets, int32_t *number, int32_t *list) {
  __shared__ int warp_sum[SCAN_THREADS / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  bool keep[SCAN_ITEMS];
  int cnt = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    keep[k] = base + k < n && pred(base + k);
    cnt += keep[k];
  }
  // exclusive scan of cnt across the block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_sum[warp] = incl;
  __syncthreads();
  int before = 0;
  for (int w = 0; w < warp; ++w) before += warp_sum[w];
  int next = tile_offsets[blockIdx.x] + before + incl - cnt;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    if (base + k >= n) break;
    if (keep[k]) {
      if (number) number[base + k] = next;
      if (list) list[next] = (int32_t)(base + k);
      ++next;
    } else if (number) {
      number[base + k] = -1;
    }
  }
}

int64_t scan_scratch_elems(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

template <class P>
static int64_t compact(P pred, int64_t n, int32_t *number, int32_t *list, int32_t *scratch, cudaStream_t s) {
  const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles == 0) return 0;
  k_scan_count<<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(pred, n, scratch);
  k_scan_tiles<<<1, 1024, 0, s>>>(scratch, tiles);
  k_scan_apply<<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(pred, n, scratch, number, list);
  int32_t total = 0;
  cudaMemcpyAsync(&total, scratch + tiles, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  return total;
}

int64_t build_node_list(const uint8_t *solid, int64_t ncell, int32_t *node_of, int32_t *cells, int32_t *scratch,
                        int64_t scratch_elems, cudaStream_t s) {
  if (scratch_elems < scan_scratch_elems(ncell)) return -1;
  return compact(FluidPred{solid}, ncell, node_of, cells, scratch, s);
}

// ---------------------------------------------------------------------------
// IDX[i-1][k]: node reached from node k along c_i, -1 for a wall or solid.
__device__ __forceinline__ int64_t cell_step(int x, int y, int z, int i, int nx, int ny, int nz, int px, int py,
                                             int pz) {
  int a = x + CX(i), b = y + CY(i), c = z + CZ(i);
  if (!wrap_axis(a, nx, px) || !wrap_axis(b, ny, py) || !wrap_axis(c, nz, pz)) return -1;
  return (int64_t)a + (int64_t)nx * ((int64_t)b + (int64_t)ny * c);
}

__global__ void k_build_idx(const int32_t *cells, const int32_t *node_of, int64_t N, int nx, int ny, int nz, int px,
                            int py, int pz, int32_t *idx, int64_t ipad) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = cells[k];
    const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((int64_t)nx * ny));
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int64_t d = cell_step(x, y, z, i, nx, ny, nz, px, py, pz);
      idx[(int64_t)(i - 1) * ipad + k] = d >= 0 ? node_of[d] : -1;
    }
  }
}

static unsigned grid_for(int64_t n, int threads) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 1 << 20));
}

void launch_build_idx(const int32_t *cells, const int32_t *node_of, int64_t N, int nx, int ny, int nz,
                      const int *periodic, int32_t *idx, int64_t ipad, cudaStream_t s) {
  if (N == 0) return;
  k_build_idx<<<grid_for(N, 256), 256, 0, s>>>(cells, node_of, N, nx, ny, nz, periodic[0], periodic[1], periodic[2],
                                               idx, ipad);
}

// Bounce-back folded into IDX for the AA pattern on SoA storage: a solid
// link k of node s becomes the slot that, in the array the odd step uses with
// IDX[k], lands on the node's own slot of the reflected direction:
//   read  f_opp(k)(x) <- array k at IDX[k], BB: array opp(k) at s
//   write g_k(x)      -> array k at IDX[k], BB: array opp(k) at s
// so IDX'[k][s] = s + (opp(k) - k) npad in both cases.  Values are < 0 or
// >= npad (>= the node count) exactly for folded links.
__global__ void k_fold_idx(int32_t *idx, int64_t ipad, int64_t N, int64_t npad) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 1; k < Q; ++k) {
      int32_t &v = idx[(int64_t)(k - 1) * ipad + s];
      if (v < 0) v = (int32_t)(s + (int64_t)(OPP(k) - k) * npad);
    }
  }
}

void launch_fold_idx(int32_t *idx, int64_t ipad, int64_t N, int64_t npad, cudaStream_t s) {
  if (N == 0) return;
  k_fold_idx<<<grid_for(N, 256), 256, 0, s>>>(idx, ipad, N, npad);
}

// ---------------------------------------------------------------------------
// Esoteric twist index.  Position x + c_i (odd i) on an extended box with a
// one-cell margin: wrapped on periodic axes, in the margin beyond a wall.
__device__ __forceinline__ int64_t ext_cell(int x, int y, int z, int i, int nx, int ny, int nz, int px, int py, int pz,
                                            bool &in_box) {
  int a = x + CX(i), b = y + CY(i), c = z + CZ(i);
  if (px) wrap_axis(a, nx, 1);
  if (py) wrap_axis(b, ny, 1);
  if (pz) wrap_axis(c, nz, 1);
  in_box = a >= 0 && a < nx && b >= 0 && b < ny && c >= 0 && c < nz;
  return (int64_t)(a + 1) + (int64_t)(nx + 2) * ((int64_t)(b + 1) + (int64_t)(ny + 2) * (c + 1));
}

__global__ void k_et_mark(const int32_t *cells, const int32_t *node_of, int64_t N, int nx, int ny, int nz, int px,
                          int py, int pz, int32_t *ghost_flag) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = cells[k];
    const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((int64_t)nx * ny));
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
      bool in_box;
      const int64_t e = ext_cell(x, y, z, i, nx, ny, nz, px, py, pz, in_box);
      bool ghost = !in_box;
      if (in_box) {
        const int64_t d = cell_step(x, y, z, i, nx, ny, nz, px, py, pz);
        ghost = node_of[d] < 0;
      }
      if (ghost) ghost_flag[e] = 1;
    }
  }
}

__global__ void k_et_pack(const int32_t *cells, const int32_t *node_of, int64_t N, int nx, int ny, int nz, int px,
                          int py, int pz, const int32_t *ghost_id, int32_t *etidx, int64_t ipad) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = cells[k];
    const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((int64_t)nx * ny));
#pragma unroll
    for (int kk = 0; kk < 9; ++kk) {
      const int i = 2 * kk + 1;
      bool in_box;
      const int64_t e = ext_cell(x, y, z, i, nx, ny, nz, px, py, pz, in_box);
      int64_t slot = -1;
      if (in_box) slot = node_of[cell_step(x, y, z, i, nx, ny, nz, px, py, pz)];
      if (slot < 0) slot = N + ghost_id[e];
      const int64_t dm = cell_step(x, y, z, i + 1, nx, ny, nz, px, py, pz);
      const bool solid_m = dm < 0 || node_of[dm] < 0;
      etidx[(int64_t)kk * ipad + k] = (int32_t)((uint32_t)slot | (solid_m ? 0x80000000u : 0u));
    }
  }
}

int64_t build_et_index(const int32_t *cells, const int32_t *node_of, int64_t N, int nx, int ny, int nz,
                       const int *periodic, int32_t *ghost_map, int32_t *etidx, int64_t ipad, int32_t *scratch,
                       int64_t scratch_elems, cudaStream_t s) {
  const int64_t next = (int64_t)(nx + 2) * (ny + 2) * (nz + 2);
  if (scratch_elems < scan_scratch_elems(next)) return -1;
  cudaMemsetAsync(ghost_map, 0, sizeof(int32_t) * next, s);
  if (N > 0)
    k_et_mark<<<grid_for(N, 256), 256, 0, s>>>(cells, node_of, N, nx, ny, nz, periodic[0], periodic[1], periodic[2],
                                              ghost_map);
  // number the ghosts in place: ghost_map becomes ghost ids (-1 where none)
  const int64_t G = compact(FlagPred{ghost_map}, next, ghost_map, nullptr, scratch, s);
  if (N > 0)
    k_et_pack<<<grid_for(N, 256), 256, 0, s>>>(cells, node_of, N, nx, ny, nz, periodic[0], periodic[1], periodic[2],
                                              ghost_map, etidx, ipad);
  return G;
}

// Fixed-order sum of per-block partials: thread t adds partials t, t+256, ...
// in order, then a fixed shuffle tree.
__global__ void __launch_bounds__(256) k_final_sum(const double *partials, int nblocks, double *out) {
  double m = 0.0, j = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    m += partials[2 * b];
    j += partials[2 * b + 1];
  }
  __shared__ double sm[8], sj[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m += __shfl_xor_sync(0xffffffffu, m, o);
    j += __shfl_xor_sync(0xffffffffu, j, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sm[threadIdx.x >> 5] = m;
    sj[threadIdx.x >> 5] = j;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < 8; ++w) {
      a += sm[w];
      b += sj[w];
    }
    out[0] = a;
    out[1] = b;
  }
}

template <class C>
void state_op_t(int op, const StateDesc &d, const double *fin, double *fout, const double *rho,
                double *rout, const double *u, double *uout, double *partials, int nb, cudaStream_t s);
static void state_op(int precision, int op, const StateDesc &d, const double *fin, double *fout, const double *rho,
                     double *rout, const double *u, double *uout, double *partials, int nb, cudaStream_t s) {
  if (precision == 0)
    state_op_t<CodecF64>(op, d, fin, fout, rho, rout, u, uout, partials, nb, s);
  else if (precision == 1)
    state_op_t<CodecF32>(op, d, fin, fout, rho, rout, u, uout, partials, nb, s);
  else
    state_op_t<CodecF16S>(op, d, fin, fout, rho, rout, u, uout, partials, nb, s);
}

void launch_put_state(const StateDesc &d, const double *f_nat, const double *rho, const double *u, cudaStream_t s) {
  state_op(d.k.precision, 0, d, f_nat, (double *)nullptr, rho,
                     (double *)nullptr, u, (double *)nullptr, (double *)nullptr, 0, s);
}
void launch_get_state(const StateDesc &d, double *f_nat, cudaStream_t s) {
  state_op(d.k.precision, 1, d, (const double *)nullptr, f_nat,
                     (const double *)nullptr, (double *)nullptr, (const double *)nullptr, (double *)nullptr,
                     (double *)nullptr, 0, s);
}
void launch_macroscopics(const StateDesc &d, double *rho, double *u, cudaStream_t s) {
  state_op(d.k.precision, 2, d, (const double *)nullptr,
                     (double *)nullptr, (const double *)nullptr, rho, (const double *)nullptr, u, (double *)nullptr,
                     0, s);
}
int reduce_blocks_for(int64_t nnodes) { return (int)std::max<int64_t>(1, std::min<int64_t>((nnodes + 255) / 256, 2048)); }
void launch_flux_partials(const StateDesc &d, double *partials, int nblocks, cudaStream_t s) {
  state_op(d.k.precision, 3, d, (const double *)nullptr,
                     (double *)nullptr, (const double *)nullptr, (double *)nullptr, (const double *)nullptr,
                     (double *)nullptr, partials, nblocks, s);
}
void launch_final_sum(const double *partials, int nblocks, double *out, cudaStream_t s) {
  k_final_sum<<<1, 256, 0, s>>>(partials, nblocks, out);
}

}  // namespace lbmk
