// Compressed grid (Sec. 4, Fig. 2, Tab. 3) on a full grid, pull form.
// (Kernels use DirectNode from lbm_core.cuh.)
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
#include "lbm_steps.cuh"  // zp_collide_pair

namespace lbmk {

// Resident blocks per SM of the node-list slab kernel (as the other node-list
// kernels: one more block than the full-grid ones in FP32/FP16).
template <class C>
constexpr int step_min_cg() {
  return C::kMinBlocks == 3 ? 4 : C::kMinBlocks;
}

// One node of a slab: gather at the old offset (the grid's zoff), collide,
// store at the new offset.  FAST: no wall or solid link.
template <bool FAST, class C, int AOS, bool FORCE, class Node>
__device__ __forceinline__ void cg_node(const StepParams &p, Node &nd, const Lattice<C, AOS> &A,
                                        int64_t shift, double &m, double &j) {
  using T = typename C::T;
  T d[Q];
  d[0] = A.ld(0, nd.s);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const int src = nd.template nbf<FAST>(p, OPP(i));
    d[i] = (FAST || src >= 0) ? A.ld(i, src) : A.ld(OPP(i), nd.s);
  }
  T drho, rjx;
  collide_stored<C, FORCE>(d, coll_of<T>(p), p.scale, p.inv_scale, drho, rjx);
  m += 1.0 + (double)drho;
  j += (double)rjx;
  nd.launder_all();
  const int64_t w = nd.s + shift;
#pragma unroll
  for (int i = 0; i < Q; ++i) A.st(i, w, d[i]);
}

// Planes [z0, z1) of one sweep; the launch's grid covers (x, y) with 2D
// blocks and grid z over the slab's planes.  p.g.zoff is the old offset
// (plus the ghost plane), p.g.zghost is set on a periodic z axis.
template <class C, int AOS, bool IND, bool FORCE, bool RED>
__global__ void __launch_bounds__(256, C::kMinBlocks) k_cg_slab(StepParams p) {
  chain_wait();
  Lattice<C, AOS> A{static_cast<typename C::S *>(p.A), p.npad, p.scale, p.inv_scale};
  const int64_t shift = p.g.sxy * (int64_t)(p.zo_write - p.zo_read);
  double m = 0.0, j = 0.0;
  for (int z = p.z0 + blockIdx.z; z < p.z1; z += gridDim.z) {
    DirectNode nd;
    if (!nd.init_it(p, z)) continue;
    if (nd.fast)
      cg_node<true, C, AOS, FORCE>(p, nd, A, shift, m, j);
    else
      cg_node<false, C, AOS, FORCE>(p, nd, A, shift, m, j);
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

// Copy plane nz-1 to ghost plane -1 and plane 0 to ghost plane nz (offset zo),
// raw storage values, all 19 arrays.
template <class S, int AOS>
__global__ void k_cg_ghost(S *A, int64_t npad, Grid g, int zo) {
  chain_wait();
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

// ---------------------------------------------------------------------------
// FP16 / FP32 storage in y pairs (Grid::ypair): cells y and y + ny/2 of a
// row share one 4- or 8-byte word of every array (PairWord), so one thread
// updates both with one access per word; z pairs would not survive the
// plane shifts.
// Across the seam between the halves (word row 0 against word row ny/2 - 1)
// the neighbour word holds the two cells the other way round.  The per-node
// arithmetic is that of cg_node, so the PDFs equal the unpaired ones bit for
// bit.

// Node of the y-pair layout for the general case (a wall face next to either
// cell): slots from coordinates at the read offset; along a periodic z axis
// the ghost planes stand in for the wrapped neighbours, as in DirectNode.
struct YPairNode {
  int x, y, z, s;
  static constexpr bool fast = false;
  __device__ __forceinline__ void set(const Grid &g, int x_, int y_, int z_) {
    x = x_;
    y = y_;
    z = z_;
    s = (int)grid_slot(g, x, y, z);
  }
  __device__ __forceinline__ void launder_all() { s = launder(s); }
  template <bool FAST>
  __device__ __forceinline__ int nbf(const StepParams &p, int i) const {
    return nb(p, i);
  }
  __device__ __forceinline__ int nb(const StepParams &p, int i) const {
    const Grid &g = p.g;
    int a = x + CX(i), b = y + CY(i), c = z + CZ(i);
    if (!wrap_axis(a, g.nx, g.px) || !wrap_axis(b, g.ny, g.py)) return -1;
    if (!g.pz && (c < 0 || c >= g.nz)) return -1;
    return (int)grid_slot(g, a, b, c);
  }
};

// FP16 y pairs at four resident blocks per SM (64 registers; the loads are
// neighbour words, as in the AA odd step: 256^3 73.7 against 68.8 GFLUP/s
// at three); FP32 pairs at PairWord's two.
template <class C, bool FORCE, bool RED>
__global__ void __launch_bounds__(256, (std::is_same<C, CodecF16S>::value ? 4 : PairWord<C>::kMinBlocks))
    k_cg_slab_yp(StepParams p) {
  chain_wait();
  using PW = PairWord<C>;
  using W = typename PW::W;
  const Grid &g = p.g;
  const int H = g.ny >> 1;
  const int pw = (int)(g.sxy >> 1);  // words per plane
  const int x = blockIdx.x * blockDim.x + threadIdx.x, yw = blockIdx.y * blockDim.y + threadIdx.y;
  const int shift_w = pw * (p.zo_write - p.zo_read);
  double m = 0.0, j = 0.0;
  if (x < g.nx && yw < H) {
    W *A = static_cast<W *>(p.A);
    const int64_t nw = p.npad >> 1;
    const bool row = (g.px || (x > 0 && x < g.nx - 1)) && (g.py || (yw > 0 && yw < H - 1));
    const int dxm = x == 0 ? g.nx - 1 : -1, dxp = x == g.nx - 1 ? 1 - g.nx : 1;
    for (int z = p.z0 + blockIdx.z; z < p.z1; z += gridDim.z) {
      if (row && (g.pz || (z > 0 && z < g.nz - 1))) {
        const int w = x + (int)g.sx * yw + pw * (z + g.hz + (int)g.zoff);
        W v[Q];
        v[0] = A[w];
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          // source cell x - c_i; z neighbours are the adjacent planes (ghost
          // planes on a periodic axis); along y the seam exchanges halves
          const int ex = CX(i) > 0 ? dxm : (CX(i) < 0 ? dxp : 0);
          int ey = 0;
          bool seam = false;
          if (CY(i) > 0) {
            seam = yw == 0;
            ey = seam ? (H - 1) * (int)g.sx : -(int)g.sx;
          } else if (CY(i) < 0) {
            seam = yw == H - 1;
            ey = seam ? -(H - 1) * (int)g.sx : (int)g.sx;
          }
          const W t = A[i * nw + (w + ex + ey - CZ(i) * pw)];
          v[i] = seam ? PW::swap(t) : t;
        }
        zp_collide_pair<C, FORCE>(v, p, m, j);
        const int ws = launder(w) + shift_w;
#pragma unroll
        for (int i = 0; i < Q; ++i) A[i * nw + ws] = v[i];
      } else {
        const Lattice<C, 0> L{static_cast<typename C::S *>(p.A), p.npad, p.scale, p.inv_scale};
        const int64_t shift = g.sxy * (int64_t)(p.zo_write - p.zo_read);
        for (int h = 0; h < 2; ++h) {
          YPairNode a;
          a.set(g, x, yw + h * H, z);
          cg_node<false, C, 0, FORCE>(p, a, L, shift, m, j);
        }
      }
    }
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

template <class C, int AOS, bool IND, bool FORCE, bool RED>
struct LaunchCG {
  static void run(const StepParams &p, const LaunchShape &L) {
    StepParams q = p;
    q.g.zoff = p.zo_read;
    q.g.zghost = p.g.pz;
    if (p.g.ypair) {
      if constexpr (kPairable<C> && AOS == 0)
        launch_chained(k_cg_slab_yp<C, FORCE, RED>, L.grid, L.block, 0, L.stream, q);
      return;
    }
    launch_chained(k_cg_slab<C, AOS, false, FORCE, RED>, L.grid, L.block, 0, L.stream, q);
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
      launch_chained(k_cg_ghost<double, 1>, grid, 256, 0, s, static_cast<double *>(p.A), p.npad, p.g, zo);
    else
      launch_chained(k_cg_ghost<double, 0>, grid, 256, 0, s, static_cast<double *>(p.A), p.npad, p.g, zo);
  } else if (precision == 1) {
    if (aos)
      launch_chained(k_cg_ghost<float, 1>, grid, 256, 0, s, static_cast<float *>(p.A), p.npad, p.g, zo);
    else
      launch_chained(k_cg_ghost<float, 0>, grid, 256, 0, s, static_cast<float *>(p.A), p.npad, p.g, zo);
  } else {
    if (aos)
      launch_chained(k_cg_ghost<__half, 1>, grid, 256, 0, s, static_cast<__half *>(p.A), p.npad, p.g, zo);
    else
      launch_chained(k_cg_ghost<__half, 0>, grid, 256, 0, s, static_cast<__half *>(p.A), p.npad, p.g, zo);
  }
}

}  // namespace lbmk

namespace lbmk {

// ---------------------------------------------------------------------------
// Compressed grid on a node list.  The post-collision state of node n lives at
// slot n + o + G, o alternating between 0 and K, G = nodes of the last plane
// (room for the lower ghost copies).  Neighbour references are "unwrapped":
// a link that wraps across the periodic z faces points at a ghost copy
// (m - N below node 0, m + N above node N - 1) instead of node m, so every
// link spans at most D node numbers.  A sweep reads at offset o and writes at
// o'; writing slot n + o' overwrites the old data of position n + o' - o,
// whose readers lie within D of it; with slabs of B consecutive nodes and
// K >= D + B, descending slabs when o' > o and ascending slabs otherwise, all
// of those readers are in earlier slabs.  Ghost copies are refreshed before
// each sweep on a periodic z axis.

constexpr int32_t kCgSolid = INT32_MIN;

// Unwrapped index cidx[i-1][n] (kCgSolid for a solid/wall link), the largest
// |u - n| (atomicMax into dmax), and the node counts of planes 0 and nz-1.
__global__ void k_cg_ind_prep(const int32_t *idx, int64_t ipad, const int32_t *cells, int64_t N, int nx, int ny,
                              int nz, int32_t *cidx, int *dmax, int *count_first, int *count_last) {
  const int64_t plane = (int64_t)nx * ny;
  int local_max = 0;
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    const int z = (int)(cells[n] / plane);
    if (z == 0) atomicAdd(count_first, 1);
    if (z == nz - 1) atomicAdd(count_last, 1);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int32_t m = idx[(int64_t)(i - 1) * ipad + n];
      int64_t u = m;
      if (m < 0) {
        cidx[(int64_t)(i - 1) * ipad + n] = kCgSolid;
        continue;
      }
      if (CZ(i) < 0 && z == 0) u = (int64_t)m - N;
      if (CZ(i) > 0 && z == nz - 1) u = (int64_t)m + N;
      cidx[(int64_t)(i - 1) * ipad + n] = (int32_t)u;
      const int64_t d = u > n ? u - n : n - u;
      if (d > local_max) local_max = (int)d;
    }
  }
  atomicMax(dmax, local_max);
}

void launch_cg_ind_prep(const int32_t *idx, int64_t ipad, const int32_t *cells, int64_t N, int nx, int ny, int nz,
                        int32_t *cidx, int *counters, cudaStream_t s) {
  if (N == 0) return;
  const unsigned grid = (unsigned)std::min<int64_t>((N + 255) / 256, 1 << 16);
  k_cg_ind_prep<<<grid, 256, 0, s>>>(idx, ipad, cells, N, nx, ny, nz, cidx, counters, counters + 1, counters + 2);
}

// Lower ghosts: copies of the last-plane nodes at positions m - N; upper
// ghosts: copies of the first-plane nodes at m + N.  A points at position 0
// of the current offset.
template <class S, int AOS>
__global__ void k_cg_ind_ghost(S *A, int64_t npad, int64_t N, int64_t nfirst, int64_t nlast) {
  chain_wait();
  const int64_t per = nfirst + nlast;
  const int64_t total = per * Q;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / per);
    const int64_t r = t % per;
    int64_t src, dst;
    if (r < nlast) {
      src = N - nlast + r;
      dst = src - N;
    } else {
      src = r - nlast;
      dst = src + N;
    }
    if (AOS)
      A[dst * Q + i] = A[src * Q + i];
    else
      A[(int64_t)i * npad + dst] = A[(int64_t)i * npad + src];
  }
}

void launch_cg_ind_ghost(void *A, int64_t npad, int precision, int aos, int64_t N, int64_t nfirst, int64_t nlast,
                         cudaStream_t s) {
  const int64_t total = (nfirst + nlast) * Q;
  if (total == 0) return;
  const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, 1 << 20);
  if (precision == 0) {
    if (aos) launch_chained(k_cg_ind_ghost<double, 1>, grid, 256, 0, s, static_cast<double *>(A), npad, N, nfirst, nlast);
    else launch_chained(k_cg_ind_ghost<double, 0>, grid, 256, 0, s, static_cast<double *>(A), npad, N, nfirst, nlast);
  } else if (precision == 1) {
    if (aos) launch_chained(k_cg_ind_ghost<float, 1>, grid, 256, 0, s, static_cast<float *>(A), npad, N, nfirst, nlast);
    else launch_chained(k_cg_ind_ghost<float, 0>, grid, 256, 0, s, static_cast<float *>(A), npad, N, nfirst, nlast);
  } else {
    if (aos) launch_chained(k_cg_ind_ghost<__half, 1>, grid, 256, 0, s, static_cast<__half *>(A), npad, N, nfirst, nlast);
    else launch_chained(k_cg_ind_ghost<__half, 0>, grid, 256, 0, s, static_cast<__half *>(A), npad, N, nfirst, nlast);
  }
}

// One slab [z0, z1) of node numbers (p.z0/p.z1 reused as node bounds): gather
// from p.A (old offset) through the unwrapped index p.idx, collide, store to
// p.B (new offset).
template <class C, int AOS, bool IND, bool FORCE, bool RED>
__global__ void __launch_bounds__(256, (step_min_cg<C>())) k_cg_ind_slab(StepParams p) {
  chain_wait();
  using T = typename C::T;
  Lattice<C, AOS> A{static_cast<typename C::S *>(p.A), p.npad, p.scale, p.inv_scale};
  Lattice<C, AOS> B{static_cast<typename C::S *>(p.B), p.npad, p.scale, p.inv_scale};
  double m = 0.0, j = 0.0;
  for (int64_t n64 = p.slab0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n64 < p.slab1;
       n64 += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)n64;
    T d[Q];
    d[0] = A.ld(0, n);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int32_t src = __ldg(p.idx + (int64_t)(OPP(i) - 1) * p.ipad + n);
      d[i] = src != kCgSolid ? A.ld(i, src) : A.ld(OPP(i), n);
    }
    T drho, rjx;
    collide_stored<C, FORCE>(d, coll_of<T>(p), p.scale, p.inv_scale, drho, rjx);
    m += 1.0 + (double)drho;
    j += (double)rjx;
    const int w = launder(n);
#pragma unroll
    for (int i = 0; i < Q; ++i) B.st(i, w, d[i]);
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

template <class C, int AOS, bool IND, bool FORCE, bool RED>
struct LaunchCGInd {
  static void run(const StepParams &p, const LaunchShape &L) {
    launch_chained(k_cg_ind_slab<C, AOS, false, FORCE, RED>, L.grid, L.block, 0, L.stream, p);
  }
};

void launch_cg_ind_slab(const StepParams &p, const KernelKey &k, const LaunchShape &L) {
  dispatch<LaunchCGInd>(k.precision, k.aos, false, k.force, k.red, p, L);
}

}  // namespace lbmk
