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
// tile of a later colour is left reversed for that tile to complete.
#include <algorithm>

#include "lbm_dispatch.cuh"
#include "lbm_internal.h"

namespace lbmk {

struct SwapPass {
  int tx, ty, tz;              // tile extent
  int ntx, nty, ntz;           // tiles per axis
  int cx, cy, cz;              // colours per axis
  int colour;                  // colour of this pass (cx-fastest)
  int start[3], count[3];      // tiles of this colour per axis: start + 2k (or the odd tail tile)
};

__device__ __forceinline__ int axis_colour(int t, int nt, int periodic) {
  if (nt == 1) return 0;
  if (periodic && (nt & 1)) return t == nt - 1 ? 2 : (t & 1);
  return t & 1;
}

// Index of a neighbour-tile offset (ox, oy, oz) in {-1, 0, 1}^3.
__host__ __device__ constexpr int tile_bit(int ox, int oy, int oz) { return (ox + 1) + 3 * ((oy + 1) + 3 * (oz + 1)); }

// One pass: the tiles of one colour.  Thread (lx, ly, lz) of the block owns
// cell org + (lx, ly, lz) of its tile.
template <class C, int AOS, bool IND, bool FORCE, bool RED>
__global__ void __launch_bounds__(256, 2) k_swap_pass(StepParams p, SwapPass sp) {
  using T = typename C::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *S = reinterpret_cast<T *>(smem_raw);
  __shared__ unsigned earlier_mask, self_mask;
  Lattice<C, AOS> L{static_cast<typename C::S *>(p.A), p.npad, p.scale, p.inv_scale};
  const Grid &g = p.g;
  const int TN = sp.tx * sp.ty * sp.tz;
  const int tile[3] = {sp.start[0] + 2 * (int)blockIdx.x, sp.start[1] + 2 * (int)blockIdx.y,
                       sp.start[2] + 2 * (int)blockIdx.z};
  const int org[3] = {tile[0] * sp.tx, tile[1] * sp.ty, tile[2] * sp.tz};
  const int t = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  if (t == 0) {
    // classify the 26 neighbouring tiles once per block
    const int nt[3] = {sp.ntx, sp.nty, sp.ntz};
    const int per[3] = {g.px, g.py, g.pz};
    unsigned em = 0, sm = 0;
    for (int oz = -1; oz <= 1; ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          const int o[3] = {ox, oy, oz};
          int nb[3];
          bool exists = true;
          for (int a = 0; a < 3; ++a) {
            nb[a] = tile[a] + o[a];
            if (nb[a] < 0 || nb[a] >= nt[a]) {
              if (!per[a]) exists = false;
              nb[a] = (nb[a] + nt[a]) % nt[a];
            }
          }
          if (!exists) continue;
          if (nb[0] == tile[0] && nb[1] == tile[1] && nb[2] == tile[2]) {
            sm |= 1u << tile_bit(ox, oy, oz);
            continue;
          }
          const int col = axis_colour(nb[0], nt[0], per[0]) +
                          sp.cx * (axis_colour(nb[1], nt[1], per[1]) + sp.cy * axis_colour(nb[2], nt[2], per[2]));
          if (col < sp.colour) em |= 1u << tile_bit(ox, oy, oz);
        }
    earlier_mask = em;
    self_mask = sm;
  }
  const int lx = threadIdx.x, ly = threadIdx.y, lz = threadIdx.z;
  // extent of this tile inside the box (the last tile of an axis may be cut)
  const int ex = min(sp.tx, g.nx - org[0]), ey = min(sp.ty, g.ny - org[1]), ez = min(sp.tz, g.nz - org[2]);
  DirectNode nd;
  bool active = lx < ex && ly < ey && lz < ez;
  if (active) {
    nd.x = org[0] + lx;
    nd.y = org[1] + ly;
    nd.z = org[2] + lz;
    active = nd.setup(g);
  }
  double m = 0.0, jsum = 0.0;
  if (active) {
    T d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = L.ld(i, nd.s);
    T drho, rjx;
    collide_stored<C, FORCE>(d, coll_of<T>(p), p.scale, p.inv_scale, drho, rjx);
    m = 1.0 + (double)drho;
    jsum = (double)rjx;
#pragma unroll
    for (int i = 0; i < Q; ++i) S[i * TN + t] = d[i];
  }
  __syncthreads();
  if (active) {
    // Gather every incoming value first (the loads from earlier tiles are
    // independent and overlap), then write: the remote slots written below
    // belong to earlier tiles and are never read by this pass again.
    const unsigned em = earlier_mask, sm = self_mask;
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
      // source slot, or -1 across a wall or from a solid cell (the fast path
      // has neither: walls lie on tile faces and there is no solid cell)
      const int src = nd.fast ? nd.nb_fast(p, OPP(i)) : nd.nb(p, OPP(i));
      if (src < 0) {
        v[i] = S[OPP(i) * TN + t];  // bounce-back: the node's own reversed PDF
        continue;
      }
      if (in_x && in_y && in_z) {
        v[i] = S[i * TN + t + dx + sp.tx * (dy + sp.ty * dz)];  // inside the tile
        continue;
      }
      const int bit = tile_bit(in_x ? 0 : dx, in_y ? 0 : dy, in_z ? 0 : dz);
      if (sm & (1u << bit)) {
        // the tile is its own neighbour across a periodic face
        const int wx = in_x ? lx + dx : (dx < 0 ? ex - 1 : 0);
        const int wy = in_y ? ly + dy : (dy < 0 ? ey - 1 : 0);
        const int wz = in_z ? lz + dz : (dz < 0 ? ez - 1 : 0);
        v[i] = S[i * TN + wx + sp.tx * (wy + sp.ty * wz)];
      } else if (em & (1u << bit)) {
        // earlier tile: its reversed slot holds the PDF for us; ours goes there
        remote[i] = src;
        v[i] = L.ld(OPP(i), src);
      } else {
        v[i] = S[OPP(i) * TN + t];  // a later tile completes the link
      }
    }
    nd.launder_all();
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      L.st(i, nd.s, v[i]);
      if (i > 0 && remote[i] >= 0) L.st(OPP(i), remote[i], S[OPP(i) * TN + t]);
    }
  }
  if (RED) block_reduce_store(m, jsum, p.partials);
}

template <class C, int AOS, bool IND, bool FORCE, bool RED>
struct LaunchSwap {
  static void run(const StepParams &p, const SwapPass &sp, size_t smem, dim3 blocks, cudaStream_t s) {
    auto k = k_swap_pass<C, AOS, false, FORCE, RED>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<blocks, dim3(sp.tx, sp.ty, sp.tz), smem, s>>>(p, sp);
  }
};

// tiles are at most 32 x 4 x 2 = 256 cells (one thread each)
size_t swap_smem_bytes(const SwapTiles &t, int precision) {
  return (size_t)Q * t.tx * t.ty * t.tz * (precision == 0 ? 8 : 4);
}

static void axis_set(int nt, int periodic, int colour, int &start, int &count) {
  if (nt == 1) {
    start = 0;
    count = colour == 0 ? 1 : 0;
    return;
  }
  if (periodic && (nt & 1)) {
    if (colour == 2) {
      start = nt - 1;
      count = 1;
    } else {
      start = colour;
      count = (nt - 1 - colour + 1) / 2;  // even tiles 0..nt-3 or odd 1..nt-2
    }
    return;
  }
  start = colour;
  count = colour < nt ? (nt - colour + 1) / 2 : 0;
}

void launch_swap_pass(const StepParams &p, const SwapTiles &t, const KernelKey &k, cudaStream_t s) {
  SwapPass sp;
  sp.tx = t.tx;
  sp.ty = t.ty;
  sp.tz = t.tz;
  sp.ntx = t.ntx;
  sp.nty = t.nty;
  sp.ntz = t.ntz;
  auto ncol = [](int nt, int periodic) { return nt == 1 ? 1 : ((periodic && (nt & 1)) ? 3 : 2); };
  sp.cx = ncol(t.ntx, p.g.px);
  sp.cy = ncol(t.nty, p.g.py);
  sp.cz = ncol(t.ntz, p.g.pz);
  sp.colour = t.colour;
  const int c0 = t.colour % sp.cx, c1 = (t.colour / sp.cx) % sp.cy, c2 = t.colour / (sp.cx * sp.cy);
  axis_set(t.ntx, p.g.px, c0, sp.start[0], sp.count[0]);
  axis_set(t.nty, p.g.py, c1, sp.start[1], sp.count[1]);
  axis_set(t.ntz, p.g.pz, c2, sp.start[2], sp.count[2]);
  if (sp.count[0] * sp.count[1] * sp.count[2] == 0) return;
  const dim3 blocks(sp.count[0], sp.count[1], sp.count[2]);
  dispatch<LaunchSwap>(k.precision, k.aos, false, k.force, k.red, p, sp, swap_smem_bytes(t, k.precision), blocks, s);
}

int swap_colours(const SwapTiles &t, int px, int py, int pz) {
  auto ncol = [](int nt, int periodic) { return nt == 1 ? 1 : ((periodic && (nt & 1)) ? 3 : 2); };
  return ncol(t.ntx, px) * ncol(t.nty, py) * ncol(t.ntz, pz);
}

int swap_blocks(const SwapTiles &t, int px, int py, int pz, int colour) {
  auto ncol = [](int nt, int periodic) { return nt == 1 ? 1 : ((periodic && (nt & 1)) ? 3 : 2); };
  const int cx = ncol(t.ntx, px), cy = ncol(t.nty, py);
  int st, c0, c1, c2;
  axis_set(t.ntx, px, colour % cx, st, c0);
  axis_set(t.nty, py, (colour / cx) % cy, st, c1);
  axis_set(t.ntz, pz, colour / (cx * cy), st, c2);
  return c0 * c1 * c2;
}

}  // namespace lbmk

namespace lbmk {

// Swap on a node list (Sec. 5, Tab. 4), order-free form.  After the nodes
// have been collided into their reversed slots (the AA pattern's even kernel:
// the post-collision PDF along c_i sits in the node's slot of the opposite
// direction), every link is completed by exchanging the two PDFs that travel
// along it.  Thread n owns the links to its neighbours along the nine odd
// directions: it exchanges slot opp(i) of n with slot i of IDX[i][n].  Local
// slots (even directions) and remote slots (odd directions) are disjoint and
// each link has one owner, so the exchanges need no ordering; a solid or wall
// link needs none (its reversed slot already holds the bounced-back PDF).
template <class S, int AOS>
__global__ void __launch_bounds__(256) k_swap_links(S *A, int64_t npad, const int32_t *idx, int64_t ipad,
                                                    int64_t nnodes) {
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < nnodes; n += (int64_t)gridDim.x * blockDim.x) {
    // load every value of the nine links, then store (no load waits on a store)
    int m[Q];
    S va[Q], vb[Q];
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
      m[i] = __ldg(idx + (int64_t)(i - 1) * ipad + n);
      if (m[i] < 0) continue;
      va[i] = AOS ? A[n * Q + OPP(i)] : A[(int64_t)OPP(i) * npad + n];
      vb[i] = AOS ? A[(int64_t)m[i] * Q + i] : A[(int64_t)i * npad + m[i]];
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
      if (m[i] < 0) continue;
      (AOS ? A[n * Q + OPP(i)] : A[(int64_t)OPP(i) * npad + n]) = vb[i];
      (AOS ? A[(int64_t)m[i] * Q + i] : A[(int64_t)i * npad + m[i]]) = va[i];
    }
  }
}

void launch_swap_links(const StepParams &p, int precision, int aos, cudaStream_t s) {
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((p.nnodes + 255) / 256, 1 << 20));
  if (precision == 0) {
    if (aos) k_swap_links<double, 1><<<grid, 256, 0, s>>>(static_cast<double *>(p.A), p.npad, p.idx, p.ipad, p.nnodes);
    else k_swap_links<double, 0><<<grid, 256, 0, s>>>(static_cast<double *>(p.A), p.npad, p.idx, p.ipad, p.nnodes);
  } else if (precision == 1) {
    if (aos) k_swap_links<float, 1><<<grid, 256, 0, s>>>(static_cast<float *>(p.A), p.npad, p.idx, p.ipad, p.nnodes);
    else k_swap_links<float, 0><<<grid, 256, 0, s>>>(static_cast<float *>(p.A), p.npad, p.idx, p.ipad, p.nnodes);
  } else {
    if (aos) k_swap_links<__half, 1><<<grid, 256, 0, s>>>(static_cast<__half *>(p.A), p.npad, p.idx, p.ipad, p.nnodes);
    else k_swap_links<__half, 0><<<grid, 256, 0, s>>>(static_cast<__half *>(p.A), p.npad, p.idx, p.ipad, p.nnodes);
  }
}

}  // namespace lbmk
