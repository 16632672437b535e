// Fused collide-and-propagate kernels for the order-free propagation schemes:
// two-step (Sec. 2), one-step push and pull (Sec. 3), AA pattern (Sec. 6) and
// esoteric twist (Sec. 7).  One thread updates one node per loop iteration
// (grid-stride loop, so a launch may give each thread several nodes).  All
// kernels load the 19 PDFs of a node, run the collision in registers and
// store 19 PDFs: q loads + q stores per update, no read-for-ownership on the
// GPU (full-sector stores allocate in L2 without a DRAM read).
#pragma once

#include "lbm_dispatch.cuh"
#include "lbm_internal.h"

namespace lbmk {

template <class C, int AOS, bool CS = false>
__device__ __forceinline__ Lattice<C, AOS, CS> lattice_of(void *p, const StepParams &P) {
  Lattice<C, AOS, CS> L;
  L.p = static_cast<typename C::S *>(p);
  L.npad = P.npad;
  L.scale = P.scale;
  L.inv_scale = P.inv_scale;
  return L;
}

// Launch bounds of the step kernels: at most LBM_STEP_MAXT threads per block
// and at least C::kMinBlocks resident blocks per SM (the register budget
// that keeps enough loads in flight to cover HBM latency).
#ifndef LBM_STEP_MAXT
#define LBM_STEP_MAXT 256
#endif
// Node-list kernels get one more resident block in FP32/FP16 (64 registers):
// their PDF loads wait for IDX loads, two memory round trips per node, so
// they need more warps in flight to cover HBM latency.
template <class C, bool IND>
constexpr int step_min_blocks() {
  return (IND && C::kMinBlocks == 3) ? 4 : C::kMinBlocks;
}
#define LBM_STEP_BOUNDS \
  __launch_bounds__(LBM_STEP_MAXT, (step_min_blocks<C, std::is_same<Node, IndirectNode>::value>()))
#define LBM_STEP_BOUNDS_IND __launch_bounds__(LBM_STEP_MAXT, (step_min_blocks<C, IND>()))
// The esoteric twist with FP16 storage runs faster with 64 registers and four
// resident blocks on full grids too (measured: +12 % at 256^3).
template <class C, bool IND>
constexpr int et_min_blocks() {
  return sizeof(typename C::S) == 2 ? 4 : step_min_blocks<C, IND>();
}
#define LBM_ET_BOUNDS __launch_bounds__(LBM_STEP_MAXT, (et_min_blocks<C, IND>()))

template <bool IND>
using NodeOf = typename std::conditional<IND, IndirectNode, DirectNode>::type;

template <class C, bool FORCE>
__device__ __forceinline__ void run_collision(typename C::T (&d)[Q], const StepParams &p, double &m, double &j) {
  using T = typename C::T;
  T drho, rjx;
  collide_stored<C, FORCE>(d, coll_of<T>(p), p.scale, p.inv_scale, drho, rjx);
  m += 1.0 + (double)drho;
  j += (double)rjx;
}

// Iterate this thread's nodes: a flat grid-stride loop over the node list
// (IDX addressing), or the planes of this thread's (x, y) column (full grid).
#define LBM_NODE_LOOP(Node, it) for (int64_t it = Node::it_begin(p); it < Node::it_end(p); it += Node::it_step(p))

// ---------------------------------------------------------------------------
// Two-step, kernel 1 (Tab. 1, collision): A -> B at the same slot.
template <class C, int AOS, class Node, bool FORCE, bool RED>
__global__ void LBM_STEP_BOUNDS k_ts_collide(StepParams p) {
  chain_wait();
  using T = typename C::T;
  const auto A = lattice_of<C, AOS>(p.A, p);
  const auto B = lattice_of<C, AOS>(p.B, p);
  double m = 0.0, j = 0.0;
  LBM_NODE_LOOP(Node, it) {
    Node nd;
    if (!nd.init_it(p, it)) continue;
    T d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = A.ld(i, nd.s);
    run_collision<C, FORCE>(d, p, m, j);
    nd.launder_all();
#pragma unroll
    for (int i = 0; i < Q; ++i) B.st(i, nd.s, d[i]);
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

// Two-step, kernel 2 (Tab. 1, propagation), pull form: A_i(x) = B_i(x - c_i),
// or B_opp(i)(x) across a solid/wall link.  Raw copies: bit-exact.
// All 19 values are loaded before any store: a store to A might alias a later
// load from B as far as the compiler knows, which would serialise the copies.
template <bool FAST, class C, int AOS, class Node>
__device__ __forceinline__ void ts_stream_node(const StepParams &p, Node &nd, const Lattice<C, AOS> &A,
                                               const Lattice<C, AOS> &B) {
  typename C::S v[Q];
  v[0] = *B.at(0, nd.s);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const int src = nd.template nbf<FAST>(p, OPP(i));
    v[i] = (FAST || src >= 0) ? *B.at(i, src) : *B.at(OPP(i), nd.s);
  }
  nd.launder_all();
#pragma unroll
  for (int i = 0; i < Q; ++i) *A.at(i, nd.s) = v[i];
}

template <class C, int AOS, class Node>
__global__ void LBM_STEP_BOUNDS k_ts_stream(StepParams p) {
  chain_wait();
  const auto A = lattice_of<C, AOS>(p.A, p);
  const auto B = lattice_of<C, AOS>(p.B, p);
  LBM_NODE_LOOP(Node, it) {
    Node nd;
    if (!nd.init_it(p, it)) continue;
    if (nd.fast)
      ts_stream_node<true, C, AOS, Node>(p, nd, A, B);
    else
      ts_stream_node<false, C, AOS, Node>(p, nd, A, B);
  }
}

// One-step push (Fig. 1a,b): read A at the node, write B at the neighbours.
// FAST: the node has no solid or wall link (no bounce-back branch).
template <bool FAST, class C, int AOS, class Node, bool FORCE, class LB>
__device__ __forceinline__ void os_push_node(const StepParams &p, Node &nd, const Lattice<C, AOS> &A,
                                             const LB &B, double &m, double &j) {
  using T = typename C::T;
  T d[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) d[i] = A.ld(i, nd.s);
  run_collision<C, FORCE>(d, p, m, j);
  nd.launder_all();
  B.st(0, nd.s, d[0]);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const int dst = nd.template nbf<FAST>(p, i);
    if (FAST || dst >= 0)
      B.st(i, dst, d[i]);
    else
      B.st(OPP(i), nd.s, d[i]);
  }
}

template <class C, int AOS, class Node, bool FORCE, bool RED, bool CS>
__global__ void LBM_STEP_BOUNDS k_os_push(StepParams p) {
  chain_wait();
  const auto A = lattice_of<C, AOS>(p.A, p);
  const auto B = lattice_of<C, AOS, CS>(p.B, p);
  double m = 0.0, j = 0.0;
  LBM_NODE_LOOP(Node, it) {
    Node nd;
    if (!nd.init_it(p, it)) continue;
    if (nd.fast)
      os_push_node<true, C, AOS, Node, FORCE>(p, nd, A, B, m, j);
    else
      os_push_node<false, C, AOS, Node, FORCE>(p, nd, A, B, m, j);
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

// One-step pull (Fig. 1c,d): gather from the neighbours in A, write B at the
// node.  The stored state is post-collision.
template <bool FAST, class C, int AOS, class Node, bool FORCE, class LB>
__device__ __forceinline__ void os_pull_node(const StepParams &p, Node &nd, const Lattice<C, AOS> &A,
                                             const LB &B, double &m, double &j) {
  using T = typename C::T;
  T d[Q];
  d[0] = A.ld(0, nd.s);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const int src = nd.template nbf<FAST>(p, OPP(i));
    d[i] = (FAST || src >= 0) ? A.ld(i, src) : A.ld(OPP(i), nd.s);
  }
  run_collision<C, FORCE>(d, p, m, j);
  nd.launder_all();
#pragma unroll
  for (int i = 0; i < Q; ++i) B.st(i, nd.s, d[i]);
}

template <class C, int AOS, class Node, bool FORCE, bool RED, bool CS>
__global__ void LBM_STEP_BOUNDS k_os_pull(StepParams p) {
  chain_wait();
  const auto A = lattice_of<C, AOS>(p.A, p);
  const auto B = lattice_of<C, AOS, CS>(p.B, p);
  double m = 0.0, j = 0.0;
  LBM_NODE_LOOP(Node, it) {
    Node nd;
    if (!nd.init_it(p, it)) continue;
    if (nd.fast)
      os_pull_node<true, C, AOS, Node, FORCE>(p, nd, A, B, m, j);
    else
      os_pull_node<false, C, AOS, Node, FORCE>(p, nd, A, B, m, j);
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

// AA pattern, even step (Fig. 5a,b): node-local; the post-collision PDF of
// direction i goes to the node's slot of the opposite direction.
template <class C, int AOS, class Node, bool FORCE, bool RED>
__global__ void LBM_STEP_BOUNDS k_aa_even(StepParams p) {
  chain_wait();
  using T = typename C::T;
  const auto A = lattice_of<C, AOS>(p.A, p);
  double m = 0.0, j = 0.0;
  LBM_NODE_LOOP(Node, it) {
    Node nd;
    if (!nd.init_it(p, it)) continue;
    T d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = A.ld(i, nd.s);
    run_collision<C, FORCE>(d, p, m, j);
    nd.launder_all();
#pragma unroll
    for (int i = 0; i < Q; ++i) A.st(OPP(i), nd.s, d[i]);
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

// AA pattern, odd step (Fig. 5c,d): f_i comes from the opposite slot of the
// node at x - c_i (own slot i across a solid link); the result goes to slot i
// of x + c_i (own opposite slot across a solid link).  Every slot written was
// read by the same thread.
template <bool FAST, class C, int AOS, class Node, bool FORCE>
__device__ __forceinline__ void aa_odd_node(const StepParams &p, Node &nd, const Lattice<C, AOS> &A, double &m,
                                            double &j) {
  using T = typename C::T;
  // Full-grid neighbours are recomputed after the collision; IDX entries are
  // loaded again for the stores (L1 hits) unless LBM_AA_HOLD_IDX keeps them
  // in registers across the collision.
#ifdef LBM_AA_HOLD_IDX
  constexpr bool kHold = std::is_same<Node, IndirectNode>::value;
#else
  constexpr bool kHold = false;
#endif
  int nb[Q];
  if (kHold) {
#pragma unroll
    for (int i = 1; i < Q; ++i) nb[i] = nd.nb(p, i);
  }
  T d[Q];
  d[0] = A.ld(0, nd.s);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const int src = kHold ? nb[OPP(i)] : nd.template nbf<FAST>(p, OPP(i));
    d[i] = (FAST || src >= 0) ? A.ld(OPP(i), src) : A.ld(i, nd.s);
  }
  run_collision<C, FORCE>(d, p, m, j);
  nd.launder_all();
  A.st(0, nd.s, d[0]);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const int dst = kHold ? nb[i] : nd.template nbf<FAST>(p, i);
    if (FAST || dst >= 0)
      A.st(i, dst, d[i]);
    else
      A.st(OPP(i), nd.s, d[i]);
  }
}

// Nodes the odd step may treat as having no bounce-back branch: full-grid
// nodes without wall or solid links, every node of a folded IDX.
__device__ __forceinline__ bool aa_fast(const DirectNode &nd, const StepParams &) { return nd.fast; }
__device__ __forceinline__ bool aa_fast(const IndirectNode &, const StepParams &p) { return p.idx_folded != 0; }

template <class C, int AOS, class Node, bool FORCE, bool RED>
__global__ void LBM_STEP_BOUNDS k_aa_odd(StepParams p) {
  chain_wait();
  const auto A = lattice_of<C, AOS>(p.A, p);
  double m = 0.0, j = 0.0;
  LBM_NODE_LOOP(Node, it) {
    Node nd;
    if (!nd.init_it(p, it)) continue;
    if (aa_fast(nd, p))
      aa_odd_node<true, C, AOS, Node, FORCE>(p, nd, A, m, j);
    else
      aa_odd_node<false, C, AOS, Node, FORCE>(p, nd, A, m, j);
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

// FP16 / FP32 storage on a full grid without solid cells, nodes in z pairs
// (Grid::zpair; AA pattern, two-step, one-step push and pull, and the
// esoteric twist on a periodic box): cells z and z + nz/2 of a column share
// one word of every array (PairWord), so one thread updates both with one
// access per word (half the load and store instructions and twice the bytes
// per access of one node per thread).  The two updates are the per-node ones
// above, node by node, so the results equal the one-node-per-thread kernels
// bit for bit.  Along z the pair's words are those of the column's
// neighbour plane, except across the seam between the halves (plane 0 <->
// plane nz/2 - 1), where the neighbour word holds the two cells the other
// way round.

// Node of the z-pair layout for the general case (a wall face next to either
// cell of the pair): neighbour slots from coordinates.
struct ZPairNode {
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
  // slot of the neighbour along c_i, or -1 across a wall
  __device__ __forceinline__ int nb(const StepParams &p, int i) const {
    int a = x + CX(i), b = y + CY(i), c = z + CZ(i);
    if (!wrap_axis(a, p.g.nx, p.g.px) || !wrap_axis(b, p.g.ny, p.g.py) || !wrap_axis(c, p.g.nz, p.g.pz)) return -1;
    return (int)grid_slot(p.g, a, b, c);
  }
};

// Resident 256-thread blocks per SM of the FP16 AA odd-step and one-step
// pair kernels: four (64 registers; 256^3: AA 82.1 against 80.0 GFLUP/s,
// pull 84.3 against 79.2, push 77.9 against 76.2 with the next plane
// prefetched at three); the others keep PairWord's three (four measured
// slower: AA even step 78.6, esoteric twist 69.8).
template <class C>
constexpr int pair_four_min_blocks() {
  return std::is_same<C, CodecF16S>::value ? 4 : PairWord<C>::kMinBlocks;
}

// Collide both cells of a pair word by word: v[i] holds f_i of the lower and
// of the upper cell, raw storage units.
template <class C, bool FORCE>
__device__ __forceinline__ void zp_collide_pair(typename PairWord<C>::W (&v)[Q], const StepParams &p, double &m,
                                                double &j) {
  using PW = PairWord<C>;
  float d[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) d[i] = PW::lo(v[i]);
  run_collision<C, FORCE>(d, p, m, j);
#pragma unroll
  for (int i = 0; i < Q; ++i) v[i] = PW::with_lo(v[i], d[i]);
#pragma unroll
  for (int i = 0; i < Q; ++i) d[i] = PW::hi(v[i]);
  run_collision<C, FORCE>(d, p, m, j);
#pragma unroll
  for (int i = 0; i < Q; ++i) v[i] = PW::with_hi(v[i], d[i]);
}

// Even step: node-local, the pair's post-collision PDFs go to the opposite
// slots of its own word.  The next pair plane's words are loaded before this
// plane's collision (a thread's planes are independent: the even step reads
// and writes the pair's own word only), so their latency overlaps the
// arithmetic (FP16 78.1 -> 80.3 GFLUP/s on 256^3 with four planes per
// thread; FP32 unchanged).
template <class C, bool FORCE, bool RED>
__global__ void __launch_bounds__(LBM_STEP_MAXT, (PairWord<C>::kMinBlocks)) k_aa_even_zp(StepParams p) {
  chain_wait();
  using W = typename PairWord<C>::W;
  const Grid &g = p.g;
  const int H = g.nz >> 1;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  double m = 0.0, j = 0.0;
  if (x < g.nx && y < g.ny) {
    W *A = static_cast<W *>(p.A);
    const int64_t nw = p.npad >> 1;  // words per array
    const int step = (int)g.sxy * (int)gridDim.z;
    int zw = blockIdx.z;
    int w = x + (int)g.sx * y + (int)g.sxy * zw;
    W v[Q];
    if (zw < H) {
#pragma unroll
      for (int i = 0; i < Q; ++i) v[i] = A[i * nw + w];
    }
    for (; zw < H; zw += gridDim.z) {
      W n[Q];
      if (zw + (int)gridDim.z < H) {
#pragma unroll
        for (int i = 0; i < Q; ++i) n[i] = A[i * nw + w + step];
      }
      zp_collide_pair<C, FORCE>(v, p, m, j);
      w = launder(w);  // recompute the store addresses instead of holding 19
#pragma unroll
      for (int i = 0; i < Q; ++i) A[OPP(i) * nw + w] = v[i];
      w += step;
#pragma unroll
      for (int i = 0; i < Q; ++i) v[i] = n[i];
    }
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

// Pair planes next to a column without a wall face (two-step and one-step
// schemes in z pairs): word of the pair at x + SIGN c_i and whether the seam
// exchanges its halves.
struct ZPairCol {
  int dxm, dxp, dym, dyp;  // word deltas to the -1 / +1 column, periodic wrap
  __device__ __forceinline__ void set(const Grid &g, int x, int y) {
    dxm = x == 0 ? g.nx - 1 : -1;
    dxp = x == g.nx - 1 ? 1 - g.nx : 1;
    dym = (y == 0 ? g.ny - 1 : -1) * (int)g.sx;
    dyp = (y == g.ny - 1 ? 1 - g.ny : 1) * (int)g.sx;
  }
  template <int SIGN>
  __device__ __forceinline__ int nbw(const Grid &g, int H, int w, int zw, int i, bool &seam) const {
    const int cx = SIGN * CX(i), cy = SIGN * CY(i), cz = SIGN * CZ(i);
    const int ex = cx < 0 ? dxm : (cx > 0 ? dxp : 0);
    const int ey = cy < 0 ? dym : (cy > 0 ? dyp : 0);
    int ez = 0;
    seam = false;
    if (cz < 0) {
      seam = zw == 0;
      ez = seam ? (H - 1) * (int)g.sxy : -(int)g.sxy;
    } else if (cz > 0) {
      seam = zw == H - 1;
      ez = seam ? -(H - 1) * (int)g.sxy : (int)g.sxy;
    }
    return w + ex + ey + ez;
  }
  // INNER: the pair's column is not on an x or y face and its plane is not
  // next to the seam, so the neighbour word is at the launch-uniform offset
  // c_i . (1, sx, sxy) and never across the seam
  template <int SIGN, bool INNER>
  __device__ __forceinline__ int nbw(const Grid &g, int H, int w, int zw, int i, bool &seam) const {
    if (INNER) {
      seam = false;
      return w + SIGN * (CX(i) + CY(i) * (int)g.sx + CZ(i) * (int)g.sxy);
    }
    return nbw<SIGN>(g, H, w, zw, i, seam);
  }
};

// Whether every active lane of the warp holds an interior column (no x or
// y face), decided per warp so that a warp with a face column takes the
// general path alone instead of running both.
__device__ __forceinline__ bool zp_inner_warp(const Grid &g, int x, int y) {
  return __all_sync(__activemask(), x > 0 && x < g.nx - 1 && y > 0 && y < g.ny - 1);
}
__device__ __forceinline__ bool zp_inner_plane(int H, int zw) { return zw > 0 && zw < H - 1; }
using InnerTag = std::true_type;
using FaceTag = std::false_type;

// a pair's column and plane have no wall face next to either cell
__device__ __forceinline__ bool zp_open_column(const Grid &g, int x, int y) {
  return (g.px || (x > 0 && x < g.nx - 1)) && (g.py || (y > 0 && y < g.ny - 1));
}
__device__ __forceinline__ bool zp_open_plane(const Grid &g, int H, int zw) { return g.pz || (zw > 0 && zw < H - 1); }

// AA pattern, odd step in z pairs: the words at x - c_i (opposite arrays)
// in, the words at x + c_i out.  A pair with a wall face next to either cell
// takes the per-node path.
template <class C, bool FORCE, bool RED>
__global__ void __launch_bounds__(LBM_STEP_MAXT, (pair_four_min_blocks<C>())) k_aa_odd_zp(StepParams p) {
  chain_wait();
  using PW = PairWord<C>;
  using W = typename PW::W;
  const Grid &g = p.g;
  const int H = g.nz >> 1;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  double m = 0.0, j = 0.0;
  if (x < g.nx && y < g.ny) {
    W *A = static_cast<W *>(p.A);
    const int64_t nw = p.npad >> 1;
    const bool col = zp_open_column(g, x, y);
    const bool inner = zp_inner_warp(g, x, y);
    for (int zw = blockIdx.z; zw < H; zw += gridDim.z) {
      auto pair = [&](auto tag) {
        constexpr bool INNER = decltype(tag)::value;
        const int w = x + (int)g.sx * y + (int)g.sxy * zw;
        W v[Q];
        {
          ZPairCol c;
          if (!INNER) c.set(g, x, y);
          v[0] = A[w];
#pragma unroll
          for (int i = 1; i < Q; ++i) {
            bool seam;
            const W t = A[OPP(i) * nw + c.template nbw<-1, INNER>(g, H, w, zw, i, seam)];
            v[i] = seam ? PW::swap(t) : t;
          }
        }
        zp_collide_pair<C, FORCE>(v, p, m, j);
        // recompute the addresses rather than hold them across the collision
        const int ws = launder(w), xs = launder(x), ys = launder(y);
        ZPairCol c;
        if (!INNER) c.set(g, xs, ys);
        A[ws] = v[0];
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          bool seam;
          const int d = c.template nbw<1, INNER>(g, H, ws, zw, i, seam);
          A[i * nw + d] = seam ? PW::swap(v[i]) : v[i];
        }
      };
      if (inner && zp_inner_plane(H, zw)) {
        pair(InnerTag{});
      } else if (col && zp_open_plane(g, H, zw)) {
        pair(FaceTag{});
      } else {
        const Lattice<C, 0> L = lattice_of<C, 0>(p.A, p);
        for (int h = 0; h < 2; ++h) {
          ZPairNode a;
          a.set(g, x, y, zw + h * H);
          aa_odd_node<false, C, 0, ZPairNode, FORCE>(p, a, L, m, j);
        }
      }
    }
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

// AA pattern on a node list (SoA, IDX with the bounce-back slots folded in)
// with FP16 storage, two consecutive nodes per thread: nodes 2t and 2t + 1
// share word t of every array, so the even step's node-local loads and
// stores move one 4-byte word for both, and the odd step loads both nodes'
// IDX entries of a direction as one 8-byte word and gathers the two PDFs
// into one register word.  The per-node arithmetic is that of the
// one-node-per-thread kernels (bit-identical results); the last node of an
// odd count takes the per-node path.  64 registers (four 256-thread blocks
// per SM; the odd kernel spills a few dozen bytes with a force), two pairs
// per thread by default: 512^3 sphere pack 50.4 against 45.4 GFLUP/s one
// node per thread (three blocks: 47.5; two: 43.2).  FP32 pairs (30.5-33.3
// against 34.7) measured slower and are not built.
template <class C, bool FORCE, bool RED>
__global__ void __launch_bounds__(LBM_STEP_MAXT, 4) k_aa_even_np(StepParams p) {
  chain_wait();
  using W = typename PairWord<C>::W;
  const int64_t nn = p.nnodes, nt = (nn + 1) >> 1;
  W *A = static_cast<W *>(p.A);
  const int64_t nw = p.npad >> 1;
  double m = 0.0, j = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
    if (2 * t + 1 < nn) {
      int w = (int)t;
      W v[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) v[i] = A[i * nw + w];
      zp_collide_pair<C, FORCE>(v, p, m, j);
      w = launder(w);
#pragma unroll
      for (int i = 0; i < Q; ++i) A[OPP(i) * nw + w] = v[i];
    } else {
      const Lattice<C, 0> L = lattice_of<C, 0>(p.A, p);
      typename C::T d[Q];
      const int s = (int)(2 * t);
#pragma unroll
      for (int i = 0; i < Q; ++i) d[i] = L.ld(i, s);
      run_collision<C, FORCE>(d, p, m, j);
      const int s2 = launder(s);
#pragma unroll
      for (int i = 0; i < Q; ++i) L.st(OPP(i), s2, d[i]);
    }
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

template <class C, bool FORCE, bool RED>
__global__ void __launch_bounds__(LBM_STEP_MAXT, 4) k_aa_odd_np(StepParams p) {
  chain_wait();
  using PW = PairWord<C>;
  using W = typename PW::W;
  using S = typename C::S;
  const int64_t nn = p.nnodes, nt = (nn + 1) >> 1;
  S *E = static_cast<S *>(p.A);
  W *A = static_cast<W *>(p.A);
  const int64_t nw = p.npad >> 1;
  const int2 *I = reinterpret_cast<const int2 *>(p.idx);
  const int64_t iw = p.ipad >> 1;  // IDX words (two nodes) per direction
  double m = 0.0, j = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
    if (2 * t + 1 < nn) {
      const int w = (int)t;
      W v[Q];
      v[0] = A[w];
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const int2 src = __ldg(I + (OPP(i) - 1) * iw + w);  // x - c_i of both nodes
        v[i] = PW::pack(E[OPP(i) * p.npad + src.x], E[OPP(i) * p.npad + src.y]);
      }
      zp_collide_pair<C, FORCE>(v, p, m, j);
      const int ws = launder(w);
      A[ws] = v[0];
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const int2 dst = __ldg(I + (i - 1) * iw + ws);  // x + c_i
        E[i * p.npad + dst.x] = PW::lo_s(v[i]);
        E[i * p.npad + dst.y] = PW::hi_s(v[i]);
      }
    } else {
      const Lattice<C, 0> L = lattice_of<C, 0>(p.A, p);
      IndirectNode nd;
      nd.init(p, 2 * t);
      aa_odd_node<true, C, 0, IndirectNode, FORCE>(p, nd, L, m, j);
    }
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

// Two-step, kernel 1 in z pairs: A -> B at the same words.
template <class C, bool FORCE, bool RED>
__global__ void __launch_bounds__(LBM_STEP_MAXT, PairWord<C>::kMinBlocks) k_ts_collide_zp(StepParams p) {
  chain_wait();
  using W = typename PairWord<C>::W;
  const Grid &g = p.g;
  const int H = g.nz >> 1;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  double m = 0.0, j = 0.0;
  if (x < g.nx && y < g.ny) {
    const W *A = static_cast<const W *>(p.A);
    W *B = static_cast<W *>(p.B);
    const int64_t nw = p.npad >> 1;
    for (int zw = blockIdx.z; zw < H; zw += gridDim.z) {
      int w = x + (int)g.sx * y + (int)g.sxy * zw;
      W v[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) v[i] = A[i * nw + w];
      zp_collide_pair<C, FORCE>(v, p, m, j);
      w = launder(w);
#pragma unroll
      for (int i = 0; i < Q; ++i) B[i * nw + w] = v[i];
    }
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

// Two-step, kernel 2 in z pairs: A_i(x) = B_i(x - c_i), raw word copies.
template <class C>
__global__ void __launch_bounds__(LBM_STEP_MAXT, PairWord<C>::kMinBlocks) k_ts_stream_zp(StepParams p) {
  chain_wait();
  using PW = PairWord<C>;
  using W = typename PW::W;
  const Grid &g = p.g;
  const int H = g.nz >> 1;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  W *A = static_cast<W *>(p.A);
  const W *B = static_cast<const W *>(p.B);
  const int64_t nw = p.npad >> 1;
  const bool col = zp_open_column(g, x, y);
  const bool inner = zp_inner_warp(g, x, y);
  ZPairCol c;
  c.set(g, x, y);
  for (int zw = blockIdx.z; zw < H; zw += gridDim.z) {
    auto pair = [&](auto tag) {
      constexpr bool INNER = decltype(tag)::value;
      int w = x + (int)g.sx * y + (int)g.sxy * zw;
      W v[Q];
      v[0] = B[w];
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        bool seam;
        const W t = B[i * nw + c.template nbw<-1, INNER>(g, H, w, zw, i, seam)];
        v[i] = seam ? PW::swap(t) : t;
      }
      w = launder(w);
#pragma unroll
      for (int i = 0; i < Q; ++i) A[i * nw + w] = v[i];
    };
    if (inner && zp_inner_plane(H, zw)) {
      pair(InnerTag{});
    } else if (col && zp_open_plane(g, H, zw)) {
      pair(FaceTag{});
    } else {
      const Lattice<C, 0> LA = lattice_of<C, 0>(p.A, p), LB = lattice_of<C, 0>(p.B, p);
      ZPairNode a;
      a.set(g, x, y, zw);
      ts_stream_node<false, C, 0, ZPairNode>(p, a, LA, LB);
      ZPairNode b;
      b.set(g, x, y, zw + H);
      ts_stream_node<false, C, 0, ZPairNode>(p, b, LA, LB);
    }
  }
}

// One-step push (PUSH) or pull in z pairs.
template <class C, bool PUSH, bool FORCE, bool RED>
__global__ void __launch_bounds__(LBM_STEP_MAXT, (pair_four_min_blocks<C>())) k_os_zp(StepParams p) {
  chain_wait();
  using PW = PairWord<C>;
  using W = typename PW::W;
  const Grid &g = p.g;
  const int H = g.nz >> 1;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  double m = 0.0, j = 0.0;
  if (x < g.nx && y < g.ny) {
    const W *A = static_cast<const W *>(p.A);
    W *B = static_cast<W *>(p.B);
    const int64_t nw = p.npad >> 1;
    const bool col = zp_open_column(g, x, y);
    const bool inner = zp_inner_warp(g, x, y);
    for (int zw = blockIdx.z; zw < H; zw += gridDim.z) {
      auto pair = [&](auto tag) {
        constexpr bool INNER = decltype(tag)::value;
        const int w = x + (int)g.sx * y + (int)g.sxy * zw;
        W v[Q];
        if (PUSH) {
#pragma unroll
          for (int i = 0; i < Q; ++i) v[i] = A[i * nw + w];
        } else {
          ZPairCol c;
          if (!INNER) c.set(g, x, y);
          v[0] = A[w];
#pragma unroll
          for (int i = 1; i < Q; ++i) {
            bool seam;
            const W t = A[i * nw + c.template nbw<-1, INNER>(g, H, w, zw, i, seam)];
            v[i] = seam ? PW::swap(t) : t;
          }
        }
        zp_collide_pair<C, FORCE>(v, p, m, j);
        // recompute the addresses rather than hold them across the collision
        const int ws = launder(w), xs = launder(x), ys = launder(y);
        if (PUSH) {
          ZPairCol c;
          if (!INNER) c.set(g, xs, ys);
          B[ws] = v[0];
#pragma unroll
          for (int i = 1; i < Q; ++i) {
            bool seam;
            const int d = c.template nbw<1, INNER>(g, H, ws, zw, i, seam);
            B[i * nw + d] = seam ? PW::swap(v[i]) : v[i];
          }
        } else {
#pragma unroll
          for (int i = 0; i < Q; ++i) B[i * nw + ws] = v[i];
        }
      };
      if (inner && zp_inner_plane(H, zw)) {
        pair(InnerTag{});
      } else if (col && zp_open_plane(g, H, zw)) {
        pair(FaceTag{});
      } else {
        const Lattice<C, 0> LA = lattice_of<C, 0>(p.A, p), LB = lattice_of<C, 0>(p.B, p);
        for (int h = 0; h < 2; ++h) {
          ZPairNode a;
          a.set(g, x, y, zw + h * H);
          if (PUSH)
            os_push_node<false, C, 0, ZPairNode, FORCE>(p, a, LA, LB, m, j);
          else
            os_pull_node<false, C, 0, ZPairNode, FORCE>(p, a, LA, LB, m, j);
        }
      }
    }
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

// Esoteric-twist helpers on a full grid (unused for node lists).
__device__ __forceinline__ int et_pos(const DirectNode &nd, const StepParams &p, int i) { return nd.pos(p, i); }
__device__ __forceinline__ int et_pos(const IndirectNode &nd, const StepParams &, int) { return nd.s; }
__device__ __forceinline__ bool et_linked(const DirectNode &nd, const StepParams &p, int i) {
  return nd.fast || nd.nb(p, i) >= 0;
}
__device__ __forceinline__ bool et_linked(const IndirectNode &, const StepParams &, int) { return true; }

// Esoteric twist (Fig. 6): PDF f_i of node x lives in array map[i] at x for
// the rest and odd directions, and at x + c_{i-1} for even i (the neighbour
// along the odd direction i-1).  Post-collision f_i goes to array map[opp i]
// at x + s(opp i); across a solid link to array map[i] at the same slot.  The
// host then exchanges map[i] and map[opp i].
//   direct:   positions and solid tests from coordinates; beyond a wall the
//             position is a halo slot
//   indirect: word k of the packed index (k = 0..8, direction 2k+1) holds the
//             slot of x + c_{2k+1} in bits 0..30 (a ghost slot >= nfluid when
//             that cell is solid) and in bit 31 whether x + c_{2k+2} is solid.
// One node of the esoteric twist.  FAST (full grid only): the node has no
// wall or solid link, so every position is the wrapped neighbour slot and no
// store is redirected.
template <bool FAST, class C, int AOS, bool IND, bool FORCE>
__device__ __forceinline__ void et_node(const StepParams &p, NodeOf<IND> &nd, const Lattice<C, AOS> &A, double &m,
                                        double &j) {
  using T = typename C::T;
  using S = typename C::S;
  // array map[k] at slot pos: SoA through the per-array start pointers
  auto ld = [&](int k, int pos) -> T {
    if constexpr (AOS == 0) return C::raw(static_cast<const S *>(p.mapbase[k])[pos]);
    return A.ld(p.map[k], pos);
  };
  // store into array map[ka] if `first`, else map[kb] (ka, kb compile-time)
  auto st = [&](bool first, int ka, int kb, int pos, T v) {
    if constexpr (AOS == 0)
      static_cast<S *>(first ? p.mapbase[ka] : p.mapbase[kb])[pos] = C::unraw(v);
    else
      A.st(first ? p.map[ka] : p.map[kb], pos, v);
  };
  uint32_t w[10];  // packed index words (IDX addressing), kept across the collision
  if (IND) {
#pragma unroll
    for (int k = 1; k <= 9; ++k) w[k] = (uint32_t)__ldg(p.idx + (int64_t)(k - 1) * p.ipad + nd.s);
  }
  T d[Q];
  d[0] = ld(0, nd.s);
#pragma unroll
  for (int k = 1; k <= 9; ++k) {
    const int i = 2 * k - 1;
    d[i] = ld(i, nd.s);
    const int pos = IND ? (int)(w[k] & 0x7fffffffu) : et_pos(nd, p, i);
    d[i + 1] = ld(i + 1, pos);
  }
  run_collision<C, FORCE>(d, p, m, j);
  nd.launder_all();
  if (IND) {
#pragma unroll
    for (int k = 1; k <= 9; ++k) w[k] = (uint32_t)launder((int)w[k]);
  }
  st(true, 0, 0, nd.s, d[0]);
#pragma unroll
  for (int k = 1; k <= 9; ++k) {
    const int i = 2 * k - 1;
    int pos;
    bool lp, lm;
    if (IND) {
      pos = (int)(w[k] & 0x7fffffffu);
      lp = pos < p.nfluid;
      lm = (w[k] >> 31) == 0u;
    } else {
      pos = et_pos(nd, p, i);
      lp = FAST || et_linked(nd, p, i);
      lm = FAST || et_linked(nd, p, i + 1);
    }
    // odd direction i: to x + c_i; even direction i+1: to x itself
    st(lp, i + 1, i, pos, d[i]);
    st(lm, i, i + 1, nd.s, d[i + 1]);
  }
}

template <class C, int AOS, bool IND, bool FORCE, bool RED>
__global__ void LBM_ET_BOUNDS k_et(StepParams p) {
  chain_wait();
  using Node = NodeOf<IND>;
  const auto A = lattice_of<C, AOS>(p.A, p);
  double m = 0.0, j = 0.0;
  LBM_NODE_LOOP(Node, it) {
    Node nd;
    if (!nd.init_it(p, it)) continue;
    if (!IND && nd.fast)
      et_node<true, C, AOS, IND, FORCE>(p, nd, A, m, j);
    else
      et_node<false, C, AOS, IND, FORCE>(p, nd, A, m, j);
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

// Esoteric twist in z pairs (FP16 / FP32 storage, periodic box without solid cells:
// every neighbour word exists, no halo).  Array map[i] holds the pair's word
// at x for the rest and odd directions and at x + c_{i-1} for even i; the
// post-collision PDFs go back to the same words with the arrays of each
// opposite pair exchanged, as in et_node.
template <class C, bool FORCE, bool RED>
__global__ void __launch_bounds__(LBM_STEP_MAXT, (PairWord<C>::kMinBlocks)) k_et_zp(StepParams p) {
  chain_wait();
  using PW = PairWord<C>;
  using W = typename PW::W;
  const Grid &g = p.g;
  const int H = g.nz >> 1;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  double m = 0.0, j = 0.0;
  auto arr = [&](int k) { return static_cast<W *>(p.mapbase[k]); };
  if (x < g.nx && y < g.ny) {
    for (int zw = blockIdx.z; zw < H; zw += gridDim.z) {
      const int w = x + (int)g.sx * y + (int)g.sxy * zw;
      W v[Q];
      {
        ZPairCol c;
        c.set(g, x, y);
        v[0] = arr(0)[w];
#pragma unroll
        for (int k = 1; k <= 9; ++k) {
          const int i = 2 * k - 1;
          v[i] = arr(i)[w];
          bool seam;
          const W t = arr(i + 1)[c.nbw<1>(g, H, w, zw, i, seam)];
          v[i + 1] = seam ? PW::swap(t) : t;
        }
      }
      zp_collide_pair<C, FORCE>(v, p, m, j);
      const int ws = launder(w), xs = launder(x), ys = launder(y);
      ZPairCol c;
      c.set(g, xs, ys);
      arr(0)[ws] = v[0];
#pragma unroll
      for (int k = 1; k <= 9; ++k) {
        const int i = 2 * k - 1;
        bool seam;
        const int q = c.nbw<1>(g, H, ws, zw, i, seam);
        arr(i + 1)[q] = seam ? PW::swap(v[i]) : v[i];
        arr(i)[ws] = v[i + 1];
      }
    }
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

// Esoteric twist on an FP16 node list (SoA) in node pairs: nodes 2t and
// 2t + 1 share word t of every array, so the own-slot loads and stores
// (rest and odd directions in, even directions out) move one word for both
// nodes, and the packed index words of both come as one 8-byte word per
// direction; the neighbour positions are gathered and scattered per node.
// The index words are loaded again for the stores (L1 hits) instead of
// being held across the collision.  Where the two nodes send an even
// direction to different arrays (one of them has a solid link) the two
// halves are stored apart.  The per-node arithmetic is et_node's
// (bit-identical results).  80 registers (three blocks per SM), two pairs
// per thread: 512^3 sphere pack 44.0 against 42.6 GFLUP/s one node per
// thread (four blocks 42.3; the index words held in registers 41.2).
template <class C, bool FORCE, bool RED>
__global__ void __launch_bounds__(LBM_STEP_MAXT, 3) k_et_np(StepParams p) {
  chain_wait();
  using PW = PairWord<C>;
  using W = typename PW::W;
  using S = typename C::S;
  const int64_t nn = p.nnodes, nt = (nn + 1) >> 1;
  auto arr = [&](int k) { return static_cast<W *>(p.mapbase[k]); };
  auto el = [&](int k) { return static_cast<S *>(p.mapbase[k]); };
  const uint2 *I = reinterpret_cast<const uint2 *>(p.idx);
  const int64_t iw = p.ipad >> 1;
  double m = 0.0, j = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
    if (2 * t + 1 < nn) {
      const int w = (int)t;
      W v[Q];
      v[0] = arr(0)[w];
#pragma unroll
      for (int k = 1; k <= 9; ++k) {
        const int i = 2 * k - 1;
        const uint2 q = __ldg(I + (k - 1) * iw + w);
        v[i] = arr(i)[w];
        v[i + 1] = PW::pack(el(i + 1)[q.x & 0x7fffffffu], el(i + 1)[q.y & 0x7fffffffu]);
      }
      zp_collide_pair<C, FORCE>(v, p, m, j);
      const int ws = launder(w);
      arr(0)[ws] = v[0];
#pragma unroll
      for (int k = 1; k <= 9; ++k) {
        const int i = 2 * k - 1;
        const uint2 q = __ldg(I + (k - 1) * iw + ws);
        const int pa = (int)(q.x & 0x7fffffffu), pb = (int)(q.y & 0x7fffffffu);
        el(pa < p.nfluid ? i + 1 : i)[pa] = PW::lo_s(v[i]);
        el(pb < p.nfluid ? i + 1 : i)[pb] = PW::hi_s(v[i]);
        const bool la = (q.x >> 31) == 0u, lb = (q.y >> 31) == 0u;
        if (la == lb) {
          arr(la ? i : i + 1)[ws] = v[i + 1];
        } else {
          el(la ? i : i + 1)[2 * ws] = PW::lo_s(v[i + 1]);
          el(lb ? i : i + 1)[2 * ws + 1] = PW::hi_s(v[i + 1]);
        }
      }
    } else {
      const Lattice<C, 0> L = lattice_of<C, 0>(p.A, p);
      IndirectNode nd;
      nd.init(p, 2 * t);
      et_node<false, C, 0, true, FORCE>(p, nd, L, m, j);
    }
  }
  if (RED) block_reduce_store(m, j, p.partials);
}

// ---------------------------------------------------------------------------
// Launchers.

template <class C, int AOS, bool IND, bool FORCE, bool RED>
struct LaunchTS {
  // phase 0 collide, 1 stream; 2 collide, 3 stream in z pairs (FP16 / FP32, SoA full grid)
  static void run(const StepParams &p, int phase, const LaunchShape &L) {
    if (phase >= 2) {
      if constexpr (kPairable<C> && AOS == 0 && !IND) {
        if (phase == 2)
          launch_chained(k_ts_collide_zp<C, FORCE, RED>, L.grid, L.block, 0, L.stream, p);
        else
          launch_chained(k_ts_stream_zp<C>, L.grid, L.block, 0, L.stream, p);
      }
      return;
    }
    if (phase == 0)
      launch_chained(k_ts_collide<C, AOS, NodeOf<IND>, FORCE, RED>, L.grid, L.block, 0, L.stream, p);
    else
      launch_chained(k_ts_stream<C, AOS, NodeOf<IND>>, L.grid, L.block, 0, L.stream, p);
  }
};
// sub: bit 0 = push (else pull), bit 1 = streaming stores (SoA only), bit 2
// = z pairs (FP16 / FP32 storage, SoA full grid, no streaming stores)
template <class C, int AOS, bool IND, bool FORCE, bool RED>
struct LaunchOS {
  template <bool CS>
  static void go(const StepParams &p, bool push, const LaunchShape &L) {
    if (push)
      launch_chained(k_os_push<C, AOS, NodeOf<IND>, FORCE, RED, CS>, L.grid, L.block, 0, L.stream, p);
    else
      launch_chained(k_os_pull<C, AOS, NodeOf<IND>, FORCE, RED, CS>, L.grid, L.block, 0, L.stream, p);
  }
  static void run(const StepParams &p, int sub, const LaunchShape &L) {
    if (sub & 4) {
      if constexpr (kPairable<C> && AOS == 0 && !IND) {
        if (sub & 1)
          launch_chained(k_os_zp<C, true, FORCE, RED>, L.grid, L.block, 0, L.stream, p);
        else
          launch_chained(k_os_zp<C, false, FORCE, RED>, L.grid, L.block, 0, L.stream, p);
      }
      return;
    }
    if constexpr (AOS == 0) {
      if (sub & 2) {
        go<true>(p, sub & 1, L);
        return;
      }
    }
    go<false>(p, sub & 1, L);
  }
};
// sub: 0 even, 1 odd (one node per thread); 4 even, 5 odd (z pairs, FP16 /
// FP32 storage, SoA full grid); 6 even, 7 odd (node pairs, FP16 storage,
// SoA node list with folded IDX)
template <class C, int AOS, bool IND, bool FORCE, bool RED>
struct LaunchAA {
  static void run(const StepParams &p, int sub, const LaunchShape &L) {
    if (sub >= 4) {
      if constexpr (std::is_same<C, CodecF16S>::value && AOS == 0 && IND) {
        if (sub == 7)
          launch_chained(k_aa_odd_np<C, FORCE, RED>, L.grid, L.block, 0, L.stream, p);
        else if (sub == 6)
          launch_chained(k_aa_even_np<C, FORCE, RED>, L.grid, L.block, 0, L.stream, p);
      }
      if constexpr (kPairable<C> && AOS == 0 && !IND) {
        if (sub == 5)
          launch_chained(k_aa_odd_zp<C, FORCE, RED>, L.grid, L.block, 0, L.stream, p);
        else
          launch_chained(k_aa_even_zp<C, FORCE, RED>, L.grid, L.block, 0, L.stream, p);
      }
      return;
    }
    if (sub)
      launch_chained(k_aa_odd<C, AOS, NodeOf<IND>, FORCE, RED>, L.grid, L.block, 0, L.stream, p);
    else
      launch_chained(k_aa_even<C, AOS, NodeOf<IND>, FORCE, RED>, L.grid, L.block, 0, L.stream, p);
  }
};
// sub: 0 one node per thread, 1 z pairs (FP16 / FP32 storage, SoA, periodic
// full grid), 2 node pairs (FP16 storage, SoA node list)
template <class C, int AOS, bool IND, bool FORCE, bool RED>
struct LaunchET {
  static void run(const StepParams &p, int sub, const LaunchShape &L) {
    if (sub == 1) {
      if constexpr (kPairable<C> && AOS == 0 && !IND)
        launch_chained(k_et_zp<C, FORCE, RED>, L.grid, L.block, 0, L.stream, p);
      return;
    }
    if (sub == 2) {
      if constexpr (std::is_same<C, CodecF16S>::value && AOS == 0 && IND)
        launch_chained(k_et_np<C, FORCE, RED>, L.grid, L.block, 0, L.stream, p);
      return;
    }
    launch_chained(k_et<C, AOS, IND, FORCE, RED>, L.grid, L.block, 0, L.stream, p);
  }
};

template <class C>
void launch_step_kernel_t(int variant, int sub, const StepParams &p, const KernelKey &k, const LaunchShape &L) {
  switch (variant) {
    case VAR_TS:
      dispatch_layout<LaunchTS, C>(k.aos, k.ind, k.force, k.red, p, sub, L);
      break;
    case VAR_OS_PUSH:
      dispatch_layout<LaunchOS, C>(k.aos, k.ind, k.force, k.red, p, 1 | (sub & 6), L);
      break;
    case VAR_OS_PULL:
      dispatch_layout<LaunchOS, C>(k.aos, k.ind, k.force, k.red, p, sub & 6, L);
      break;
    case VAR_AA:
      dispatch_layout<LaunchAA, C>(k.aos, k.ind, k.force, k.red, p, sub, L);
      break;
    case VAR_ET:
      dispatch_layout<LaunchET, C>(k.aos, k.ind, k.force, k.red, p, sub, L);
      break;
    default:
      break;
  }
}

}  // namespace lbmk
