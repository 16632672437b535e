// Host side of the swap scheme (Sec. 5): pass bookkeeping for the blocked
// full-grid swap (kernels in lbm_swap.cuh), the node-list link exchange, and
// the bounded-wait self-test.
#include <map>
#include <utility>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_swap.cuh"

namespace lbmk {

// Per-precision instantiations live in lbm_swap_<precision>.cu.
extern template void swap_pass_t<CodecF64>(const StepParams &, const SwapPass &, const KernelKey &, size_t,
                                           cudaStream_t);
extern template void swap_pass_t<CodecF32>(const StepParams &, const SwapPass &, const KernelKey &, size_t,
                                           cudaStream_t);
extern template void swap_pass_t<CodecF16S>(const StepParams &, const SwapPass &, const KernelKey &, size_t,
                                            cudaStream_t);
extern template void swap_pass_pair_t<CodecPair<CodecF32>>(const StepParams &, const SwapPass &, const KernelKey &,
                                                           size_t, cudaStream_t);
extern template void swap_pass_pair_t<CodecPair<CodecF16S>>(const StepParams &, const SwapPass &, const KernelKey &,
                                                            size_t, cudaStream_t);
extern template int swap_pass_tma_t<CodecF64>(const StepParams &, const SwapPass &, const KernelKey &,
                                              const CUtensorMap *, int, int, cudaStream_t);
extern template int swap_pass_tma_t<CodecF32>(const StepParams &, const SwapPass &, const KernelKey &,
                                              const CUtensorMap *, int, int, cudaStream_t);
extern template int swap_pass_tma_t<CodecF16S>(const StepParams &, const SwapPass &, const KernelKey &,
                                               const CUtensorMap *, int, int, cudaStream_t);

// Self-test of the bounded wait: one thread waits on a barrier that expects
// one arrival which never comes.
__device__ int g_wait_selftest;
__global__ void k_wait_selftest(uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  g_wait_selftest = mbar_wait(&bar, 0, limit_ns) ? 1 : 2;
}

// tiles are at most kSwapTX x kSwapTY x kSwapTZ = 256 cells (one thread each)
// ---------------------------------------------------------------------------
// Link-class tables of the tiles (see SwapTiles).  A tile's colour is fixed
// by its per-axis colours; a neighbour at offset o is "earlier" when its
// colour index is lower (its pass ran first) and "self" when the tile wraps
// onto itself across a periodic face.
static int axis_colour_host(int t, int nt, int periodic) {
  if (nt == 1) return 0;
  if (periodic && (nt & 1)) return t == nt - 1 ? 2 : (t & 1);
  return t & 1;
}

void build_swap_tables(const SwapTiles &t, const int per[3], std::vector<uint16_t> &tcls,
                       std::vector<uint32_t> &tables) {
  auto ncol = [](int nt, int periodic) { return nt == 1 ? 1 : ((periodic && (nt & 1)) ? 3 : 2); };
  const int nt[3] = {t.ntx, t.nty, t.ntz};
  const int cx = ncol(t.ntx, per[0]), cy = ncol(t.nty, per[1]);
  auto colour = [&](const int a[3]) {
    return axis_colour_host(a[0], nt[0], per[0]) +
           cx * (axis_colour_host(a[1], nt[1], per[1]) + cy * axis_colour_host(a[2], nt[2], per[2]));
  };
  std::map<std::pair<uint32_t, uint32_t>, int> seen;
  tcls.assign((size_t)nt[0] * nt[1] * nt[2], 0);
  tables.clear();
  for (int tz = 0; tz < nt[2]; ++tz)
    for (int ty = 0; ty < nt[1]; ++ty)
      for (int tx = 0; tx < nt[0]; ++tx) {
        const int tile[3] = {tx, ty, tz};
        const int own = colour(tile);
        uint32_t em = 0, sm = 0;
        for (int l = 0; l < 27; ++l) {
          const int o[3] = {l % 3 - 1, (l / 3) % 3 - 1, l / 9 - 1};
          int nb[3];
          bool exists = true, self = true;
          for (int a = 0; a < 3; ++a) {
            nb[a] = tile[a] + o[a];
            if (nb[a] < 0 || nb[a] >= nt[a]) {
              if (!per[a]) exists = false;
              nb[a] = (nb[a] + nt[a]) % nt[a];
            }
            self = self && nb[a] == tile[a];
          }
          if (!exists) continue;
          if (self)
            sm |= 1u << l;
          else if (colour(nb) < own)
            em |= 1u << l;
        }
        auto key = std::make_pair(em, sm);
        auto it = seen.find(key);
        int index;
        if (it == seen.end()) {
          index = (int)seen.size();
          seen[key] = index;
          tables.push_back(em);
          tables.push_back(sm);
          // cell classes of a full tile: x low/inner/high,
          // y low/inner/high, z low/high
          for (int c = 0; c < 18; ++c) {
            const int xc = c % 3, yc = (c / 3) % 3, zc = c / 9;
            uint32_t om = 0, rm = 0, smk = 0;
            for (int i = 1; i < Q; ++i) {
              const int ci[3] = {CX(i), CY(i), CZ(i)};
              const bool ox = ci[0] > 0 ? xc == 0 : (ci[0] < 0 ? xc == 2 : false);
              const bool oy = ci[1] > 0 ? yc == 0 : (ci[1] < 0 ? yc == 2 : false);
              const bool oz = ci[2] > 0 ? zc == 0 : (ci[2] < 0 ? zc == 1 : false);
              if (!(ox || oy || oz)) continue;
              om |= 1u << i;
              const int bit = tile_bit(ox ? -ci[0] : 0, oy ? -ci[1] : 0, oz ? -ci[2] : 0);
              if (sm & (1u << bit))
                smk |= 1u << i;
              else if (em & (1u << bit))
                rm |= 1u << i;
            }
            tables.push_back(om);
            tables.push_back(rm);
            tables.push_back(smk);
          }
        } else {
          index = it->second;
        }
        tcls[tx + (size_t)nt[0] * (ty + (size_t)nt[1] * tz)] = (uint16_t)index;
      }
}

// S (19 post-collision PDFs per cell, compute type) and the remote-prefetch
// buffer (18 words per cell, the stored element or its 4-byte word)
size_t swap_smem_bytes(const SwapTiles &t, int precision) {
  const size_t cells = (size_t)t.tx * t.ty * t.tz;
  if (t.pairs) {  // a float2 per PDF; remote words of 8 (FP32) or 4 (FP16) bytes
    const size_t word = precision == 2 ? 4 : 8;
    return ((size_t)Q * cells * 8 + 15) / 16 * 16 + (size_t)(Q - 1) * cells * word;
  }
  const size_t comp = precision == 0 ? 8 : 4, word = precision == 0 ? 8 : 4;
  return ((size_t)Q * cells * comp + 15) / 16 * 16 + (size_t)(Q - 1) * cells * word;
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

static SwapPass pass_of(const StepParams &p, const SwapTiles &t) {
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
  sp.stride = 2;
  sp.tcls = t.tcls;
  sp.tables = t.tables;
  return sp;
}

void launch_swap_pass(const StepParams &p, const SwapTiles &t, const KernelKey &k, cudaStream_t s) {
  const SwapPass sp = pass_of(p, t);
  if (sp.count[0] * sp.count[1] * sp.count[2] == 0) return;
  const size_t smem = swap_smem_bytes(t, k.precision);
  if (t.pairs) {
    if (k.precision == 1)
      swap_pass_pair_t<CodecPair<CodecF32>>(p, sp, k, smem, s);
    else if (k.precision == 2)
      swap_pass_pair_t<CodecPair<CodecF16S>>(p, sp, k, smem, s);
    return;
  }
  if (k.precision == 0)
    swap_pass_t<CodecF64>(p, sp, k, smem, s);
  else if (k.precision == 1)
    swap_pass_t<CodecF32>(p, sp, k, smem, s);
  else
    swap_pass_t<CodecF16S>(p, sp, k, smem, s);
}

int launch_swap_pass_tma(const StepParams &p, const SwapTiles &t, const KernelKey &k, const CUtensorMap *map,
                         int nsm, cudaStream_t s) {
  const SwapPass sp = pass_of(p, t);
  const int ntiles = sp.count[0] * sp.count[1] * sp.count[2];
  if (ntiles == 0) return 0;
  if (k.precision == 0) return swap_pass_tma_t<CodecF64>(p, sp, k, map, nsm, ntiles, s);
  if (k.precision == 1) return swap_pass_tma_t<CodecF32>(p, sp, k, map, nsm, ntiles, s);
  return swap_pass_tma_t<CodecF16S>(p, sp, k, map, nsm, ntiles, s);
}

size_t swap_tma_smem_bytes(int tile_cells, size_t stored, size_t computed) {
  const size_t stage = ((size_t)Q * tile_cells * stored + 127) / 128 * 128;
  const size_t sx = stored == computed ? 0 : ((size_t)Q * tile_cells * computed + 15) / 16 * 16;
  const size_t word = stored < 4 ? 4 : stored;
  return 128 + 2 * stage + sx + (size_t)(Q - 1) * tile_cells * word;
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

extern "C" lbm_status lbm_selftest_bounded_wait(int64_t limit_ns, void *stream) {
  if (limit_ns < 1000 || limit_ns > 1000000000) return LBM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int zero = 0;
  if (cudaMemcpyToSymbolAsync(lbmk::g_wait_selftest, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return LBM_ERR_CUDA;
  lbmk::k_wait_selftest<<<1, 1, 0, s>>>((uint64_t)limit_ns);
  int r = 0;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyFromSymbolAsync(&r, lbmk::g_wait_selftest, sizeof r, 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return LBM_ERR_CUDA;
  return r == 2 ? LBM_ERR_TIMEOUT : (r == 1 ? LBM_OK : LBM_ERR_CUDA);
}
