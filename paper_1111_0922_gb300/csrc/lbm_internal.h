// Host-side internals shared by the library's translation units: kernel
// selection keys, launch shapes, and the launchers each .cu file exports.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <vector>

#include "lbm_core.cuh"

namespace lbmk {

enum { VAR_TS = 0, VAR_OS_PUSH = 1, VAR_OS_PULL = 2, VAR_CG = 3, VAR_SWAP = 4, VAR_AA = 5, VAR_ET = 6 };

// How the natural state f_i(x) maps to storage.
enum {
  MAP_NATURAL = 0,  // slot i of x (TS, OS push, swap, AA at even step count)
  MAP_PULL = 1,     // post-collision storage: f_i(x) = A_i(x - c_i), or A_opp(i)(x) across a solid link
  MAP_ET = 2        // esoteric twist: array map[i] at x + s(i)
};

struct KernelKey {
  int precision;  // 0 F64, 1 F32, 2 F16S
  int aos;        // 0 SoA, 1 AoS
  bool ind;       // IDX addressing
  bool force;     // nonzero body force
  bool red;       // fused (mass, flux) reduction
};

struct LaunchShape {
  dim3 grid, block;
  cudaStream_t stream;
};

// lbm_steps_*.cu: TS (sub 0 collide, 1 stream), OS push/pull, AA (sub = odd), ET
template <class C>
void launch_step_kernel_t(int variant, int sub, const StepParams &p, const KernelKey &k, const LaunchShape &L);
extern template void launch_step_kernel_t<CodecF64>(int, int, const StepParams &, const KernelKey &, const LaunchShape &);
extern template void launch_step_kernel_t<CodecF32>(int, int, const StepParams &, const KernelKey &, const LaunchShape &);
extern template void launch_step_kernel_t<CodecF16S>(int, int, const StepParams &, const KernelKey &, const LaunchShape &);
inline void launch_step_kernel(int variant, int sub, const StepParams &p, const KernelKey &k, const LaunchShape &L) {
  if (k.precision == 0)
    launch_step_kernel_t<CodecF64>(variant, sub, p, k, L);
  else if (k.precision == 1)
    launch_step_kernel_t<CodecF32>(variant, sub, p, k, L);
  else
    launch_step_kernel_t<CodecF16S>(variant, sub, p, k, L);
}

// lbm_cg.cu: one slab of the compressed grid, and its periodic ghost planes
void launch_cg_slab(const StepParams &p, const KernelKey &k, const LaunchShape &L);
inline void launch_step_kernel_cg(const StepParams &p, const KernelKey &k, const LaunchShape &L) {
  launch_cg_slab(p, k, L);
}
void launch_cg_ghost(const StepParams &p, int precision, int aos, int zo, cudaStream_t s);
// node lists: unwrapped index + counters {D, nodes in plane 0, nodes in plane nz-1}
void launch_cg_ind_prep(const int32_t *idx, int64_t ipad, const int32_t *cells, int64_t N, int nx, int ny, int nz,
                        int32_t *cidx, int *counters, cudaStream_t s);
void launch_cg_ind_ghost(void *A, int64_t npad, int precision, int aos, int64_t N, int64_t nfirst, int64_t nlast,
                         cudaStream_t s);
void launch_cg_ind_slab(const StepParams &p, const KernelKey &k, const LaunchShape &L);

// lbm_swap.cu: one colour pass of the blocked swap.  Full tile box (cells):
// 64 along x (two warps per row), 2 along y, 2 along z; smaller boxes use
// their own extent.  Measured against 32 x 4 x 2 (FP32, 256^3): the wider
// rows give longer contiguous runs per array in each colour pass, and more
// of the links between tiles cross y and z faces, where a warp exchanges
// whole rows.  The cell classes of the link tables assume kSwapTZ == 2.
constexpr int kSwapTX = 64, kSwapTY = 2, kSwapTZ = 2;
struct SwapTiles {
  int tx, ty, tz;       // tile extent in cells
  int ntx, nty, ntz;    // tiles per axis
  int colour;           // pass being run
  int ncolours;
  // link-class tables (built once per geometry): per tile (x fastest) the
  // index of its table; a table is 2 + 3 x 18 words: the earlier-colour and
  // self neighbour masks of the 27 tile offsets, then for each of the 18
  // cell classes of a full tile the outside / remote / self link masks.
  const uint16_t *tcls = nullptr;
  const uint32_t *tables = nullptr;
  int pairs = 0;  // tiles of the grid of cell-pair words (Grid::zpair)
};
constexpr int kSwapTableWords = 2 + 3 * 18;
void build_swap_tables(const SwapTiles &t, const int per[3], std::vector<uint16_t> &tcls,
                       std::vector<uint32_t> &tables);
void launch_swap_pass(const StepParams &p, const SwapTiles &t, const KernelKey &k, cudaStream_t s);
// the same pass with tensor-copy staging (full grid, SoA, strides multiple of
// 16 bytes); `map` describes the lattice as a 4D tensor (x, y, z, array) with
// the tile as its box.  Launches persistent blocks (as many as are resident
// at once on nsm SMs, at most one per tile) and returns how many.
int launch_swap_pass_tma(const StepParams &p, const SwapTiles &t, const KernelKey &k, const CUtensorMap *map,
                         int nsm, cudaStream_t s);
size_t swap_tma_smem_bytes(int tile_cells, size_t stored, size_t computed);
size_t swap_smem_bytes(const SwapTiles &t, int precision);
int swap_colours(const SwapTiles &t, int px, int py, int pz);
// node lists: link exchanges after a collide-into-reversed-slots pass
void launch_swap_links(const StepParams &p, int precision, int aos, cudaStream_t s);
int swap_blocks(const SwapTiles &t, int px, int py, int pz, int colour);

// lbm_setup.cu
void launch_sphere_mask(uint8_t *solid, int nx, int ny, int nz, const int *periodic, int64_t nsph,
                        const int64_t *centres, int64_t radius, int64_t unit, cudaStream_t s);
// exclusive prefix count of nonzero bytes; node_of[c] = number or -1; cells[k] = c
int64_t build_node_list(const uint8_t *solid, int64_t ncell, int32_t *node_of, int32_t *cells,
                        int32_t *scratch, int64_t scratch_elems, cudaStream_t s);
int64_t scan_scratch_elems(int64_t n);
void launch_build_idx(const int32_t *cells, const int32_t *node_of, int64_t N, int nx, int ny, int nz,
                      const int *periodic, int32_t *idx, int64_t ipad, cudaStream_t s);
// AA pattern, SoA: solid links of IDX replaced by their bounce-back slots
void launch_fold_idx(int32_t *idx, int64_t ipad, int64_t N, int64_t npad, cudaStream_t s);
// esoteric twist packed index; ghost_map is (nx+2)(ny+2)(nz+2) int32 scratch
int64_t build_et_index(const int32_t *cells, const int32_t *node_of, int64_t N, int nx, int ny, int nz,
                       const int *periodic, int32_t *ghost_map, int32_t *etidx, int64_t ipad,
                       int32_t *scratch, int64_t scratch_elems, cudaStream_t s);

// state <-> natural FP64 arrays, moments and reductions
struct StateDesc {
  StepParams p;       // A (state), npad, grid/idx, map, scale
  KernelKey k;        // precision, aos, ind
  int mapkind;        // MAP_*
  const int32_t *cells;  // indirect: node -> cell (for rho/u outputs this is not needed)
};
// f_nat: 19 x n FP64 (n = nodes), or computed as f_eq(rho, u) when f_nat is null
void launch_put_state(const StateDesc &d, const double *f_nat, const double *rho, const double *u,
                      cudaStream_t s);
// write natural FP64 (solid cells of a direct grid get 0)
void launch_get_state(const StateDesc &d, double *f_nat, cudaStream_t s);
void launch_macroscopics(const StateDesc &d, double *rho, double *u, cudaStream_t s);
// per-block partials then one fixed-order final sum into out[2]
int reduce_blocks_for(int64_t nnodes);
void launch_flux_partials(const StateDesc &d, double *partials, int nblocks, cudaStream_t s);
void launch_final_sum(const double *partials, int nblocks, double *out, cudaStream_t s);

}  // namespace lbmk
