/*
 * liblbm — GB300 (sm_103a) D3Q19 lattice Boltzmann time step, C ABI.
 *
 * One time step is the BGK collision, or the two-relaxation-time (TRT)
 * collision of the paper's solver (Sec. 10), with a constant body force
 * (Guo's forcing term) at every fluid node, followed by the propagation of the
 * post-collision PDFs to the neighbours, with half-way bounce-back at solid
 * nodes and at non-periodic box faces.  The propagation is done by one of the
 * schemes compared by Wittmann, Zeiser, Hager and Wellein, "Comparison of
 * different Propagation Steps for the Lattice Boltzmann Method":
 *
 *   LBM_TS       two-step: collide kernel + separate stream kernel  (Sec. 2, Tab. 1)
 *   LBM_OS_PUSH  one-step push, two lattices                         (Sec. 3, Fig. 1a,b, Tab. 2)
 *   LBM_OS_PULL  one-step pull, two lattices                         (Sec. 3, Fig. 1c,d)
 *   LBM_CG       compressed grid, one lattice shifted between steps  (Sec. 4, Fig. 2, Tab. 3)
 *   LBM_SWAP     swap, one lattice, link exchanges                   (Sec. 5, Fig. 3, Tab. 4)
 *   LBM_AA       AA pattern, one lattice, even/odd kernels           (Sec. 6, Fig. 5, Tab. 5)
 *   LBM_ET       esoteric twist, one lattice, array pointer swap     (Sec. 7, Fig. 6, Tab. 6)
 *
 * on a full grid (LBM_DIRECT: neighbours by index arithmetic) or on a list of
 * fluid nodes with an int32 adjacency array IDX (LBM_INDIRECT), with the PDFs
 * in structure-of-arrays (LBM_SOA, one array per direction) or
 * array-of-structures (LBM_AOS) layout (Sec. 1).
 *
 * Precision: LBM_F64 stores f_i - w_i in FP64 and computes in FP64;
 * LBM_F32 stores f_i - w_i in FP32 and computes in FP32; LBM_F16S stores
 * round((f_i - w_i) * S) in FP16 with a power-of-two scale S and computes in
 * FP32.  Mass and flux sums are always accumulated in FP64.
 *
 * Conventions
 *   velocities  0:(0,0,0) 1:(+1,0,0) 2:(-1,0,0) 3:(0,+1,0) 4:(0,-1,0)
 *               5:(0,0,+1) 6:(0,0,-1) 7:(+1,+1,0) 8:(-1,-1,0) 9:(+1,-1,0)
 *               10:(-1,+1,0) 11:(+1,0,+1) 12:(-1,0,-1) 13:(+1,0,-1)
 *               14:(-1,0,+1) 15:(0,+1,+1) 16:(0,-1,-1) 17:(0,+1,-1)
 *               18:(0,-1,+1); weights 1/3, 1/18 (1-6), 1/36 (7-18).
 *   cells       x fastest: cell = x + nx * (y + ny * z).
 *   nodes       fluid cells numbered in that order (lexicographic).
 *   natural     the pre-collision state f_i(x) after a whole number of
 *               steps, as a host or device array f[i * n + k] (FP64), k the
 *               cell (direct) or node (indirect).
 *   velocity    u = (sum_i c_i f_i + rho g / 2) / rho.
 *
 * Ownership: the library owns every device buffer it allocates; it allocates
 * through cfg->dev_alloc / cfg->dev_free when given (e.g. PyTorch's caching
 * allocator), else cudaMalloc / cudaFree, and only inside lbm_create,
 * lbm_set_geometry* and lbm_destroy.  Host pointers are borrowed for the call.
 * Device pointers passed with on_device = 1 must be on the handle's device.
 *
 * Errors: every call returns a status and never throws.  lbm_last_error
 * gives a one-line reason.  Kernels are enqueued on cfg->stream and run
 * asynchronously; launch errors are reported by the call, device-side errors
 * (bounds flags of a checked build) by the next synchronising call.
 * A handle must not be used from two threads at once.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LBM_OK = 0,
  LBM_ERR_INVALID_ARG = 1,  /* bad pointer, size, enum or configuration */
  LBM_ERR_OOM = 2,          /* a device allocation failed */
  LBM_ERR_CUDA = 3,         /* a CUDA call or kernel launch failed */
  LBM_ERR_STATE = 4,        /* call not valid in the handle's current state */
  LBM_ERR_BOUNDS = 5,       /* a kernel's bounds check tripped */
  LBM_ERR_TIMEOUT = 6,      /* a bounded device wait gave up */
  LBM_ERR_NOT_CONVERGED = 7,/* a solve hit its step cap */
  LBM_ERR_UNSUPPORTED = 8   /* valid request the library does not implement */
} lbm_status;

enum { LBM_TS = 0, LBM_OS_PUSH = 1, LBM_OS_PULL = 2, LBM_CG = 3, LBM_SWAP = 4, LBM_AA = 5, LBM_ET = 6 };
enum { LBM_DIRECT = 0, LBM_INDIRECT = 1 };
enum { LBM_SOA = 0, LBM_AOS = 1 };
enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16S = 2 };

typedef void *(*lbm_alloc_fn)(size_t bytes, void *ctx);
typedef void (*lbm_free_fn)(void *ptr, size_t bytes, void *ctx);

typedef struct lbm_config {
  int32_t nx, ny, nz;        /* bounding box, each >= 1; periodic extents >= 2 */
  int32_t periodic[3];       /* 1 = periodic axis, 0 = bounce-back walls beyond both faces */
  int32_t variant;           /* LBM_TS .. LBM_ET */
  int32_t addressing;        /* LBM_DIRECT or LBM_INDIRECT */
  int32_t layout;            /* LBM_SOA or LBM_AOS */
  int32_t precision;         /* LBM_F64, LBM_F32, LBM_F16S */
  double omega;              /* BGK relaxation rate, 0 < omega < 2 (0 = identity collision) */
  double force[3];           /* body acceleration g (Guo forcing) */
  double f16_scale;          /* LBM_F16S: scale S (power of two); 0 = choose from force */
  double trt_magic;          /* 0 = BGK; > 0 = two-relaxation-time collision with magic parameter
                                Lam = (1/omega - 1/2)(1/omega_minus - 1/2), e.g. 3/16 (walls exactly
                                half-way for Poiseuille flow) */
  int32_t block_size;        /* threads per block of the step kernels (multiple of 32, <= 256); 0 = 128
                                (256 for LBM_AA on a node list) */
  int32_t nodes_per_thread;  /* nodes each thread updates (1..16); 0 = default (full grid: 2 planes,
                                4 pair planes with FP16 cell pairs; node list: 1 node, 2 node
                                pairs with FP16 node pairs); with cell or node pairs it counts
                                pairs */
  int32_t cg_shift;          /* LBM_CG: full grid: shift k >= 2 planes (slabs of k-1 planes, k extra
                                planes of storage; 0 = slabs of about 2^22 cells);
                                node list: slab size B >= 1 nodes (0 = 2^21) */
  int32_t store_hint;        /* LBM_OS_PUSH / LBM_OS_PULL, SoA: 1 = write the second lattice with
                                cache-streaming (evict-first) stores, the GPU counterpart of the
                                non-temporal stores of OS-NT (Sec. 3); 0 = ordinary stores */
  int32_t swap_schedule;     /* LBM_SWAP, full grid: 1 = coloured passes: tiles of one colour per
                                pass, links to tiles of earlier colours completed in place;
                                2 = the same with each tile staged by one tensor copy (TMA) in
                                persistent blocks (SoA, row pitch a multiple of 16 bytes);
                                0 = default: 1 (measured fastest on GB300) */
  int32_t pair_z;            /* Cell pairs, LBM_F16S or LBM_F32 storage, SoA, full grid without
                                solid cells: LBM_AA, LBM_TS, LBM_OS_PUSH / PULL
                                (store_hint 0) and LBM_ET (periodic box) keep cells z and z + nz/2
                                (even nz) in one word per array (4 bytes FP16, 8 bytes FP32), and
                                one thread updates both; LBM_CG pairs cells y and y + ny/2 instead
                                (even ny); LBM_SWAP (swap_schedule 0 or 1) pairs z when z is
                                periodic and nz is a multiple of 4 (at least 8).  On a node list
                                (LBM_INDIRECT, SoA, LBM_F16S) LBM_AA and LBM_ET pair consecutive
                                nodes 2t and 2t + 1 instead (one thread each; the storage order
                                is unchanged).
                                0 = default (on where allowed), 1 = on where allowed, 2 = off (one
                                node per thread).  The stored layout is internal: lbm_get_pdfs and
                                friends use natural order. */
  void *stream;              /* cudaStream_t the library enqueues on; NULL = default stream */
  lbm_alloc_fn dev_alloc;    /* optional device allocator */
  lbm_free_fn dev_free;      /* required when dev_alloc is given */
  void *alloc_ctx;           /* passed to dev_alloc / dev_free */
} lbm_config;

typedef struct lbm_info {
  int64_t cells;             /* nx * ny * nz */
  int64_t nodes;             /* fluid nodes (direct: cells; the solid ones are skipped) */
  int64_t storage_nodes;     /* slots per PDF array incl. ghosts, halos, shifts, padding */
  int64_t state_bytes;       /* device bytes of PDF storage */
  int64_t index_bytes;       /* device bytes of IDX and other per-node index data */
  int64_t steps;             /* time steps done since lbm_init / lbm_set_pdfs */
  int32_t natural;           /* 1 if the state can be read out (AA: even step count) */
  int32_t kernels_per_step;  /* launches one lbm_step(h, 1) makes */
  double f16_scale;          /* scale in use (LBM_F16S) */
  int32_t reduce_blocks;     /* blocks of the fused reduction */
  int32_t tile_staged;       /* 1 if the swap passes stage tiles with tensor copies */
  int32_t pair_z;            /* 1 if cells are stored in pairs (see lbm_config.pair_z) */
} lbm_info;

typedef struct lbm lbm_t;

/* Fill *cfg with defaults: 32^3 periodic box, LBM_AA, direct, SoA, FP32,
 * omega 1, no force, default launch shape, default stream, cudaMalloc.
 * (Configuration only; the D3Q19 lattice itself is Sec. 1.) */
lbm_status lbm_config_default(lbm_config *cfg);

/* Validate cfg and create a handle on the current CUDA device: one lattice
 * of PDF arrays, or two for the two-lattice schemes (LBM_TS, LBM_OS_*,
 * Sec. 2-3; the others keep one, Sec. 4-7).  No geometry yet: call
 * lbm_set_geometry or lbm_set_geometry_spheres next.  Errors:
 * LBM_ERR_INVALID_ARG for an invalid configuration, LBM_ERR_UNSUPPORTED for
 * a valid combination the library does not build, LBM_ERR_CUDA. */
lbm_status lbm_create(const lbm_config *cfg, lbm_t **out);

/* Free every device buffer (waits for the handle's stream).  NULL is OK.
 * (Resource release; no counterpart in the paper.) */
lbm_status lbm_destroy(lbm_t *h);

/* One-line description of the last failure on h (or a global one if h is
 * NULL), and the name of a status.  (Diagnostics; no counterpart.) */
const char *lbm_last_error(const lbm_t *h);
const char *lbm_status_string(lbm_status s);

/* Geometry (Sec. 1: a full grid or the sparse representation of the fluid
 * nodes with an adjacency list; the packed bed of Fig. 7, Sec. 10).
 * solid_mask_host: nx*ny*nz bytes, x fastest, nonzero = solid, or NULL for
 * an all-fluid box; borrowed for the call.  Builds on the GPU the fluid-node
 * list (lexicographic) and, for LBM_INDIRECT, IDX[18][N] (IDX[i-1][k] = node
 * reached from node k along c_i, -1 for a solid or wall link) plus the
 * variant's own index data; allocates the PDF storage.  Resets the state to
 * rest (f = w).  Synchronises.  LBM_ERR_OOM when the storage does not fit. */
lbm_status lbm_set_geometry(lbm_t *h, const uint8_t *solid_mask_host);

/* Same, with the solid mask generated on the GPU from overlapping spheres
 * (the packed bed of spheres of Sec. 10, Fig. 7): a cell is solid iff the
 * minimum-image distance (periodic axes) between its centre and some sphere
 * centre is <= radius.  centres_host: nsph x 3 int64 positions and the
 * radius in units of 1/unit cells (exact integer test). */
lbm_status lbm_set_geometry_spheres(lbm_t *h, int64_t nsph, const int64_t *centres_host,
                                    int64_t radius, int64_t unit);

/* Read back geometry (Sec. 1: the node list and its adjacency array IDX):
 * the solid mask (nx*ny*nz bytes), the node list (node -> cell, N int32)
 * and IDX (18*N int32, direction-major).  Host buffers the caller owns.
 * lbm_get_idx is valid for LBM_INDIRECT only (else LBM_ERR_STATE).
 * Synchronise. */
lbm_status lbm_get_mask(lbm_t *h, uint8_t *mask_host);
lbm_status lbm_get_nodes(lbm_t *h, int32_t *cells_host);
lbm_status lbm_get_idx(lbm_t *h, int32_t *idx_host);
lbm_status lbm_get_info(const lbm_t *h, lbm_info *info);

/* Initial state f_i = f_eq(rho, u) per node (the equilibrium of the
 * collision, Sec. 1; direct: per cell, solid cells ignored).  rho: n doubles
 * or NULL (= 1); u: 3n doubles (x,y,z per node) or NULL (= 0).  on_device =
 * 1: the pointers are device memory.  Each scheme stores it in its own form:
 * pull-type schemes (Sec. 3-4) the pre-image under streaming, the esoteric
 * twist its shifted arrays (Sec. 7).  Step count 0. */
lbm_status lbm_init(lbm_t *h, const double *rho, const double *u, int on_device);

/* Set / get the natural state f[i * n + k] (FP64, n = nodes or cells),
 * mapped to and from each scheme's storage (Sec. 2-7).  get requires a
 * natural state (LBM_AA: even step count, Sec. 6) else LBM_ERR_STATE; solid
 * cells of a direct grid read back as 0.  get synchronises. */
lbm_status lbm_set_pdfs(lbm_t *h, const double *f, int on_device);
lbm_status lbm_get_pdfs(lbm_t *h, double *f, int on_device);

/* Enqueue n >= 0 time steps (collision and propagation, Sec. 1) by the
 * configured scheme (Sec. 2-7) on cfg->stream; returns without waiting.
 * LBM_ERR_STATE without a geometry. */
lbm_status lbm_step(lbm_t *h, int n);

/* Enqueue n >= 1 steps; the first kernel also reduces, in FP64 with a fixed
 * summation order, the mass sum(rho) and the flux sum(rho u_x) of the state
 * the call starts from, over all fluid nodes (the flow quantities of the
 * porous-media solver of Sec. 10; the paper gives no formula).  Requires a
 * natural starting state.  mass / jx are host pointers; synchronises. */
lbm_status lbm_step_flux(lbm_t *h, int n, double *mass, double *jx);

/* Mass and flux of the current (natural) state, FP64, fixed order (as
 * lbm_step_flux).  Synchronises. */
lbm_status lbm_flux(lbm_t *h, double *mass, double *jx);

/* Density (n) and velocity (3n) of the current natural state, the moments
 * of the collision (Sec. 1); either pointer may be NULL.  Synchronises when
 * on_device = 0. */
lbm_status lbm_macroscopics(lbm_t *h, double *rho, double *u, int on_device);

/* Wait for the handle's stream and report device-side errors. */
lbm_status lbm_sync(lbm_t *h);

/* Steady flow through a porous geometry and its permeability (the flow
 * through packed beds the paper's solver is built for, Sec. 10; Darcy's
 * law, which the paper does not state).  From the current state, runs rounds
 * of `check` steps (even, >= 2) with lbm_step_flux until the flux sum(rho
 * u_x) of two consecutive rounds differs by less than tol * |flux| (tol >=
 * 0), or until max_steps (>= check) steps are done.  Outputs (host pointers,
 * each may be NULL): permeability k = nu <rho u_x> / g_x with the average
 * over every cell of the box and nu = (1/omega - 1/2)/3 (NaN when g_x = 0),
 * the last round's mass and flux, and the steps done.  Returns LBM_OK when
 * steady, LBM_ERR_NOT_CONVERGED (outputs still written) at the step cap. */
lbm_status lbm_solve_permeability(lbm_t *h, int32_t check, double tol, int64_t max_steps, double *permeability,
                                  double *mass, double *flux, int64_t *steps);

/* ------------------------------------------------------------------------
 * Batches: many geometries advanced together (continuous batching; the
 * paper solves one geometry at a time, Sec. 10, so this layer has no
 * counterpart there, while every step of it is the node-list AA pattern of
 * Sec. 6 or esoteric twist of Sec. 7).
 *
 * Each admitted geometry is a fluid-node list stored as one segment of
 * shared SoA arrays (segments start on multiples of 4096 slots; IDX entries
 * are absolute slot numbers).  One round of k steps covers the nodes of
 * every active geometry, each with its own omega, force and step count, so
 * geometries admitted at different times run side by side.  A round is
 * replayed from a captured CUDA graph: one launch per step, or one
 * persistent cooperative launch for all k steps (round_mode).  Its first
 * step also reduces each geometry's mass and flux (FP64, per 4096-aligned
 * chunk, then summed in chunk order), so a geometry's results are
 * bit-identical alone and in any mix, in either round mode (its PDFs with
 * any launch shape, its sums with the same block size and nodes per
 * thread; other shapes differ in the last bits).  After each
 * round the library applies each geometry's steady-flux test (relative flux
 * change between consecutive rounds below its tol) and computes its
 * permeability.  Admissions build their geometry on a second stream, so
 * they overlap a round in flight; the next round waits for them. */
typedef struct lbm_batch_config {
  int32_t variant;           /* LBM_AA or LBM_ET (the starting variant when tune_variant = 1) */
  int32_t precision;         /* LBM_F64, LBM_F32, LBM_F16S */
  int32_t block_size;        /* threads per block: 64, 128, 256 or 512; 0 = 256 */
  int32_t nodes_per_thread;  /* 1, 2, 4 or 8; block_size * nodes_per_thread divides 4096; 0 = 1;
                                with LBM_F16S and LBM_AA, 2 or more run the chunk's nodes in
                                consecutive pairs (nodes_per_thread / 2 pairs per thread) */
  int64_t capacity_slots;    /* node slots of the shared arrays (rounded up to 4096) */
  int32_t max_geometries;    /* size of the geometry table */
  int32_t keep_idx;          /* LBM_AA: 1 = IDX keeps -1 for solid links; 0 = bounce-back slots
                                folded into IDX when the capacity is below 2^30 (faster) */
  double f16_scale;          /* LBM_F16S: the power-of-two scale of every geometry */
  int32_t tune_variant;      /* 1 = lbm_batch_tune may switch the batch between LBM_AA and LBM_ET
                                (index arrays sized for both: 18 words per slot); 0 = fixed */
  int32_t round_mode;        /* 0 = one launch per step in the round's graph; 1 = one persistent
                                cooperative launch per round (grid-wide barrier between steps with
                                a bounded wait: LBM_ERR_TIMEOUT instead of a hang) */
  void *stream;              /* cudaStream_t; NULL = default stream */
  lbm_alloc_fn dev_alloc;    /* optional device allocator, as in lbm_config */
  lbm_free_fn dev_free;
  void *alloc_ctx;
} lbm_batch_config;

typedef struct lbm_batch_info {
  int64_t capacity_slots;    /* slots per array */
  int64_t free_slots;        /* unreserved slots */
  int64_t largest_free;      /* largest contiguous free range */
  int64_t active_nodes;      /* fluid nodes of the active geometries */
  int64_t device_bytes;      /* PDF + index arrays */
  int32_t active_geometries;
  int32_t block_size;
  int32_t nodes_per_thread;
  int32_t work_chunks;       /* chunks of block_size * nodes_per_thread nodes per step */
  int32_t variant;           /* LBM_AA or LBM_ET, as tuned */
  int32_t round_mode;        /* as tuned */
} lbm_batch_info;

typedef struct lbm_batch lbm_batch_t;

/* Device bytes per node slot of a batch: 19 PDFs + the index words
 * (18 for LBM_AA or a batch whose variant may be tuned, 9 for LBM_ET;
 * Tab. 5 and Tab. 6 count the words each step reads). */
int64_t lbm_batch_bytes_per_slot(int32_t variant, int32_t precision);

/* Allocate the shared arrays (capacity_slots x bytes per slot).
 * LBM_ERR_OOM when they do not fit. */
lbm_status lbm_batch_create(const lbm_batch_config *cfg, lbm_batch_t **out);
lbm_status lbm_batch_destroy(lbm_batch_t *b);
const char *lbm_batch_last_error(const lbm_batch_t *b);

/* Admit a geometry given as a solid mask (nx*ny*nz bytes on the host, x
 * fastest, nonzero = solid; copied, so the caller may free it on return),
 * periodic[3] as in lbm_config, with its own omega, force[3], steady-flux
 * tolerance tol (>= 0) and step cap max_steps (<= 0: none), at rest.  Builds
 * its node list and index (Sec. 1; Tab. 5 / Tab. 6 layout) on the GPU into
 * the first free range that fits.  LBM_ERR_OOM (nothing changed) when no
 * range or geometry-table entry is free.  *slot receives its id.  Returns
 * once the geometry is built; its device work may still overlap a round in
 * flight. */
lbm_status lbm_batch_admit(lbm_batch_t *b, const uint8_t *mask, int32_t nx, int32_t ny, int32_t nz,
                           const int32_t *periodic, double omega, const double *force, double tol,
                           int64_t max_steps, int32_t *slot);

/* The same for a sphere pack (the packed bed of Sec. 10, Fig. 7), as
 * lbm_set_geometry_spheres: dims[3], periodic[3], nsph x 3 centres and the
 * radius in 1/unit cells. */
lbm_status lbm_batch_admit_spheres(lbm_batch_t *b, const int32_t *dims, const int32_t *periodic, int64_t nsph,
                                   const int64_t *centres, int64_t radius, int64_t unit, double omega,
                                   const double *force, double tol, int64_t max_steps, int32_t *slot);

/* Free a geometry's range and table entry (waits for a round in flight). */
lbm_status lbm_batch_release(lbm_batch_t *b, int32_t slot);

/* Enqueue k >= 1 steps of every active geometry (graph replay).
 * Asynchronous; the results become readable with lbm_batch_poll. */
lbm_status lbm_batch_round(lbm_batch_t *b, int32_t k);

/* State of one geometry after the last completed round (waits for a round
 * in flight): *done = 0 running, 1 steady (the flux of the state the last
 * round started from differs from the previous round's by less than tol
 * times its magnitude), 2 stopped at max_steps without reaching it;
 * *permeability = nu <rho u_x> / g_x from that flux, the average over every
 * cell of the geometry's box (Darcy's law; NaN when g_x = 0); *steps done.
 * Any output pointer may be NULL.  LBM_ERR_TIMEOUT if a persistent round's
 * grid barrier gave up. */
lbm_status lbm_batch_poll(lbm_batch_t *b, int32_t slot, int32_t *done, double *permeability, int64_t *steps);

/* FP64 mass sum(rho) and flux sum(rho u_x) of the state the last completed
 * round started from, and the steps done (waits for a round in flight). */
lbm_status lbm_batch_flux(lbm_batch_t *b, int32_t slot, double *mass, double *flux, int64_t *steps);
lbm_status lbm_batch_slot_info(lbm_batch_t *b, int32_t slot, int64_t *nodes, int64_t *cells, int64_t *steps);
lbm_status lbm_batch_get_info(lbm_batch_t *b, lbm_batch_info *info);

/* Natural state of one geometry (19 x nodes FP64, host; the AA pattern's
 * read-out after an even step count, Sec. 6, else LBM_ERR_STATE; the
 * esoteric twist's array map, Sec. 7).  Synchronises. */
lbm_status lbm_batch_get_pdfs(lbm_batch_t *b, int32_t slot, double *f_host);

/* Autotuner: times `rounds` rounds of k steps with CUDA events for every
 * candidate (variant: LBM_AA and LBM_ET when tune_variant = 1, else the
 * configured one; block size 128, 256, 512; nodes per thread 1, 2, 4, 8;
 * round mode 0 and 1) on the active geometries and keeps the fastest.
 * Every active geometry restarts from rest (step 0) in the chosen
 * configuration.  Outputs may be NULL. */
lbm_status lbm_batch_tune(lbm_batch_t *b, int32_t rounds, int32_t k, int32_t *best_variant, int32_t *best_block_size,
                          int32_t *best_nodes_per_thread, int32_t *best_round_mode, double *best_mflups);

/* Mass and flux of a caller-owned natural PDF array, with no allocation.
 * (This entry point has no counterpart in the paper.)
 *
 * For callers that cannot allocate device memory: a serving loop or a host
 * application whose device memory is already handed to its own pool (such
 * as PyTorch's caching allocator) cannot get more without a device-wide
 * synchronisation or a failure, and a latency-bound loop cannot afford the
 * implicit synchronisation of cudaFree.  This call makes no cudaMalloc,
 * cudaFree or other allocating call; its only scratch, the per-block partial
 * sums, is a fixed array inside the library (LBM_NOALLOC_MAX_BLOCKS x 2
 * doubles = 256 KiB on every GPU that loads the library, kept until exit).
 *
 *   f_dev      device array of the deviations f_i - w_i of n nodes in the
 *              library's storage form: precision LBM_F64 / LBM_F32 (values
 *              as is) or LBM_F16S (FP16 holding (f_i - w_i) * f16_scale);
 *              layout LBM_SOA (direction i of node k at i * npad + k,
 *              npad >= n) or LBM_AOS (at k * 19 + i, npad ignored)
 *   gx         body acceleration along x (the flux is sum rho u_x with
 *              u = (sum c f + rho g / 2) / rho, as lbm_flux)
 *   out_dev    device pointer to 2 doubles: sum rho, sum rho u_x (FP64,
 *              fixed summation order: block b sums nodes [b c, (b+1) c) with
 *              the chunk c = ceil(n / LBM_NOALLOC_MAX_BLOCKS) rounded up to
 *              a multiple of 256, at least LBM_NOALLOC_MIN_CHUNK, so the
 *              order, and the result's bits, depend on n alone)
 *   stream     cudaStream_t to enqueue on (NULL = default stream)
 *
 * Limits and errors: n must be in [1, LBM_NOALLOC_MAX_NODES] (2^30 nodes),
 * else LBM_ERR_INVALID_ARG; bad pointers or enums give LBM_ERR_INVALID_ARG; a
 * launch failure gives LBM_ERR_CUDA.  Every call made outside a stream
 * capture looks up the scratch's device address with the device current
 * (so a context created anew on the device is always served correctly); a
 * call under capture reuses the address of the device's last call, so make
 * one call on each device before capturing (else LBM_ERR_CUDA).  All calls
 * share the one scratch array and each rewrites the partials it reads:
 * calls that may overlap on the GPU (other streams or threads) race on it
 * and must be ordered by the caller.  Asynchronous: the result is in out_dev
 * once the stream reaches it. */
#define LBM_NOALLOC_MAX_BLOCKS 16384
#define LBM_NOALLOC_MIN_CHUNK 4096
#define LBM_NOALLOC_MAX_NODES (LBM_NOALLOC_MAX_BLOCKS * (int64_t)65536)
lbm_status lbm_flux_noalloc(const void *f_dev, int32_t precision, int32_t layout, int64_t n, int64_t npad,
                            double f16_scale, double gx, double *out_dev, void *stream);

/* Diagnostic, with no counterpart in the paper: the tile-staging kernels
 * wait for their tensor copies with a time limit and record a timeout
 * instead of spinning forever.  This call exercises that bounded wait on
 * purpose: one GPU thread waits on a shared-memory barrier that nothing
 * completes, for at most limit_ns nanoseconds (1000 .. 1e9).  Returns
 * LBM_ERR_TIMEOUT when the wait gave up as designed (the expected result),
 * LBM_OK if the barrier completed, LBM_ERR_INVALID_ARG for a limit out of
 * range, LBM_ERR_CUDA on a runtime error.  stream: cudaStream_t or NULL;
 * synchronises it. */
lbm_status lbm_selftest_bounded_wait(int64_t limit_ns, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
