/*
 * Plain FP64 CPU oracle for the D3Q19 lattice Boltzmann time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load the library built from this
 * file.  It shares nothing with the CUDA library: the velocity set, the
 * weights, the neighbour rules, the collision and the geometry builder are
 * all written out here on their own.
 *
 * Method: Wittmann, Zeiser, Hager, Wellein, "Comparison of different
 * Propagation Steps for the Lattice Boltzmann Method".
 *   - A time step is a collision at every fluid node followed by the
 *     propagation of the post-collision PDFs to the neighbours (Sec. 1, 2).
 *   - The paper's propagation schemes (two-step Sec. 2, one-step push and
 *     pull Sec. 3, compressed grid Sec. 4, swap Sec. 5, AA pattern Sec. 6,
 *     esoteric twist Sec. 7) change only where PDFs are stored and in which
 *     order nodes are visited; each is written out below in its serial form
 *     and all must give the same natural state after an even number of steps.
 *   - Full-grid ("direct") and sparse node-list ("indirect", IDX holding the
 *     q-1 neighbours of every node) addressing, Sec. 1.
 *
 * Readings where the paper is silent (its solver uses TRT, Sec. 10):
 *   - collision: BGK with the Guo body-force term, velocity reported as
 *     u = (sum c_i f_i + rho g / 2) / rho;
 *   - walls and solid nodes: half-way bounce-back; a link leaving the box
 *     through a non-periodic face is a wall link;
 *   - velocity order 0, +x, -x, +y, -y, +z, -z, then the twelve diagonals in
 *     opposite pairs; opp(i) = i+1 for odd i, i-1 for even i > 0.
 *
 * Layout: every PDF array here is natural, f[i * n + node], node = cell index
 * x + nx * (y + ny * z) on full grids or the fluid-node number on node lists.
 *
 * Built with -ffp-contract=off so results are identical on x86 and Arm.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 19

static const int CX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static const double W[Q] = {
    1.0 / 3.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

int ora_q(void) { return Q; }

/* Velocity set and weights, read back by the tests to pin them against the
 * D3Q19 moment identities (sum w = 1, sum w c c = I/3, ...). */
void ora_lattice(int *c /* 3*Q */, double *w /* Q */) {
  for (int i = 0; i < Q; ++i) {
    c[3 * i] = CX[i];
    c[3 * i + 1] = CY[i];
    c[3 * i + 2] = CZ[i];
    w[i] = W[i];
  }
}

/* ------------------------------------------------------------------------ */
/* Collision: BGK relaxation towards the second-order equilibrium plus the
 * Guo forcing term.  Input: the pre-collision PDFs of one node; output: the
 * post-collision PDFs.  omega = 0 with g = 0 is the identity. */
void ora_collide(const double *f, double omega, const double *g, double *out) {
  double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
  for (int i = 0; i < Q; ++i) {
    rho += f[i];
    jx += CX[i] * f[i];
    jy += CY[i] * f[i];
    jz += CZ[i] * f[i];
  }
  double ux = (jx + 0.5 * rho * g[0]) / rho;
  double uy = (jy + 0.5 * rho * g[1]) / rho;
  double uz = (jz + 0.5 * rho * g[2]) / rho;
  double usq = ux * ux + uy * uy + uz * uz;
  double ug = ux * g[0] + uy * g[1] + uz * g[2];
  for (int i = 0; i < Q; ++i) {
    double cu = CX[i] * ux + CY[i] * uy + CZ[i] * uz;
    double cg = CX[i] * g[0] + CY[i] * g[1] + CZ[i] * g[2];
    double feq = W[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
    double force = (1.0 - 0.5 * omega) * W[i] * rho * (3.0 * (cg - ug) + 9.0 * cu * cg);
    out[i] = f[i] - omega * (f[i] - feq) + force;
  }
}

/* Two-relaxation-time collision (TRT, the paper's solver, Sec. 10 and its
 * ref. [15]).  Each opposite pair (i, opp i) is split into its symmetric half
 * f+ = (f_i + f_opp)/2 and antisymmetric half f- = (f_i - f_opp)/2; the
 * symmetric halves relax towards feq+ with rate lam_p (sets the viscosity),
 * the antisymmetric halves towards feq- with rate lam_m.  The Guo forcing term
 * is split the same way, its symmetric half weighted by (1 - lam_p/2) and its
 * antisymmetric half by (1 - lam_m/2).  lam_m = lam_p is BGK. */
void ora_collide_trt(const double *f, double lam_p, double lam_m, const double *g, double *out) {
  double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
  for (int i = 0; i < Q; ++i) {
    rho += f[i];
    jx += CX[i] * f[i];
    jy += CY[i] * f[i];
    jz += CZ[i] * f[i];
  }
  double ux = (jx + 0.5 * rho * g[0]) / rho;
  double uy = (jy + 0.5 * rho * g[1]) / rho;
  double uz = (jz + 0.5 * rho * g[2]) / rho;
  double usq = ux * ux + uy * uy + uz * uz;
  double ug = ux * g[0] + uy * g[1] + uz * g[2];
  double feq[Q], fs[Q], fa[Q];
  for (int i = 0; i < Q; ++i) {
    double cu = CX[i] * ux + CY[i] * uy + CZ[i] * uz;
    double cg = CX[i] * g[0] + CY[i] * g[1] + CZ[i] * g[2];
    feq[i] = W[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
    /* Guo term, split into its parts even and odd in c_i */
    fs[i] = W[i] * rho * (9.0 * cu * cg - 3.0 * ug);
    fa[i] = W[i] * rho * 3.0 * cg;
  }
  for (int i = 0; i < Q; ++i) {
    int o = opp(i);
    double fp = 0.5 * (f[i] + f[o]), fm = 0.5 * (f[i] - f[o]);
    double ep = 0.5 * (feq[i] + feq[o]), em = 0.5 * (feq[i] - feq[o]);
    out[i] = f[i] - lam_p * (fp - ep) - lam_m * (fm - em) + (1.0 - 0.5 * lam_p) * fs[i] +
             (1.0 - 0.5 * lam_m) * fa[i];
  }
}

/* Antisymmetric rate from the symmetric one and the "magic" parameter
 * Lam = (1/lam_p - 1/2)(1/lam_m - 1/2). */
double ora_trt_lambda_minus(double lam_p, double magic) {
  return 1.0 / (0.5 + magic / (1.0 / lam_p - 0.5));
}

/* Density and velocity of one node (the velocity includes the half force). */
void ora_node_moments(const double *f, const double *g, double *rho_out, double *u_out) {
  double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
  for (int i = 0; i < Q; ++i) {
    rho += f[i];
    jx += CX[i] * f[i];
    jy += CY[i] * f[i];
    jz += CZ[i] * f[i];
  }
  *rho_out = rho;
  u_out[0] = (jx + 0.5 * rho * g[0]) / rho;
  u_out[1] = (jy + 0.5 * rho * g[1]) / rho;
  u_out[2] = (jz + 0.5 * rho * g[2]) / rho;
}

/* Equilibrium f_eq(rho, u) of one node. */
void ora_equilibrium(double rho, const double *u, double *out) {
  double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < Q; ++i) {
    double cu = CX[i] * u[0] + CY[i] * u[1] + CZ[i] * u[2];
    out[i] = W[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
  }
}

/* ------------------------------------------------------------------------ */
/* Full grid ("direct addressing", Sec. 1).  dims = {nx, ny, nz}; periodic[a]
 * = 1 wraps axis a, 0 puts a bounce-back wall half a cell beyond each face.
 * solid may be NULL (every cell fluid). */
typedef struct {
  int n[3];
  int per[3];
  const uint8_t *solid;
} box_t;

static box_t make_box(const int *dims, const int *periodic, const uint8_t *solid) {
  box_t b;
  for (int a = 0; a < 3; ++a) {
    b.n[a] = dims[a];
    b.per[a] = periodic[a];
  }
  b.solid = solid;
  return b;
}

static int64_t ncells(const box_t *b) { return (int64_t)b->n[0] * b->n[1] * b->n[2]; }

static int64_t cell_index(const box_t *b, int x, int y, int z) {
  return (int64_t)x + (int64_t)b->n[0] * ((int64_t)y + (int64_t)b->n[1] * z);
}

static void cell_coords(const box_t *b, int64_t c, int *x, int *y, int *z) {
  *x = (int)(c % b->n[0]);
  c /= b->n[0];
  *y = (int)(c % b->n[1]);
  *z = (int)(c / b->n[1]);
}

static int is_fluid(const box_t *b, int64_t c) { return b->solid == NULL || b->solid[c] == 0; }

/* Wrap coordinate v on axis a; returns 0 if v leaves a non-periodic axis. */
static int wrap(const box_t *b, int a, int v, int *out) {
  int n = b->n[a];
  if (v >= 0 && v < n) {
    *out = v;
    return 1;
  }
  if (!b->per[a]) return 0;
  *out = ((v % n) + n) % n;
  return 1;
}

/* Cell reached from cell c along c_i, or -1 for a wall or a solid cell. */
static int64_t neighbour(const box_t *b, int64_t c, int i) {
  int x, y, z, xx, yy, zz;
  cell_coords(b, c, &x, &y, &z);
  if (!wrap(b, 0, x + CX[i], &xx)) return -1;
  if (!wrap(b, 1, y + CY[i], &yy)) return -1;
  if (!wrap(b, 2, z + CZ[i], &zz)) return -1;
  int64_t d = cell_index(b, xx, yy, zz);
  return is_fluid(b, d) ? d : -1;
}

/* The definition of one time step (Sec. 2/3, push form): f_out = S(C(f_in)).
 * Every fluid cell is collided and each post-collision PDF moves to the
 * neighbour along c_i; a PDF whose target is a wall or solid cell returns to
 * its own cell in the opposite direction (half-way bounce-back).  PDFs of
 * solid cells are copied through unchanged. */
void ora_push_full(const int *dims, const int *periodic, const uint8_t *solid, const double *fin,
                   double *fout, double omega, const double *g, int nthreads) {
  box_t b = make_box(dims, periodic, solid);
  int64_t n = ncells(&b);
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int64_t c = 0; c < n; ++c) {
    if (!is_fluid(&b, c)) {
      for (int i = 0; i < Q; ++i) fout[i * n + c] = fin[i * n + c];
      continue;
    }
    double f[Q], fs[Q];
    for (int i = 0; i < Q; ++i) f[i] = fin[i * n + c];
    ora_collide(f, omega, g, fs);
    for (int i = 0; i < Q; ++i) {
      int64_t d = (i == 0) ? c : neighbour(&b, c, i);
      if (d >= 0)
        fout[i * n + d] = fs[i];
      else
        fout[opp(i) * n + c] = fs[i];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Sparse node list ("indirect addressing", Sec. 1): fluid cells numbered in
 * lexicographic order (x fastest).  node_of[cell] = node number or -1;
 * cells[node] = cell index.  Returns the number of fluid nodes. */
int64_t ora_build_nodes(const int *dims, const int *periodic, const uint8_t *solid,
                        int32_t *node_of, int32_t *cells) {
  box_t b = make_box(dims, periodic, solid);
  int64_t n = ncells(&b), count = 0;
  for (int64_t c = 0; c < n; ++c) {
    if (is_fluid(&b, c)) {
      node_of[c] = (int32_t)count;
      cells[count] = (int32_t)c;
      ++count;
    } else {
      node_of[c] = -1;
    }
  }
  return count;
}

/* IDX (Sec. 1): idx[(i-1) * N + node] = node number of the neighbour along
 * c_i for i = 1..18, or -1 if that neighbour is a wall or solid. */
void ora_build_idx(const int *dims, const int *periodic, const uint8_t *solid,
                   const int32_t *node_of, const int32_t *cells, int64_t nnodes, int32_t *idx) {
  box_t b = make_box(dims, periodic, solid);
  for (int64_t k = 0; k < nnodes; ++k) {
    for (int i = 1; i < Q; ++i) {
      int64_t d = neighbour(&b, cells[k], i);
      idx[(int64_t)(i - 1) * nnodes + k] = d >= 0 ? node_of[d] : -1;
    }
  }
}

/* One time step on a node list, the same definition as ora_push_full with
 * neighbours taken from IDX. */
void ora_push_sparse(int64_t nnodes, const int32_t *idx, const double *fin, double *fout,
                     double omega, const double *g, int nthreads) {
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int64_t k = 0; k < nnodes; ++k) {
    double f[Q], fs[Q];
    for (int i = 0; i < Q; ++i) f[i] = fin[i * nnodes + k];
    ora_collide(f, omega, g, fs);
    fout[k] = fs[0];
    for (int i = 1; i < Q; ++i) {
      int32_t d = idx[(int64_t)(i - 1) * nnodes + k];
      if (d >= 0)
        fout[i * nnodes + d] = fs[i];
      else
        fout[opp(i) * nnodes + k] = fs[i];
    }
  }
}

/* Post-collision PDFs of a sample of nodes from a state on a node list:
 * out[s * Q + i] = C(f)(node sample[s]) (used to check single outputs of a
 * large GPU step one by one). */
void ora_collide_nodes(int64_t nnodes, const double *f, int64_t nsample, const int64_t *sample,
                       double omega, const double *g, double *out) {
  for (int64_t s = 0; s < nsample; ++s) {
    double fl[Q];
    for (int i = 0; i < Q; ++i) fl[i] = f[i * nnodes + sample[s]];
    ora_collide(fl, omega, g, out + s * Q);
  }
}

/* Density and velocity of every node of a natural state. */
void ora_macroscopics(int64_t nnodes, const double *f, const double *g, double *rho, double *u) {
  for (int64_t k = 0; k < nnodes; ++k) {
    double fl[Q];
    for (int i = 0; i < Q; ++i) fl[i] = f[i * nnodes + k];
    ora_node_moments(fl, g, rho + k, u + 3 * k);
  }
}

/* Mass sum(rho) and flux sum(rho u_x) over the listed nodes (all nodes when
 * list == NULL), summed in node order. */
void ora_flux(int64_t nnodes, const double *f, const double *g, const uint8_t *skip,
              double *mass, double *jx) {
  double m = 0.0, j = 0.0;
  for (int64_t k = 0; k < nnodes; ++k) {
    if (skip && skip[k]) continue;
    double fl[Q], rho, u[3];
    for (int i = 0; i < Q; ++i) fl[i] = f[i * nnodes + k];
    ora_node_moments(fl, g, &rho, u);
    m += rho;
    j += rho * u[0];
  }
  *mass = m;
  *jx = j;
}

/* ------------------------------------------------------------------------ */
/* Geometry: a cell is solid iff its centre lies within distance r of some
 * sphere centre (overlapping spheres, the packed bed of Fig. 7 and Sec. 10).
 * Positions are integers in units of 1/unit lattice spacing, so the test
 * d^2 <= r^2 is exact.  Distances use the minimum image on periodic axes.
 * Each sphere marks the cells of its bounding box that pass the test. */
static int64_t axis_delta(int64_t p, int64_t c, int64_t len, int periodic) {
  int64_t d = p - c;
  if (!periodic) return d;
  d %= len;
  if (d < 0) d += len;
  if (2 * d > len) d -= len;
  return d;
}

void ora_sphere_mask(const int *dims, const int *periodic, int64_t nsph, const int64_t *centres,
                     int64_t radius, int64_t unit, uint8_t *solid) {
  box_t b = make_box(dims, periodic, NULL);
  memset(solid, 0, (size_t)ncells(&b));
  int64_t r2 = radius * radius;
  for (int64_t s = 0; s < nsph; ++s) {
    int64_t lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      int64_t c = centres[3 * s + a];
      /* cells v with |v*unit - c| <= r: ceil((c-r)/unit) .. floor((c+r)/unit) */
      int64_t l = c - radius, h = c + radius;
      lo[a] = (l >= 0) ? (l + unit - 1) / unit : -((-l) / unit);
      hi[a] = (h >= 0) ? h / unit : -((-h + unit - 1) / unit);
    }
    for (int64_t vz = lo[2]; vz <= hi[2]; ++vz)
      for (int64_t vy = lo[1]; vy <= hi[1]; ++vy)
        for (int64_t vx = lo[0]; vx <= hi[0]; ++vx) {
          int64_t v[3] = {vx, vy, vz};
          int w[3], ok = 1;
          for (int a = 0; a < 3 && ok; ++a) {
            int64_t n = b.n[a];
            if (v[a] >= 0 && v[a] < n)
              w[a] = (int)v[a];
            else if (b.per[a])
              w[a] = (int)(((v[a] % n) + n) % n);
            else
              ok = 0;
          }
          if (!ok) continue;
          int64_t d2 = 0;
          for (int a = 0; a < 3; ++a) {
            int64_t len = (int64_t)b.n[a] * unit;
            int64_t d = axis_delta((int64_t)w[a] * unit, centres[3 * s + a], len, b.per[a]);
            d2 += d * d;
          }
          if (d2 <= r2) solid[cell_index(&b, w[0], w[1], w[2])] = 1;
        }
  }
}

/* ------------------------------------------------------------------------ */
/* The propagation schemes of Sec. 2-7 in their serial form on a full grid.
 * Each routine takes the natural state f (Q arrays of ncells), runs nsteps
 * time steps with its own storage scheme and returns the natural state in
 * fout.  Return value: 0 on success, -1 on bad arguments. */

enum { ORA_TS = 0, ORA_OS_PUSH, ORA_OS_PULL, ORA_CG, ORA_SWAP, ORA_AA, ORA_ET };

static void load_node(const double *a, int64_t n, int64_t c, double *f) {
  for (int i = 0; i < Q; ++i) f[i] = a[i * n + c];
}

/* Push streaming alone (S): post-collision array -> natural array. */
static void stream_push(const box_t *b, const double *post, double *nat) {
  int64_t n = ncells(b);
  for (int64_t c = 0; c < n; ++c) {
    if (!is_fluid(b, c)) continue;
    for (int i = 0; i < Q; ++i) {
      int64_t d = (i == 0) ? c : neighbour(b, c, i);
      if (d >= 0)
        nat[i * n + d] = post[i * n + c];
      else
        nat[opp(i) * n + c] = post[i * n + c];
    }
  }
}

/* Inverse streaming (S^-1): natural array -> the array whose push
 * streaming gives it.  S is a permutation of the (cell, direction) slots. */
static void stream_pull_inverse(const box_t *b, const double *nat, double *post) {
  int64_t n = ncells(b);
  for (int64_t c = 0; c < n; ++c) {
    if (!is_fluid(b, c)) continue;
    for (int i = 0; i < Q; ++i) {
      int64_t s = (i == 0) ? c : neighbour(b, c, opp(i)); /* cell c - c_i */
      if (s >= 0)
        post[i * n + s] = nat[i * n + c];
      else
        post[opp(i) * n + c] = nat[i * n + c];
    }
  }
}

/* Two-step (Sec. 2, Tab. 1): collide A -> B at the same cell, then a second
 * loop streams B -> A. */
static void run_ts(const box_t *b, double *A, double *B, int nsteps, double omega, const double *g) {
  int64_t n = ncells(b);
  for (int t = 0; t < nsteps; ++t) {
    for (int64_t c = 0; c < n; ++c) {
      if (!is_fluid(b, c)) continue;
      double f[Q], fs[Q];
      load_node(A, n, c, f);
      ora_collide(f, omega, g, fs);
      for (int i = 0; i < Q; ++i) B[i * n + c] = fs[i];
    }
    stream_push(b, B, A);
  }
}

/* One-step push (Sec. 3, Fig. 1a,b): collide in A, scatter to B, swap. */
static void run_os_push(const box_t *b, double *A, double *B, int nsteps, double omega,
                        const double *g) {
  int64_t n = ncells(b);
  for (int t = 0; t < nsteps; ++t) {
    for (int64_t c = 0; c < n; ++c) {
      if (!is_fluid(b, c)) continue;
      double f[Q], fs[Q];
      load_node(A, n, c, f);
      ora_collide(f, omega, g, fs);
      for (int i = 0; i < Q; ++i) {
        int64_t d = (i == 0) ? c : neighbour(b, c, i);
        if (d >= 0)
          B[i * n + d] = fs[i];
        else
          B[opp(i) * n + c] = fs[i];
      }
    }
    double *tmp = A;
    A = B;
    B = tmp;
  }
  if (nsteps & 1) memcpy(B, A, sizeof(double) * Q * (size_t)n); /* result back in the caller's A */
}

/* One-step pull (Sec. 3, Fig. 1c,d): gather from the neighbours of A,
 * collide, store locally into B.  The stored state is post-collision, so the
 * natural state is its push streaming. */
static void run_os_pull(const box_t *b, double *A, double *B, int nsteps, double omega,
                        const double *g) {
  int64_t n = ncells(b);
  for (int t = 0; t < nsteps; ++t) {
    for (int64_t c = 0; c < n; ++c) {
      if (!is_fluid(b, c)) continue;
      double f[Q], fs[Q];
      for (int i = 0; i < Q; ++i) {
        int64_t s = (i == 0) ? c : neighbour(b, c, opp(i));
        f[i] = (s >= 0) ? A[i * n + s] : A[opp(i) * n + c];
      }
      ora_collide(f, omega, g, fs);
      for (int i = 0; i < Q; ++i) B[i * n + c] = fs[i];
    }
    double *tmp = A;
    A = B;
    B = tmp;
  }
  if (nsteps & 1) memcpy(B, A, sizeof(double) * Q * (size_t)n);
}

/* Swap (Sec. 5, Fig. 3, push form), one lattice, strict lexicographic order.
 * A node is collided and its post-collision PDF along c_i is written into its
 * own slot of the opposite direction; every link to a fluid neighbour visited
 * earlier in this sweep is then completed by exchanging the two PDFs that
 * travel along it.  Links into walls or solids need no exchange: the
 * reversed slot already holds the bounced-back PDF. */
static void run_swap(const box_t *b, double *A, int nsteps, double omega, const double *g) {
  int64_t n = ncells(b);
  for (int t = 0; t < nsteps; ++t) {
    for (int64_t c = 0; c < n; ++c) {
      if (!is_fluid(b, c)) continue;
      double f[Q], fs[Q];
      load_node(A, n, c, f);
      ora_collide(f, omega, g, fs);
      for (int i = 0; i < Q; ++i) A[opp(i) * n + c] = fs[i];
      for (int i = 1; i < Q; ++i) {
        int64_t d = neighbour(b, c, i);
        if (d >= 0 && d < c) {
          double tmp = A[opp(i) * n + c];
          A[opp(i) * n + c] = A[i * n + d];
          A[i * n + d] = tmp;
        }
      }
    }
  }
}

/* AA pattern (Sec. 6, Fig. 5).  Even step: read the node's own PDFs, write
 * the post-collision PDF of direction i into the node's slot of the opposite
 * direction.  Odd step: read the PDFs pointing at the node from the
 * neighbours' opposite slots, write the results to the neighbours in natural
 * orientation.  After an even number of steps the array is natural. */
static void aa_even(const box_t *b, double *A, double omega, const double *g) {
  int64_t n = ncells(b);
  for (int64_t c = 0; c < n; ++c) {
    if (!is_fluid(b, c)) continue;
    double f[Q], fs[Q];
    load_node(A, n, c, f);
    ora_collide(f, omega, g, fs);
    for (int i = 0; i < Q; ++i) A[opp(i) * n + c] = fs[i];
  }
}

static void aa_odd(const box_t *b, double *A, double omega, const double *g) {
  int64_t n = ncells(b);
  for (int64_t c = 0; c < n; ++c) {
    if (!is_fluid(b, c)) continue;
    double f[Q], fs[Q];
    for (int i = 0; i < Q; ++i) {
      int64_t s = (i == 0) ? c : neighbour(b, c, opp(i)); /* cell c - c_i */
      f[i] = (s >= 0) ? A[opp(i) * n + s] : A[i * n + c];
    }
    ora_collide(f, omega, g, fs);
    for (int i = 0; i < Q; ++i) {
      int64_t d = (i == 0) ? c : neighbour(b, c, i);
      if (d >= 0)
        A[i * n + d] = fs[i];
      else
        A[opp(i) * n + c] = fs[i];
    }
  }
}

/* Padded storage used by the esoteric twist and the compressed grid: the box
 * plus h cells on both sides of every axis, so that positions one cell past a
 * face (or two for the shifted grid) have a slot of their own. */
typedef struct {
  int h;
  int64_t s[3];
} pad_t;

static pad_t make_pad(const box_t *b, int h, int extra) {
  pad_t p;
  p.h = h;
  for (int a = 0; a < 3; ++a) p.s[a] = b->n[a] + 2 * h + extra;
  return p;
}

static int64_t pad_size(const pad_t *p) { return p->s[0] * p->s[1] * p->s[2]; }

static int64_t pad_index(const pad_t *p, int x, int y, int z) {
  return (int64_t)(x + p->h) + p->s[0] * ((int64_t)(y + p->h) + p->s[1] * (int64_t)(z + p->h));
}

/* Esoteric twist (Sec. 7, Fig. 6).  Physical arrays P_k and a map a(i) from
 * direction to array (the paper's control structure of pointers).  PDF f_i of
 * node x lives in P_{a(i)} at x + s(i), with s(i) = 0 for i = 0 and the odd
 * directions and s(i) = c_{opp(i)} for the even directions, i.e. half the PDFs
 * of a node sit at the node and the other half at its neighbours along the
 * odd directions.  A node reads its 19 PDFs, collides, and writes the
 * post-collision PDF of direction i to P_{a(opp i)} at x + s(opp i); after the
 * sweep a(i) and a(opp i) are exchanged, which completes the propagation.
 * Bounce-back writes to P_{a(i)} at x + s(opp i) instead.  Positions past a
 * wall or in a solid cell are ghost slots of the padded storage. */
static void et_pos(const box_t *b, int x, int y, int z, int i, int *px, int *py, int *pz) {
  int sx = 0, sy = 0, sz = 0;
  if (i != 0 && !(i & 1)) {
    sx = CX[opp(i)];
    sy = CY[opp(i)];
    sz = CZ[opp(i)];
  }
  int v[3] = {x + sx, y + sy, z + sz};
  for (int a = 0; a < 3; ++a)
    if (b->per[a]) v[a] = ((v[a] % b->n[a]) + b->n[a]) % b->n[a];
  *px = v[0];
  *py = v[1];
  *pz = v[2];
}

static void run_et(const box_t *b, const double *fin, double *fout, int nsteps, double omega,
                   const double *g) {
  int64_t n = ncells(b);
  pad_t p = make_pad(b, 1, 0);
  int64_t ps = pad_size(&p);
  double *P = (double *)calloc((size_t)Q * ps, sizeof(double));
  int a[Q];
  for (int i = 0; i < Q; ++i) a[i] = i;
  /* initial placement */
  for (int64_t c = 0; c < n; ++c) {
    if (!is_fluid(b, c)) continue;
    int x, y, z, px, py, pz;
    cell_coords(b, c, &x, &y, &z);
    for (int i = 0; i < Q; ++i) {
      et_pos(b, x, y, z, i, &px, &py, &pz);
      P[a[i] * ps + pad_index(&p, px, py, pz)] = fin[i * n + c];
    }
  }
  for (int t = 0; t < nsteps; ++t) {
    for (int64_t c = 0; c < n; ++c) {
      if (!is_fluid(b, c)) continue;
      int x, y, z, px, py, pz;
      cell_coords(b, c, &x, &y, &z);
      double f[Q], fs[Q];
      for (int i = 0; i < Q; ++i) {
        et_pos(b, x, y, z, i, &px, &py, &pz);
        f[i] = P[a[i] * ps + pad_index(&p, px, py, pz)];
      }
      ora_collide(f, omega, g, fs);
      for (int i = 0; i < Q; ++i) {
        et_pos(b, x, y, z, opp(i), &px, &py, &pz);
        int64_t slot = pad_index(&p, px, py, pz);
        int linked = (i == 0) || neighbour(b, c, i) >= 0;
        if (linked)
          P[a[opp(i)] * ps + slot] = fs[i];
        else
          P[a[i] * ps + slot] = fs[i];
      }
    }
    int na[Q];
    for (int i = 0; i < Q; ++i) na[i] = a[opp(i)];
    memcpy(a, na, sizeof a);
  }
  for (int64_t c = 0; c < n; ++c) {
    int x, y, z, px, py, pz;
    if (!is_fluid(b, c)) {
      for (int i = 0; i < Q; ++i) fout[i * n + c] = fin[i * n + c];
      continue;
    }
    cell_coords(b, c, &x, &y, &z);
    for (int i = 0; i < Q; ++i) {
      et_pos(b, x, y, z, i, &px, &py, &pz);
      fout[i * n + c] = P[a[i] * ps + pad_index(&p, px, py, pz)];
    }
  }
  free(P);
}

/* Compressed grid (Sec. 4, Fig. 2), pull form.  One lattice enlarged by one
 * cell per axis (plus a one-cell halo on each side for the periodic copies).
 * The post-collision state of node x sits at x + o with o alternating between
 * (0,0,0) and (1,1,1).  A sweep gathers from the old position and writes to
 * the new one; it runs from high to low cells when the shift is +1 and from
 * low to high when it is -1, so a slot is overwritten only after every node
 * that reads it has been updated.  Before each sweep the periodic halo is
 * filled with copies of the opposite face, so that the sweep never wraps. */
static void cg_fill_halo(const box_t *b, const pad_t *p, double *S, int o) {
  int64_t ps = pad_size(p);
  int lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = o - 1;
    hi[a] = b->n[a] + o; /* halo cells on both sides of the data range [o, n+o) */
  }
  for (int a = 0; a < 3; ++a) {
    if (!b->per[a]) continue;
    int na = b->n[a];
    /* fill axis a's two halo faces over the full extent of the axes already
     * filled and the data range of the others */
    int r0[3], r1[3];
    for (int e = 0; e < 3; ++e) {
      if (e < a && b->per[e]) {
        r0[e] = lo[e];
        r1[e] = hi[e];
      } else {
        r0[e] = o;
        r1[e] = b->n[e] + o - 1;
      }
    }
    for (int side = 0; side < 2; ++side) {
      int dst = side == 0 ? lo[a] : hi[a];
      int src = side == 0 ? na - 1 + o : o;
      int v[3];
      for (v[2] = r0[2]; v[2] <= r1[2]; ++v[2])
        for (v[1] = r0[1]; v[1] <= r1[1]; ++v[1])
          for (v[0] = r0[0]; v[0] <= r1[0]; ++v[0]) {
            if (v[a] != r0[a]) continue; /* one layer */
            int s[3] = {v[0], v[1], v[2]}, d[3] = {v[0], v[1], v[2]};
            s[a] = src;
            d[a] = dst;
            for (int i = 0; i < Q; ++i)
              S[i * ps + pad_index(p, d[0], d[1], d[2])] = S[i * ps + pad_index(p, s[0], s[1], s[2])];
          }
    }
  }
}

static void run_cg(const box_t *b, const double *fin, double *fout, int nsteps, double omega,
                   const double *g) {
  int64_t n = ncells(b);
  pad_t p = make_pad(b, 1, 1); /* positions -1 .. n+1 on every axis */
  int64_t ps = pad_size(&p);
  double *S = (double *)calloc((size_t)Q * ps, sizeof(double));
  double *post = (double *)calloc((size_t)Q * n, sizeof(double));
  stream_pull_inverse(b, fin, post);
  int o = 0;
  for (int64_t c = 0; c < n; ++c) {
    if (!is_fluid(b, c)) continue;
    int x, y, z;
    cell_coords(b, c, &x, &y, &z);
    for (int i = 0; i < Q; ++i) S[i * ps + pad_index(&p, x + o, y + o, z + o)] = post[i * n + c];
  }
  for (int t = 0; t < nsteps; ++t) {
    int on = 1 - o; /* new shift */
    cg_fill_halo(b, &p, S, o);
    for (int64_t k = 0; k < n; ++k) {
      int64_t c = (on > o) ? (n - 1 - k) : k;
      if (!is_fluid(b, c)) continue;
      int x, y, z;
      cell_coords(b, c, &x, &y, &z);
      double f[Q], fs[Q];
      for (int i = 0; i < Q; ++i) {
        int sx = x - CX[i], sy = y - CY[i], sz = z - CZ[i];
        int64_t src = (i == 0) ? c : neighbour(b, c, opp(i));
        if (src >= 0) /* unwrapped position: the halo holds the periodic copy */
          f[i] = S[i * ps + pad_index(&p, sx + o, sy + o, sz + o)];
        else
          f[i] = S[opp(i) * ps + pad_index(&p, x + o, y + o, z + o)];
      }
      ora_collide(f, omega, g, fs);
      for (int i = 0; i < Q; ++i) S[i * ps + pad_index(&p, x + on, y + on, z + on)] = fs[i];
    }
    o = on;
  }
  for (int64_t c = 0; c < n; ++c) {
    if (!is_fluid(b, c)) continue;
    int x, y, z;
    cell_coords(b, c, &x, &y, &z);
    for (int i = 0; i < Q; ++i) post[i * n + c] = S[i * ps + pad_index(&p, x + o, y + o, z + o)];
  }
  for (int64_t k = 0; k < (int64_t)Q * n; ++k) fout[k] = fin[k]; /* solid cells pass through */
  stream_push(b, post, fout);
  free(post);
  free(S);
}

int ora_run_variant(int variant, const int *dims, const int *periodic, const uint8_t *solid,
                    const double *fin, double *fout, int nsteps, double omega, const double *g) {
  box_t b = make_box(dims, periodic, solid);
  int64_t n = ncells(&b);
  for (int a = 0; a < 3; ++a)
    if (b.n[a] < 1 || (b.per[a] && b.n[a] < 2)) return -1;
  if (nsteps < 0) return -1;
  if (variant == ORA_AA && (nsteps & 1)) return -1;
  size_t bytes = sizeof(double) * Q * (size_t)n;
  double *A = (double *)malloc(bytes), *B = (double *)malloc(bytes);
  memcpy(A, fin, bytes);
  memcpy(B, fin, bytes);
  int rc = 0;
  switch (variant) {
    case ORA_TS:
      run_ts(&b, A, B, nsteps, omega, g);
      memcpy(fout, A, bytes);
      break;
    case ORA_OS_PUSH:
      run_os_push(&b, A, B, nsteps, omega, g); /* result left in A */
      memcpy(fout, A, bytes);
      break;
    case ORA_OS_PULL:
      stream_pull_inverse(&b, fin, A);
      run_os_pull(&b, A, B, nsteps, omega, g); /* result left in A */
      memcpy(fout, fin, bytes);
      stream_push(&b, A, fout);
      break;
    case ORA_CG:
      run_cg(&b, fin, fout, nsteps, omega, g);
      break;
    case ORA_SWAP:
      run_swap(&b, A, nsteps, omega, g);
      memcpy(fout, A, bytes);
      break;
    case ORA_AA:
      for (int t = 0; t < nsteps; t += 2) {
        aa_even(&b, A, omega, g);
        aa_odd(&b, A, omega, g);
      }
      memcpy(fout, A, bytes);
      break;
    case ORA_ET:
      run_et(&b, fin, fout, nsteps, omega, g);
      break;
    default:
      rc = -1;
  }
  free(A);
  free(B);
  return rc;
}

/* One step of the definition with the TRT collision (full grid). */
void ora_push_full_trt(const int *dims, const int *periodic, const uint8_t *solid, const double *fin,
                       double *fout, double lam_p, double lam_m, const double *g, int nthreads) {
  box_t b = make_box(dims, periodic, solid);
  int64_t n = ncells(&b);
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int64_t c = 0; c < n; ++c) {
    if (!is_fluid(&b, c)) {
      for (int i = 0; i < Q; ++i) fout[i * n + c] = fin[i * n + c];
      continue;
    }
    double f[Q], fs[Q];
    for (int i = 0; i < Q; ++i) f[i] = fin[i * n + c];
    ora_collide_trt(f, lam_p, lam_m, g, fs);
    for (int i = 0; i < Q; ++i) {
      int64_t d = (i == 0) ? c : neighbour(&b, c, i);
      if (d >= 0)
        fout[i * n + d] = fs[i];
      else
        fout[opp(i) * n + c] = fs[i];
    }
  }
}

void ora_run_push_full_trt(const int *dims, const int *periodic, const uint8_t *solid, double *f, int nsteps,
                           double lam_p, double lam_m, const double *g, int nthreads) {
  box_t b = make_box(dims, periodic, solid);
  size_t bytes = sizeof(double) * Q * (size_t)ncells(&b);
  double *tmp = (double *)malloc(bytes);
  for (int t = 0; t < nsteps; ++t) {
    ora_push_full_trt(dims, periodic, solid, f, tmp, lam_p, lam_m, g, nthreads);
    memcpy(f, tmp, bytes);
  }
  free(tmp);
}

/* nsteps of the definition, the state kept in f (natural, in place). */
void ora_run_push_full(const int *dims, const int *periodic, const uint8_t *solid, double *f,
                       int nsteps, double omega, const double *g, int nthreads) {
  box_t b = make_box(dims, periodic, solid);
  size_t bytes = sizeof(double) * Q * (size_t)ncells(&b);
  double *tmp = (double *)malloc(bytes);
  for (int t = 0; t < nsteps; ++t) {
    ora_push_full(dims, periodic, solid, f, tmp, omega, g, nthreads);
    memcpy(f, tmp, bytes);
  }
  free(tmp);
}

void ora_run_push_sparse(int64_t nnodes, const int32_t *idx, double *f, int nsteps, double omega,
                         const double *g, int nthreads) {
  size_t bytes = sizeof(double) * Q * (size_t)nnodes;
  double *tmp = (double *)malloc(bytes);
  for (int t = 0; t < nsteps; ++t) {
    ora_push_sparse(nnodes, idx, f, tmp, omega, g, nthreads);
    memcpy(f, tmp, bytes);
  }
  free(tmp);
}
