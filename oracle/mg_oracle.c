/*
 * FP64 CPU oracle for the elliptic solves of Marskar, "Adaptive multiscale
 * methods for 3D streamer discharges in air" (arXiv:1809.08857).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link or call
 * this file: only the tests, the smoke check and the CPU baseline leg of the
 * benchmark use it.  It shares no code, header or table with the CUDA library.
 *
 * What it computes (Sec. 2, Eqs. 2-3 and items (ii)-(iii) of the spatial
 * discretisation list): the second-order cell-centred finite-volume system
 *
 *     (A u)_c = alpha u_c + sum_faces w_f (u_c - u_nb) / h^2 = f_c
 *
 * on a uniform Cartesian box, solved by geometric multigrid with red-black
 * Gauss-Seidel smoothing (Sec. 2, item (ii)).  Readings of what the paper
 * leaves open:
 *   - face coefficient between two free cells: harmonic mean of their beta;
 *   - face towards an electrode (masked) cell: the free cell's beta, with the
 *     electrode value held at the masked cell's centre;
 *   - Dirichlet domain face with value g: ghost 2g - u_c, so w = 2 beta_c;
 *   - Neumann domain face: homogeneous, no flux;
 *   - coarse grids: cell masked iff at least 3 of its 8 children are (a
 *     reading: the paper gives no coarsening rule; the rule shapes the coarse
 *     operators, not the converged answer), beta = mean of the free
 *     children, residual restricted by the 8-child average, correction
 *     prolonged trilinearly; the coarsest grid is solved by dense Cholesky.
 * The paper's coarse solver is BiCGStab; a dense factor on the small coarsest
 * grid reaches the same discrete answer.
 *
 * Layout: x fastest, index (k*ny + j)*nx + i.  Faces are ordered
 * -x, +x, -y, +y, -z, +z.  bc_kind 0 = Dirichlet, 1 = Neumann, 2 = Robin
 * n.grad u + a u = 0 with a = bc_value (outward normal n; the Marshak
 * condition of the radiative-transfer equations):
 *   face value (u_c + u_g)/2 and normal derivative (u_g - u_c)/h give the
 *   ghost u_g = u_c (1 - a h/2)/(1 + a h/2), so the face adds
 *   2 beta_c rho / h^2 to the diagonal with rho = (a h/2)/(1 + a h/2)
 *   (rho = 1: homogeneous Dirichlet, rho = 0: Neumann).  Coarse grids use
 *   their own h.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int nx, ny, nz;
  double h;
  int bc_kind[6];
  double bc_value[6];
  /* optional per-face-cell Dirichlet values, packed: faces -x, +x (ny*nz,
   * index k*ny + j), -y, +y (nx*nz, index k*nx + i), -z, +z (nx*ny, index
   * j*nx + i); NULL means bc_value[face] on the whole face */
  const double* face_data;
} or_grid;

#define OR_MAX_LEVELS 24

static long ncell(const or_grid* g) { return (long)g->nx * g->ny * g->nz; }
static long idx(const or_grid* g, int i, int j, int k) {
  return ((long)k * g->ny + j) * g->nx + i;
}

/* Dirichlet value of domain face d next to cell (i,j,k) */
static double face_value(const or_grid* g, int d, int i, int j, int k) {
  if (!g->face_data) return g->bc_value[d];
  const long ax = (long)g->ny * g->nz, ay = (long)g->nx * g->nz;
  long base, q;
  if (d < 2) {
    base = d * ax;
    q = (long)k * g->ny + j;
  } else if (d < 4) {
    base = 2 * ax + (d - 2) * ay;
    q = (long)k * g->nx + i;
  } else {
    base = 2 * ax + 2 * ay + (long)(d - 4) * g->nx * g->ny;
    q = (long)j * g->nx + i;
  }
  return g->face_data[base + q];
}

/* Robin face of grid g: weight factor rho (diagonal 2 beta_c rho / h^2) */
static double robin_rho(const or_grid* g, int d) {
  const double ah2 = 0.5 * g->bc_value[d] * g->h;
  return ah2 / (1.0 + ah2);
}

static const int DI[6] = {-1, 1, 0, 0, 0, 0};
static const int DJ[6] = {0, 0, -1, 1, 0, 0};
static const int DK[6] = {0, 0, 0, 0, -1, 1};

/* Diagonal and off-diagonal sum of the operator row of free cell (i,j,k).
 * L(u)_c = diag*u_c - off.  With homog != 0 the domain Dirichlet values are
 * taken as zero (the correction equation on coarse grids). */
static void row(const or_grid* g, double alpha, const double* beta,
                const uint8_t* mask, const double* u, int i, int j, int k,
                int homog, double* diag_out, double* off_out) {
  long c = idx(g, i, j, k);
  double bc = beta ? beta[c] : 1.0;
  double ih2 = 1.0 / (g->h * g->h);
  double diag = alpha, off = 0.0;
  for (int d = 0; d < 6; ++d) {
    int ii = i + DI[d], jj = j + DJ[d], kk = k + DK[d];
    int inside = ii >= 0 && ii < g->nx && jj >= 0 && jj < g->ny && kk >= 0 && kk < g->nz;
    if (inside) {
      long n = idx(g, ii, jj, kk);
      double w;
      if (mask && mask[n]) {
        w = bc; /* Dirichlet at the electrode cell centre, distance h */
      } else {
        double bn = beta ? beta[n] : 1.0;
        w = 2.0 * bc * bn / (bc + bn);
      }
      diag += w * ih2;
      off += w * ih2 * u[n];
    } else if (g->bc_kind[d] == 0) {
      double w = 2.0 * bc; /* ghost = 2 g - u_c */
      diag += w * ih2;
      if (!homog) off += w * ih2 * face_value(g, d, i, j, k);
    } else if (g->bc_kind[d] == 2) {
      diag += 2.0 * bc * robin_rho(g, d) * ih2; /* ghost = u_c (1 - ah/2)/(1 + ah/2) */
    }
  }
  *diag_out = diag;
  *off_out = off;
}

/* r = f - L(u) on free cells, 0 on masked cells.  Returns sum r^2. */
double or_residual(const or_grid* g, double alpha, const double* beta,
                   const uint8_t* mask, const double* f, const double* u,
                   double* r, int homog) {
  double ss = 0.0;
#pragma omp parallel for reduction(+ : ss) schedule(static)
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        long c = idx(g, i, j, k);
        double rc = 0.0;
        if (!(mask && mask[c])) {
          double diag, off;
          row(g, alpha, beta, mask, u, i, j, k, homog, &diag, &off);
          rc = f[c] - (diag * u[c] - off);
        }
        if (r) r[c] = rc;
        ss += rc * rc;
      }
  return ss;
}

/* One red-black Gauss-Seidel half-sweep: updates free cells with
 * (i+j+k) % 2 == color.  Cells of one colour only couple to the other. */
void or_rbgs(const or_grid* g, double alpha, const double* beta,
             const uint8_t* mask, const double* f, double* u, int color, int homog) {
#pragma omp parallel for schedule(static)
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        if (((i + j + k) & 1) != color) continue;
        long c = idx(g, i, j, k);
        if (mask && mask[c]) continue;
        double diag, off;
        row(g, alpha, beta, mask, u, i, j, k, homog, &diag, &off);
        u[c] = (f[c] + off) / diag;
      }
}

/* Coarse rhs = average of the 8 fine children (masked children carry r = 0). */
void or_restrict(const or_grid* fg, const double* rf, const or_grid* cg, double* fc) {
#pragma omp parallel for schedule(static)
  for (int K = 0; K < cg->nz; ++K)
    for (int J = 0; J < cg->ny; ++J)
      for (int I = 0; I < cg->nx; ++I) {
        double s = 0.0;
        for (int c = 0; c < 8; ++c)
          s += rf[idx(fg, 2 * I + (c & 1), 2 * J + ((c >> 1) & 1), 2 * K + (c >> 2))];
        fc[idx(cg, I, J, K)] = 0.125 * s;
      }
}

/* Ghost factor of the homogeneous face condition of grid g: u_g = s u_c
 * with s = -1 (Dirichlet), +1 (Neumann), (1 - ah/2)/(1 + ah/2) (Robin). */
static double ghost_factor(const or_grid* g, int d) {
  if (g->bc_kind[d] == 0) return -1.0;
  if (g->bc_kind[d] == 1) return 1.0;
  return 1.0 - 2.0 * robin_rho(g, d);
}

/* Coarse correction value at a possibly out-of-box coarse index: the ghost
 * of the homogeneous face condition (ghost_factor times the cell inside);
 * masked coarse cells hold a zero correction. */
static double coarse_val(const or_grid* cg, const uint8_t* cmask, const double* ec,
                         int I, int J, int K) {
  double s = 1.0;
  if (I < 0) { I = 0; s *= ghost_factor(cg, 0); }
  if (I >= cg->nx) { I = cg->nx - 1; s *= ghost_factor(cg, 1); }
  if (J < 0) { J = 0; s *= ghost_factor(cg, 2); }
  if (J >= cg->ny) { J = cg->ny - 1; s *= ghost_factor(cg, 3); }
  if (K < 0) { K = 0; s *= ghost_factor(cg, 4); }
  if (K >= cg->nz) { K = cg->nz - 1; s *= ghost_factor(cg, 5); }
  long c = idx(cg, I, J, K);
  if (cmask && cmask[c]) return 0.0;
  return s * ec[c];
}

/* u_fine += trilinear interpolation of the coarse correction (weights
 * 3/4 and 1/4 per axis, i.e. 27, 9, 3, 1 over 64); masked fine cells are
 * left alone. */
void or_prolong_add(const or_grid* cg, const uint8_t* cmask, const double* ec,
                    const or_grid* fg, const uint8_t* fmask, double* uf) {
#pragma omp parallel for schedule(static)
  for (int k = 0; k < fg->nz; ++k)
    for (int j = 0; j < fg->ny; ++j)
      for (int i = 0; i < fg->nx; ++i) {
        long c = idx(fg, i, j, k);
        if (fmask && fmask[c]) continue;
        int I = i / 2, J = j / 2, K = k / 2;
        int si = (i & 1) ? 1 : -1, sj = (j & 1) ? 1 : -1, sk = (k & 1) ? 1 : -1;
        double v = 0.0;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b)
            for (int cc = 0; cc < 2; ++cc) {
              double w = (a ? 0.25 : 0.75) * (b ? 0.25 : 0.75) * (cc ? 0.25 : 0.75);
              v += w * coarse_val(cg, cmask, ec, I + a * si, J + b * sj, K + cc * sk);
            }
        uf[c] += v;
      }
}

/* Coarse beta and mask: masked iff at least 3 of the 8 children are masked;
 * beta = mean of the free children's beta. */
void or_coarsen(const or_grid* fg, const double* bf, const uint8_t* mf,
                const or_grid* cg, double* bcoarse, uint8_t* mcoarse) {
  for (int K = 0; K < cg->nz; ++K)
    for (int J = 0; J < cg->ny; ++J)
      for (int I = 0; I < cg->nx; ++I) {
        double s = 0.0;
        int nfree = 0;
        for (int c = 0; c < 8; ++c) {
          long n = idx(fg, 2 * I + (c & 1), 2 * J + ((c >> 1) & 1), 2 * K + (c >> 2));
          if (mf && mf[n]) continue;
          s += bf ? bf[n] : 1.0;
          ++nfree;
        }
        long C = idx(cg, I, J, K);
        if (mcoarse) mcoarse[C] = 8 - nfree >= 3;
        if (bcoarse) bcoarse[C] = nfree ? s / nfree : 1.0;
      }
}

/* ---- dense Cholesky for the coarsest grid ---------------------------- */

typedef struct {
  int n;        /* free unknowns */
  long* cells;  /* free cell index of each unknown */
  double* L;    /* n x n lower Cholesky factor, row major */
} or_dense;

static int dense_build(const or_grid* g, double alpha, const double* beta,
                       const uint8_t* mask, or_dense* D) {
  long nc = ncell(g);
  long* cells = (long*)malloc(sizeof(long) * nc);
  long* pos = (long*)malloc(sizeof(long) * nc);
  int n = 0;
  for (long c = 0; c < nc; ++c) {
    pos[c] = -1;
    if (!(mask && mask[c])) { pos[c] = n; cells[n++] = c; }
  }
  double* M = (double*)calloc((size_t)n * n, sizeof(double));
  double* e = (double*)calloc(nc, sizeof(double));
  /* column j of the matrix = homogeneous operator applied to unit vector j */
  for (int col = 0; col < n; ++col) {
    e[cells[col]] = 1.0;
    for (int k = 0; k < g->nz; ++k)
      for (int j = 0; j < g->ny; ++j)
        for (int i = 0; i < g->nx; ++i) {
          long c = idx(g, i, j, k);
          if (pos[c] < 0) continue;
          /* only rows that touch the unit entry are nonzero */
          double diag, off;
          row(g, alpha, beta, mask, e, i, j, k, 1, &diag, &off);
          double v = diag * e[c] - off;
          if (v != 0.0) M[(size_t)pos[c] * n + col] = v;
        }
    e[cells[col]] = 0.0;
  }
  free(e);
  /* in-place Cholesky M = L L^T (lower triangle) */
  for (int j = 0; j < n; ++j) {
    double d = M[(size_t)j * n + j];
    for (int p = 0; p < j; ++p) d -= M[(size_t)j * n + p] * M[(size_t)j * n + p];
    if (!(d > 0.0)) { free(M); free(cells); free(pos); return -1; }
    d = sqrt(d);
    M[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = M[(size_t)i * n + j];
      for (int p = 0; p < j; ++p) s -= M[(size_t)i * n + p] * M[(size_t)j * n + p];
      M[(size_t)i * n + j] = s / d;
    }
  }
  free(pos);
  D->n = n;
  D->cells = cells;
  D->L = M;
  return 0;
}

static void dense_solve(const or_dense* D, const double* f, double* u) {
  int n = D->n;
  double* y = (double*)malloc(sizeof(double) * (n ? n : 1));
  for (int i = 0; i < n; ++i) {
    double s = f[D->cells[i]];
    for (int p = 0; p < i; ++p) s -= D->L[(size_t)i * n + p] * y[p];
    y[i] = s / D->L[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = y[i];
    for (int p = i + 1; p < n; ++p) s -= D->L[(size_t)p * n + i] * y[p];
    y[i] = s / D->L[(size_t)i * n + i];
  }
  for (int i = 0; i < n; ++i) u[D->cells[i]] = y[i];
  free(y);
}

/* ---- multigrid hierarchy --------------------------------------------- */

typedef struct {
  int nlev;
  or_grid g[OR_MAX_LEVELS];
  double* beta[OR_MAX_LEVELS];
  uint8_t* mask[OR_MAX_LEVELS];
  double* f[OR_MAX_LEVELS];
  double* u[OR_MAX_LEVELS];
  double* r[OR_MAX_LEVELS];
  or_dense coarse;
} or_mg;

/* Coarsen while every dimension is even and at least 8 (so the coarsest
 * grid has every side >= 4 or odd). */
static int can_coarsen(const or_grid* g) {
  return g->nx % 2 == 0 && g->ny % 2 == 0 && g->nz % 2 == 0 && g->nx >= 8 &&
         g->ny >= 8 && g->nz >= 8;
}

static void mg_free(or_mg* M) {
  for (int l = 0; l < M->nlev; ++l) {
    if (l > 0) { free(M->beta[l]); free(M->mask[l]); free(M->f[l]); free(M->u[l]); }
    free(M->r[l]);
  }
  free(M->coarse.cells);
  free(M->coarse.L);
}

static int mg_build(or_mg* M, const or_grid* g, double alpha, const double* beta,
                    const uint8_t* mask) {
  memset(M, 0, sizeof(*M));
  M->g[0] = *g;
  M->beta[0] = (double*)beta;
  M->mask[0] = (uint8_t*)mask;
  M->r[0] = (double*)malloc(sizeof(double) * ncell(g));
  int l = 0;
  while (can_coarsen(&M->g[l]) && l + 1 < OR_MAX_LEVELS) {
    or_grid cg = M->g[l];
    cg.nx /= 2; cg.ny /= 2; cg.nz /= 2;
    cg.h *= 2.0;
    /* corrections are homogeneous: Dirichlet values 0; a Robin face keeps
     * its coefficient */
    for (int d = 0; d < 6; ++d)
      if (cg.bc_kind[d] != 2) cg.bc_value[d] = 0.0;
    cg.face_data = NULL;
    long nc = ncell(&cg);
    M->g[l + 1] = cg;
    M->beta[l + 1] = (double*)malloc(sizeof(double) * nc);
    M->mask[l + 1] = (uint8_t*)malloc(nc);
    or_coarsen(&M->g[l], M->beta[l], M->mask[l], &cg, M->beta[l + 1], M->mask[l + 1]);
    M->f[l + 1] = (double*)malloc(sizeof(double) * nc);
    M->u[l + 1] = (double*)malloc(sizeof(double) * nc);
    M->r[l + 1] = (double*)malloc(sizeof(double) * nc);
    ++l;
  }
  M->nlev = l + 1;
  if (dense_build(&M->g[l], alpha, M->beta[l], M->mask[l], &M->coarse) != 0) {
    mg_free(M);
    return -1;
  }
  return 0;
}

static void vcycle(or_mg* M, int l, double alpha, int nu1, int nu2) {
  const or_grid* g = &M->g[l];
  int homog = l > 0;
  if (l == M->nlev - 1) {
    /* exact solve of the correction equation A e = f - L(u), u += e */
    long n = ncell(g);
    or_residual(g, alpha, M->beta[l], M->mask[l], M->f[l], M->u[l], M->r[l], homog);
    double* e = (double*)calloc(n, sizeof(double));
    dense_solve(&M->coarse, M->r[l], e);
    for (long c = 0; c < n; ++c) M->u[l][c] += e[c];
    free(e);
    return;
  }
  for (int s = 0; s < nu1; ++s) {
    or_rbgs(g, alpha, M->beta[l], M->mask[l], M->f[l], M->u[l], 0, homog);
    or_rbgs(g, alpha, M->beta[l], M->mask[l], M->f[l], M->u[l], 1, homog);
  }
  or_residual(g, alpha, M->beta[l], M->mask[l], M->f[l], M->u[l], M->r[l], homog);
  or_restrict(g, M->r[l], &M->g[l + 1], M->f[l + 1]);
  memset(M->u[l + 1], 0, sizeof(double) * ncell(&M->g[l + 1]));
  vcycle(M, l + 1, alpha, nu1, nu2);
  or_prolong_add(&M->g[l + 1], M->mask[l + 1], M->u[l + 1], g, M->mask[l], M->u[l]);
  for (int s = 0; s < nu2; ++s) {
    or_rbgs(g, alpha, M->beta[l], M->mask[l], M->f[l], M->u[l], 0, homog);
    or_rbgs(g, alpha, M->beta[l], M->mask[l], M->f[l], M->u[l], 1, homog);
  }
}

/* Norm of the right-hand side including boundary lifts: the residual of the
 * zero guess (free cells 0, electrode cells keep their values in u). */
double or_rhs_norm(const or_grid* g, double alpha, const double* beta,
                   const uint8_t* mask, const double* f, const double* u) {
  long n = ncell(g);
  double* z = (double*)malloc(sizeof(double) * n);
  for (long c = 0; c < n; ++c) z[c] = (mask && mask[c]) ? u[c] : 0.0;
  double ss = or_residual(g, alpha, beta, mask, f, z, NULL, 0);
  free(z);
  return sqrt(ss);
}

/* Solve L(u) = f by V(nu1,nu2)-cycles from the guess in u (electrode cells of
 * u carry their fixed values and are not changed).  Stops when
 * ||r||/||b|| <= tol, when the residual stops decreasing (round-off floor),
 * or after max_cycles.  hist (length >= max_cycles+1, nullable) receives the
 * relative residual before each cycle and after the last.
 * Returns the number of cycles, or -1 if the coarse factorisation failed. */
int or_solve(const or_grid* g, double alpha, const double* beta, const uint8_t* mask,
             const double* f, double* u, double tol, int max_cycles, int nu1, int nu2,
             double* hist, double* rel_out) {
  or_mg M;
  if (mg_build(&M, g, alpha, beta, mask) != 0) return -1;
  M.f[0] = (double*)f;
  M.u[0] = u;
  double bnorm = or_rhs_norm(g, alpha, beta, mask, f, u);
  if (bnorm == 0.0) bnorm = 1.0;
  double rel = sqrt(or_residual(g, alpha, beta, mask, f, u, NULL, 0)) / bnorm;
  if (hist) hist[0] = rel;
  int cyc = 0;
  int stalls = 0;
  while (cyc < max_cycles && rel > tol) {
    vcycle(&M, 0, alpha, nu1, nu2);
    ++cyc;
    double nrel = sqrt(or_residual(g, alpha, beta, mask, f, u, NULL, 0)) / bnorm;
    if (hist) hist[cyc] = nrel;
    /* round-off floor: three cycles in a row without a 1% reduction */
    stalls = nrel > 0.99 * rel ? stalls + 1 : 0;
    rel = nrel;
    if (stalls >= 3) break;
  }
  if (rel_out) *rel_out = rel;
  mg_free(&M);
  return cyc;
}

/* Homogeneous-or-not operator application used by tests to assemble small
 * matrices: out = L(u) on free cells, 0 on masked cells. */
void or_apply(const or_grid* g, double alpha, const double* beta, const uint8_t* mask,
              const double* u, double* out, int homog) {
  long n = ncell(g);
  double* z = (double*)calloc(n, sizeof(double));
  or_residual(g, alpha, beta, mask, z, u, out, homog);
  for (long c = 0; c < n; ++c) out[c] = -out[c];
  free(z);
}

/* Number of multigrid levels the oracle builds for a grid (for tests). */
int or_num_levels(const or_grid* g) {
  or_grid c = *g;
  int l = 1;
  while (can_coarsen(&c) && l < OR_MAX_LEVELS) {
    c.nx /= 2; c.ny /= 2; c.nz /= 2;
    ++l;
  }
  return l;
}
