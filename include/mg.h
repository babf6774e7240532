/*
 * mg.h -- C ABI of libmg.so: GB300 (sm_103a) geometric multigrid for the two
 * elliptic equations of Marskar, "Adaptive multiscale methods for 3D streamer
 * discharges in air" (arXiv:1809.08857):
 *
 *   Poisson (Sec. 2, Eq. 2, with a cell-wise relative permittivity eps_r):
 *       -div(eps_r grad phi) = rho / eps0
 *   Radiative transfer in the Helmholtz form of Eq. 3, one photon group j:
 *       (kappa_j^2 - lap) Psi_j = S
 *
 * discretised with the second-order cell-centred finite-volume scheme of
 * Sec. 2, items (ii)-(iii), and solved with geometric multigrid and red-black
 * Gauss-Seidel smoothing (Sec. 2, item (ii)).
 *
 * Conventions shared by every entry point
 *  - Grid: nx*ny*nz cells of side h; arrays are contiguous, x fastest:
 *    index (k*ny + j)*nx + i.  Faces are numbered -x,+x,-y,+y,-z,+z.
 *  - Array arguments are DEVICE pointers owned by the caller, FP64, unless the
 *    comment says otherwise.  The library never frees them and keeps none of
 *    them after the call returns, except that mg_create copies eps_r, mask and
 *    mask_value into its own storage.
 *  - Work is enqueued on the context's CUDA stream (mg_create / mg_set_stream).
 *    A solve synchronises that stream because its convergence test reads the
 *    residual norm on the host; on return the outputs are complete.
 *  - Discretisation readings (the paper leaves these open):
 *      face between two free cells: harmonic mean of eps_r;
 *      face towards an electrode (masked) cell: the free cell's eps_r, with
 *        the electrode value held at the masked cell's centre;
 *      Dirichlet domain face with value g: ghost value 2g - u (distance h/2);
 *      Neumann domain face: homogeneous (zero flux).
 *  - Convergence: relative residual ||b - A u||_2 / ||b||_2 over free cells,
 *    where b holds rho/eps0 plus the boundary and electrode lifts, i.e. ||b||
 *    is the residual norm of the zero guess.
 *  - Every function returns an mg_status; no C++ exception crosses the ABI.
 *    On error, mg_last_error() gives a message for the calling thread.
 */
#ifndef MG_H
#define MG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_ctx mg_ctx; /* opaque, library-owned */

typedef enum {
  MG_OK = 0,
  MG_ERR_INVALID_ARG = 1,   /* bad pointer, size, option or boundary spec */
  MG_ERR_CUDA = 2,          /* a CUDA runtime call failed (see mg_last_error) */
  MG_ERR_OOM = 3,           /* device allocation failed */
  MG_ERR_NOT_CONVERGED = 4, /* max_cycles reached; outputs hold the last iterate */
  MG_ERR_NONFINITE = 5,     /* NaN/Inf in the input or the residual */
  MG_ERR_UNSUPPORTED = 6,   /* valid request this build does not implement */
  MG_ERR_DIVERGED = 7       /* the relative residual rose at each of the last
                               three cycles (steps, FAC iterations) and is over
                               twice what it was three cycles earlier; outputs
                               hold the last iterate */
} mg_status;

typedef enum { MG_BC_DIRICHLET = 0, MG_BC_NEUMANN = 1 } mg_bc_kind;

/* Uniform box: nx*ny*nz cells of side h, lower corner at origin. */
typedef struct {
  int nx, ny, nz;
  double h;
  double origin[3];
} mg_grid;

/* Boundary conditions of the Poisson problem, per face (-x,+x,-y,+y,-z,+z):
 * kind[f] is an mg_bc_kind; value[f] is the Dirichlet potential (ignored for
 * Neumann, which is homogeneous).  The Helmholtz problems use Psi = 0 on
 * electrode cells and, on every domain face, the condition chosen by
 * mg_options.rte_bc (the paper leaves it open, Sec. 2 (iii)). */
typedef struct {
  int kind[6];
  double value[6];
} mg_bc;

typedef enum { MG_PREC_FP64 = 0, MG_PREC_MIXED = 1 } mg_precision;

/* Boundary condition of the radiative-transfer (Helmholtz) problems on the
 * domain faces; the paper leaves it open (Sec. 2 item (iii)).
 *   MG_RTE_BC_DIRICHLET  Psi = 0 (free-space absorption).
 *   MG_RTE_BC_MARSHAK    the Marshak condition of the Eddington closure,
 *                        n.grad Psi + (3 kappa_p / 2) Psi = 0 for Eq. 3's
 *                        kappa_p, i.e. n.grad Psi + (sqrt(3)/2) kappa Psi = 0
 *                        in the Helmholtz form (kappa = sqrt(3) kappa_p);
 *                        discretised with the face value (u_c + u_g)/2 and
 *                        the normal derivative (u_g - u_c)/h. */
typedef enum { MG_RTE_BC_DIRICHLET = 0, MG_RTE_BC_MARSHAK = 1 } mg_rte_bc;

/* Coarse-grid operator of a variable-coefficient (eps_r) context.  The paper
 * names geometric multigrid (Sec. 2 item (ii)) without its coarse operators;
 * they shape the convergence rate, not the converged answer.
 *   MG_COARSE_FACE  each coarse face weight is built from the finer level's
 *                   face weights: on each of the 4 fine lines crossing the
 *                   coarse face, the 3 fine faces between the two coarse
 *                   centres in series (weights 1/4, 1/2, 1/4), the lines in
 *                   parallel (their mean); faces towards coarse electrode
 *                   cells and domain faces as MG_COARSE_CELL.
 *   MG_COARSE_CELL  a coarse cell's eps_r is the mean of its free children and
 *                   faces take the harmonic mean, as on the finest level. */
typedef enum { MG_COARSE_FACE = 0, MG_COARSE_CELL = 1 } mg_coarse_op;

/* Solver options.  Zero-initialised fields take the defaults shown. */
typedef struct {
  int nu1;          /* pre-smoothing red-black sweeps per level, >= 1 (0: default 2) */
  int nu2;          /* post-smoothing sweeps, >= 1 (0: default 2) */
  int max_cycles;   /* cap on V-cycles (FP64) or outer refinement steps (100) */
  int precision;    /* mg_precision: FP64 V-cycles, or FP32 V-cycles inside
                       iterative refinement whose residual b - A u is formed
                       from the FP64 data in double-float arithmetic (pairs
                       of FP32, 48 significant bits) (MG_PREC_FP64 = 0) */
  int inner_cycles; /* FP32 V-cycles per refinement step in mixed mode (1) */
  int concurrency;  /* mixed mode: problems of one call solved concurrently,
                       each on a library stream with its own work arrays (4, max 4) */
  int no_graphs;    /* mixed mode: 1 = launch kernels directly instead of
                       replaying each refinement step as a CUDA graph (0) */
  int rte_bc;       /* mg_rte_bc: domain faces of the Helmholtz problems
                       (MG_RTE_BC_DIRICHLET = 0); fixed at mg_create */
  int ir_zchunk;    /* mixed mode, tile of the refinement pass: z planes
                       marched by one CTA column, 0 (automatic: enough CTAs
                       for 8 waves of three per SM) or >= 16 (half as many
                       for the two-cell kernel of constant-coefficient
                       problems, whose CTAs span twice the columns);
                       mg_autotune picks it among {auto, 16, 32, 64, 128} (0) */
  int coarse_op;    /* mg_coarse_op of a context with eps_r (MG_COARSE_FACE =
                       0); fixed at mg_create */
  int fixed_cycles; /* mixed mode: 0 = from the second refinement step on, a
                       step whose measured contraction per V-cycle (taken 15 %
                       weaker) reaches tol in fewer than inner_cycles
                       V-cycles runs only that many; 1 = every step runs
                       inner_cycles (0) */
  int coarse_visits; /* cycles on the first coarse level per cycle of the
                       finest level: 0 or 1 (a V-cycle), 2 (two V-cycles
                       there: the rate of a W-cycle on a layered medium whose
                       interfaces cut the coarse cells, for about 20 % more
                       work per cycle) (0) */
  int sweep_zchunk; /* FP32 half-sweeps of levels with at least 256 cells
                       along x: z planes per CTA of the form whose planes
                       arrive in shared memory by tensor copies, 8, 16 or 32;
                       0 = automatic (the largest of them that still gives
                       about four CTAs per SM slot, and the register-fed form
                       where even 8 gives fewer than two); -1 = the
                       register-fed form on every level (0) */
  int stack;        /* mixed mode: 1 = the Helmholtz problems of one context
                       in one solve call (those of mg_solve_helmholtz_batch,
                       mg_solve_set, mg_solve_photoionization, or of one
                       context in mg_solve_batch) run their FP32 V-cycles
                       stacked along z, one launch per level step for all of
                       them, where the grid has no electrode cells, Dirichlet
                       radiative-transfer faces and an even number of planes
                       on every level; 0 = every problem its own V-cycles on
                       its own stream (0: measured faster at 512^3, where the
                       problems' concurrency already hides the coarse levels) */
} mg_options;

/* Per-solve statistics.  hist[c] is the relative residual after c cycles
 * (hist[0] = initial guess), for c < 64. */
typedef struct {
  int cycles;       /* V-cycles (FP64) or refinement steps (mixed) taken */
  int converged;    /* 1 if rel_resid <= tol */
  double rel_resid; /* final ||b - A u|| / ||b||: r in double-float (48-bit)
                       arithmetic from FP64 data; r^2 summed per thread in
                       FP32, across thread blocks in FP64 */
  double time_ms;   /* device time of the solve (CUDA events) */
  double hist[64];
  int vcycles;      /* V-cycles run: FP64 mode = cycles; mixed mode = the inner
                       V-cycles of all refinement steps; composite AMR solve =
                       FAC iterations x inner V-cycles (per box) */
  int diverged;     /* 1 if the solve stopped with MG_ERR_DIVERGED */
} mg_stats;

/* Fill *opt with the defaults. */
void mg_default_options(mg_options* opt);

/*
 * mg_create -- build the multigrid hierarchy for one grid.
 *   grid       box description (h > 0, every n >= 1).
 *   eps_r      device, nx*ny*nz FP64 relative permittivity (> 0) of each
 *              cell, or NULL for 1 everywhere.  Copied.
 *   mask       device, nx*ny*nz uint8: nonzero marks an electrode cell whose
 *              potential is fixed (Dirichlet at its centre), or NULL.  Copied.
 *   mask_value device, nx*ny*nz FP64 potential of each electrode cell (read
 *              where mask != 0), or NULL for 0.  Copied.
 *   bc         Poisson boundary conditions (see mg_bc).  At least one
 *              Dirichlet face or electrode cell is required for the Poisson
 *              problem to be nonsingular.
 *   opt        options, or NULL for defaults.
 *   cuda_stream  cudaStream_t to enqueue on (NULL = legacy default stream).
 *   out        receives the context; free it with mg_destroy.
 * Setup is the operator assembly of Sec. 2 items (ii)-(iii) (face
 * coefficients, coarse grids by 2x coarsening, coarsest-grid inverse).
 */
mg_status mg_create(const mg_grid* grid, const double* eps_r, const uint8_t* mask,
                    const double* mask_value, const mg_bc* bc, const mg_options* opt,
                    void* cuda_stream, mg_ctx** out);

/*
 * mg_solve_poisson -- solve Eq. 2: -div(eps_r grad phi) = rho/eps0.
 *   rho  device, nx*ny*nz FP64 space charge density (C/m^3).
 *   phi  device, nx*ny*nz FP64; in: initial guess, out: solution.  Electrode
 *        cells are overwritten with their mask values.
 *   tol  stop when the relative residual <= tol (e.g. 1e-10).
 *   stats  nullable; receives cycles, residual history and device time.
 * Returns MG_ERR_NOT_CONVERGED (phi holds the last iterate) if max_cycles is
 * reached, MG_ERR_DIVERGED (phi holds the last iterate) if the residual rose
 * over three cycles and doubled, MG_ERR_NONFINITE if the residual is NaN/Inf.
 * The other solve calls return the same three statuses.
 */
mg_status mg_solve_poisson(mg_ctx* ctx, const double* rho, double* phi, double tol,
                           mg_stats* stats);

/*
 * mg_solve_screened -- solve alpha u - div(beta grad u) = f with the
 * context's cell coefficient beta (the eps_r array given to mg_create, 1
 * where it was NULL), its electrode cells (u held at mask_value) and its
 * boundary conditions (Dirichlet values lifted into b, Neumann homogeneous),
 * discretised like Eq. 2 (Sec. 2 items (ii)-(iii)).  One factor
 * (I - mu L) n = g of the semi-implicit diffusion advance of Sec. 2.2 is
 * this problem with alpha = 1/mu, f = g/mu and beta the diffusion
 * coefficient; the TGA step of that section takes two of them.
 *   alpha  >= 0; with alpha = 0 the problem needs a Dirichlet face or an
 *          electrode cell to be nonsingular.
 *   f      device, nx*ny*nz FP64 right-hand side.
 *   u      device, nx*ny*nz FP64; in: guess, out: solution.
 *   tol, stats  as in mg_solve_poisson.
 */
mg_status mg_solve_screened(mg_ctx* ctx, double alpha, const double* f, double* u, double tol,
                            mg_stats* stats);

/*
 * mg_solve_helmholtz_batch -- the three radiative-transfer solves of Eq. 3 in
 * Helmholtz form, (kappa_j^2 - lap) Psi_j = S for j = 0, 1, 2, with Psi = 0 on
 * every domain face and on electrode cells.  The paper's form
 * kappa Psi - div(grad Psi / (3 kappa)) = eta/c maps onto it by multiplying by
 * 3 kappa (kappa_j here = sqrt(3) kappa_paper, S = 3 kappa eta / c).
 *   S      device, nx*ny*nz FP64 source shared by the three groups.
 *   psi    three device pointers, nx*ny*nz FP64 each; in: guess, out: solution.
 *   kappa  host, three inverse absorption lengths (1/length, > 0).
 *   tol    relative residual target per group.
 *   stats  nullable, host array of three.
 */
mg_status mg_solve_helmholtz_batch(mg_ctx* ctx, const double* S, double* const psi[3],
                                   const double kappa[3], double tol, mg_stats stats[3]);

/*
 * mg_solve_photoionization -- the three-term radiative-transfer solves of
 * Eq. 3 with a source amplitude per term: (kappa_j^2 - lap) Psi_j = A_j S,
 * j = 0, 1, 2.  In the paper's three-group photoionisation model each group
 * has its own amplitude and absorption coefficient and the photoionisation
 * source is the sum of the three solutions; the paper prints neither set of
 * coefficients, so both come from the caller.  Boundary conditions, kappa,
 * psi, tol and stats as in mg_solve_helmholtz_batch.
 *   amp    host, three finite amplitudes A_j (A_j = 1 is
 *          mg_solve_helmholtz_batch).
 */
mg_status mg_solve_photoionization(mg_ctx* ctx, const double* S, double* const psi[3],
                                   const double kappa[3], const double amp[3], double tol,
                                   mg_stats stats[3]);

/*
 * mg_solve_set -- the elliptic solves of one time step of the paper's scheme
 * (Sec. 2.2: the field update followed by the radiative-transfer update):
 * the Poisson problem of mg_solve_poisson and the three Helmholtz problems of
 * mg_solve_helmholtz_batch, in one call.  In mixed precision the four solves
 * run concurrently on library-owned streams (see mg_options.concurrency), so
 * the FP64-bound refinement steps of one problem overlap with the
 * memory-bound FP32 V-cycles of the others.  Arguments as in the two calls
 * above; stats (nullable) is an array of four: Poisson, then j = 0, 1, 2.
 */
mg_status mg_solve_set(mg_ctx* ctx, const double* rho, double* phi, const double* S,
                       double* const psi[3], const double kappa[3], double tol,
                       mg_stats stats[4]);

/*
 * mg_efield -- the electric field E = -grad phi at cell centres and the
 * dielectric relaxation time Delta t_E = eps0 |E| / |J| (the time scale of
 * Sec. 1 that sets the coarse step of the scheme, Sec. 3), minimised over
 * the free cells.
 *   phi  device, nx*ny*nz FP64 potential (electrode cells at their values,
 *        as mg_solve_poisson leaves them).
 *   J    device, 3*nx*ny*nz FP64 current density (A/m^2): the x, y and z
 *        components one after the other, each x fastest; NULL if dt is NULL.
 *   E    device, 3*nx*ny*nz FP64 output in the same layout (V per unit of h),
 *        or NULL.  Centred differences (phi(c-1) - phi(c+1)) / (2h) per axis;
 *        outside the box the face ghost of the context's bc (Dirichlet
 *        2g - phi_c, Neumann phi_c); a masked neighbour contributes its
 *        electrode value; electrode cells get E = 0.
 *   dt   host, receives min eps0 |E| / |J| in seconds over free cells with
 *        |J| > 0 (+inf if there is none), formed in FP32 (a time step needs
 *        no more); NULL to skip.  The call then synchronises the stream.
 * Enqueued on the context's stream.
 */
mg_status mg_efield(mg_ctx* ctx, const double* phi, const double* J, double* E, double* dt);

/* ---- batches of problems and refined sub-boxes -----------------------------
 *
 * Packed Dirichlet face data of an nx*ny*nz box: faces -x, +x (ny*nz values
 * each, index k*ny + j), then -y, +y (nx*nz, index k*nx + i), then -z, +z
 * (nx*ny, index j*nx + i): mg_face_count() = 2 (ny nz + nx nz + nx ny) FP64.
 * A value is the potential (or Psi) at the centre of that boundary face.
 */
long long mg_face_count(int nx, int ny, int nz);

typedef enum {
  MG_PROBLEM_POISSON = 0,   /* Eq. 2 on the ctx's coefficients and bc */
  MG_PROBLEM_HELMHOLTZ = 1, /* Eq. 3, one group (kappa) */
  MG_PROBLEM_SCREENED = 2   /* mg_solve_screened (alpha) */
} mg_problem_kind;

typedef struct {
  mg_ctx* ctx;          /* grid, coefficients and work arrays of this problem */
  int kind;             /* mg_problem_kind */
  double kappa;         /* Helmholtz only: inverse absorption length (> 0) */
  const double* rhs;    /* device: rho (Poisson, C/m^3), S (Helmholtz) or f
                           (screened) */
  const double* faces;  /* device packed Dirichlet face data (values on the
                           Dirichlet faces of the ctx's bc for Poisson and
                           screened; every face for Helmholtz), or NULL: the
                           ctx's bc values (Poisson, screened), zero
                           (Helmholtz) */
  double* u;            /* device in/out iterate; distinct for every problem */
  double alpha;         /* MG_PROBLEM_SCREENED only: alpha >= 0 */
} mg_problem;

/*
 * mg_solve_batch -- solve a batch of problems, possibly on different grids
 * (for instance the uneven refined sub-boxes of an AMR level, which stand in
 * for the paper's patch-based hierarchy of Sec. 4).  Every context must use
 * the same precision mode.  In mixed precision up to 16 problems run
 * concurrently (at most mg_options.concurrency per context, each on a library
 * stream with its own work arrays); FP64 mode solves them one after the
 * other.  stats (nullable) has nprob entries.  Returns the worst status.
 */
mg_status mg_solve_batch(const mg_problem* probs, int nprob, double tol, mg_stats* stats);

/*
 * mg_subbox_bc -- Dirichlet data for a refined sub-box (refinement ratio 2)
 * from the parent solution: trilinear interpolation of the parent's
 * cell-centred values at the centres of the sub-box's boundary faces.
 *   parent     context of the parent grid.
 *   parent_u   device, parent solution (parent grid size).
 *   origin     parent cell index of the sub-box's lower corner (x, y, z);
 *              the sub-box covers parent cells [origin, origin + dims/2).
 *   dims       sub-box size in fine cells (x, y, z), each even; the box must
 *              stay at least one parent cell away from every parent face.
 *   faces      device, mg_face_count(dims) FP64 values (output, packed).
 * Enqueued on the parent's stream.
 */
mg_status mg_subbox_bc(const mg_ctx* parent, const double* parent_u, const int origin[3],
                       const int dims[3], double* faces);

/* ---- composite AMR hierarchy ----------------------------------------------
 *
 * The paper solves its elliptic equations with second-order cell-centred
 * finite volumes on patch-based AMR grids (Sec. 2 items (ii)-(iii); nested
 * Berger-Rigoutsos patches in Secs. 3-4).  An mg_amr is a ratio-2 hierarchy:
 * the base box (level 0, the mg_grid) and refined boxes of level l >= 1 with
 * cells of size h / 2^l.  The composite problem is one linear system over the
 * valid cells (cells not covered by a box of the next level; electrode cells
 * excluded):
 *   - same-level faces, domain faces and electrodes as on a single grid;
 *   - a fine cell on the boundary of its box sees a ghost value across it,
 *     g = (8/15) cc + (2/3) u_1 - (1/5) u_2: the quadratic along the normal
 *     through the two fine cells inside and cc, the 2D quadratic (with mixed
 *     term) of the 3 x 3 parent cells around the parent cell C holding the
 *     ghost, at the ghost's offset; fine face flux hmean(beta_f, beta_C)
 *     (g - u_1) / h_f (hmean: harmonic mean);
 *   - a coarse cell next to a covered cell takes, through that face, the mean
 *     of the four fine fluxes (refluxing): the discretisation is conservative.
 * The paper does not print its coarse-fine treatment; this is the standard
 * conservative one (refluxing, quadratic coarse-fine interpolation).
 *
 * Solve: fast adaptive composite iteration.  Per iteration and per level l
 * (base first): the composite residual, an inner V-cycle solve on every box
 * of level l (the base box with its domain faces, a refined box with Robin
 * faces standing in for its coarse-fine ghosts), the correction added to the
 * box and interpolated (trilinear) into every box refining it.  The residual
 * is FP64; the corrections use the context precision (FP32 V-cycles in mixed
 * mode), which changes the rate, not the answer.
 *
 * Arrays are per box: index 0 the base box, index q >= 1 the refined box
 * boxes[q - 1]; each is device FP64, nx*ny*nz of that box, x fastest.
 */
typedef struct mg_amr mg_amr; /* opaque, library-owned */

typedef struct {
  int level; /* >= 1 */
  int lo[3]; /* lower corner (x, y, z) in cells of this level, counted from the
                domain's low corner; even */
  int n[3];  /* cells (x, y, z); even, >= 2; the box grid must coarsen to <= 4096
                cells (as in mg_create) */
} mg_amr_box;

/*
 * mg_amr_create -- build a composite hierarchy.
 *   base        level-0 grid (the domain).
 *   nbox, boxes the refined boxes (any order).  Rules, checked: the box's
 *               footprint on the level below (cells lo/2 .. (lo+n)/2), grown
 *               by one cell (two cells when that level is itself refined),
 *               lies inside one box of that level (its parent);
 *               it does not overlap the footprint of another box of the same
 *               level; on level 0 it holds no electrode cell.
 *   eps_r       NULL (coefficient 1 everywhere) or nbox + 1 device pointers
 *               (each nullable: 1 on that box), copied at create: the cell
 *               coefficient beta (relative permittivity of Eq. 2, diffusion
 *               coefficient of a screened problem).
 *   mask, mask_value  level-0 electrode cells and values (as mg_create).
 *   bc, opt, cuda_stream  as mg_create; opt.max_cycles caps the FAC
 *               iterations, opt.inner_cycles is the V-cycles per box per
 *               iteration; rte_bc must be MG_RTE_BC_DIRICHLET for Helmholtz.
 * Errors: MG_ERR_INVALID_ARG for a bad hierarchy (mg_last_error says which
 * rule), MG_ERR_UNSUPPORTED for a box grid that does not coarsen to 4096
 * cells (or a box of 2^31 cells or more) or more than 254 refined boxes inside
 * one box.  Synchronises.
 */
mg_status mg_amr_create(const mg_grid* base, int nbox, const mg_amr_box* boxes,
                        const double* const* eps_r, const uint8_t* mask,
                        const double* mask_value, const mg_bc* bc, const mg_options* opt,
                        void* cuda_stream, mg_amr** out);

/*
 * mg_amr_solve -- solve the composite problem to ||b - A u||_2 / ||b||_2 <=
 * tol over the valid cells (||b||: the residual of the zero guess with the
 * electrode values kept).
 *   kind   MG_PROBLEM_POISSON (rhs = rho, b = rho / eps0 + lifts, param
 *          unused), MG_PROBLEM_SCREENED (param = alpha >= 0, rhs = f) or
 *          MG_PROBLEM_HELMHOLTZ (param = kappa > 0, beta = 1, Psi = 0 on the
 *          domain faces and electrodes, rhs = S).
 *   rhs    nbox + 1 device arrays (valid cells are read).
 *   u      nbox + 1 device arrays, in: guess, out: solution on the valid
 *          cells, electrode values on electrode cells, the mean of the
 *          children on covered cells.
 * stats (nullable): cycles = FAC iterations, hist per iteration.
 * Synchronises once per iteration.
 */
mg_status mg_amr_solve(mg_amr* amr, int kind, double param, const double* const* rhs,
                       double* const* u, double tol, mg_stats* stats);

/*
 * mg_amr_residual -- r = b - A u of the composite problem (kind, param, rhs
 * as in mg_amr_solve; u holds the electrode values on electrode cells):
 * valid cells the composite residual, electrode cells 0, covered cells the
 * mean of their children's values.  norm (nullable, host): ||r||_2 over the
 * valid cells, which synchronises.
 */
mg_status mg_amr_residual(mg_amr* amr, int kind, double param, const double* const* rhs,
                          const double* const* u, double* const* r, double* norm);

void mg_amr_destroy(mg_amr* amr);

/* Replace the solver options of a context (precision is fixed at create). */
mg_status mg_set_options(mg_ctx* ctx, const mg_options* opt);

/*
 * mg_autotune -- pick the smoother sweeps (nu1, nu2) in {(1,1), (2,1), (2,2),
 * (3,3)} and, in mixed precision, the inner V-cycles per refinement step in
 * {1..4}, then for the best of those the tile of the refinement pass
 * (ir_zchunk in {auto, 16, 32, 64, 128}) and the z planes per CTA of the
 * staged half-sweep (sweep_zchunk in {auto, 16, 32}), by timing mg_solve_set on the
 * caller's problem (each candidate run twice from a zero guess, the faster
 * counts; candidates that do not reach tol are rejected).  The fastest is installed in the context and returned in
 * *best (*best_ms, nullable: its device time).  Allocates four scratch fields
 * for the duration of the call.  Arguments as in mg_solve_set.
 */
mg_status mg_autotune(mg_ctx* ctx, const double* rho, const double* S, const double kappa[3],
                      double tol, mg_options* best, double* best_ms);

/* ---- learned warm start ----------------------------------------------------
 *
 * A 3D U-Net (4 levels with 16/32/48/64 channels, two 3x3x3 convolutions
 * with ReLU per level, 2x average pooling, nearest 2x upsampling followed by a
 * 3x3x3 convolution, skip connections by concatenation, 1x1x1 head) predicts
 * the change of the potential between two time steps of the paper's scheme,
 * whose elliptic solves are re-done only every coarse step (Sec. 2.2), from
 * the new charge and the previous potential:
 *     phi_guess = phi_prev + U(rho_n * s_rho, phi_prev * s_phi) / s_out.
 * Activations and weights are BF16 with FP32 accumulation on the tensor
 * cores (tcgen05 MMAs into tensor memory, operands staged by tiled tensor
 * copies); FP32 master weights are trained with Adam.  The paper has
 * no network: this is the warm start of the solver, and multigrid corrects
 * its guess to the same tolerance, so it cannot change the answer.
 * Field arguments are device FP64 [n][d][h][w] (x fastest), d, h, w
 * multiples of 8.
 */
typedef struct mg_unet mg_unet;

/* New network with He-normal weights from the seed (the head starts at 0,
 * so an untrained network predicts phi_prev). */
mg_status mg_unet_create(unsigned long long seed, mg_unet** out);
void mg_unet_destroy(mg_unet* net);
/* Input / output scales (all > 0). */
mg_status mg_unet_set_scales(mg_unet* net, double s_rho, double s_phi, double s_out);
mg_status mg_unet_get_scales(const mg_unet* net, double scales[3]);
/* One training step on a batch of n crops: forward, MSE loss against
 * (phi - phi_prev) * s_out, backward, Adam (lr, beta = 0.9/0.999).  loss
 * (host, nullable) receives the batch loss before the update (synchronises). */
mg_status mg_unet_train_step(mg_unet* net, const double* rho, const double* phi_prev,
                             const double* phi, int n, int d, int h, int w, float lr, float* loss,
                             void* cuda_stream);
/* phi_guess = phi_prev + U(...) / s_out (asynchronous on the stream). */
mg_status mg_unet_predict(mg_unet* net, const double* rho, const double* phi_prev,
                          double* phi_guess, int n, int d, int h, int w, void* cuda_stream);
/* Loss and FP32 gradients of every parameter (no update), for checking;
 * host_grads has mg_unet_num_params entries in mg_unet_get_params order. */
mg_status mg_unet_grads(mg_unet* net, const double* rho, const double* phi_prev,
                        const double* phi, int n, int d, int h, int w, float* host_grads,
                        float* loss);
mg_status mg_unet_num_params(const mg_unet* net, long long* n);
/* FP32 master parameters to / from host memory, in a fixed order: every
 * conv's weights [Cout][27][Cin] then bias, in the order enc0a, enc0b, enc1a,
 * enc1b, enc2a, enc2b, enc3a, enc3b, then per level l = 0, 1, 2: up_l, dec_l_a,
 * dec_l_b; then the head's 16 weights and bias. */
mg_status mg_unet_get_params(const mg_unet* net, float* host);
mg_status mg_unet_set_params(mg_unet* net, const float* host);
/* Weights and scales to / from a versioned binary file. */
mg_status mg_unet_save(const mg_unet* net, const char* path);
mg_status mg_unet_load(mg_unet* net, const char* path);

/* Single 3x3x3 convolution (zero padding) on channels-last BF16 tensors, the
 * network's kernel exposed for tests: y = relu?(conv(concat(x1, x2)) + bias),
 * weights [cout][27][c1 + c2] BF16, c1 >= 16 and c2 multiples of 16, cout in
 * {16, 32, 48, 64, 96}; bias (FP32, nullable).  x1, x2 and w are read by the
 * tensor memory accelerator and must be 16-byte aligned (MG_ERR_INVALID_ARG
 * otherwise). */
mg_status mg_nn_conv3d(const void* x1, int c1, const void* x2, int c2, const void* w,
                       const float* bias, int relu, int cout, int n, int d, int h, int w_,
                       void* y, void* cuda_stream);
/* Self-check of the bounded waits of the tensor-core kernels: the same
 * convolution, except that the first chunk's shared-memory barrier expects
 * 16 bytes more than its copies deliver, so its wait cannot complete.  Every
 * wait of the kernel gives up after 50 ms (normally 2 s), the kernel waits
 * (bounded) for its copies and MMAs in flight, frees its tensor memory and
 * returns without writing y; the call synchronises the stream and returns
 * MG_ERR_CUDA ("a tensor-core completion wait gave up"), as a real stall
 * would be reported, and the context stays usable.  Returns MG_OK only if the
 * wait did not give up (a broken check). */
mg_status mg_nn_conv3d_stalled(const void* x1, int c1, const void* x2, int c2, const void* w,
                               const float* bias, int relu, int cout, int n, int d, int h,
                               int w_, void* y, void* cuda_stream);
/* Its weight gradient dW[co][t][ci] = sum_v dy[v][co] x[v + off(t)][ci] (FP32, overwritten)
 * and, when db is not NULL, the bias gradient db[co] = sum_v dy[v][co] (FP32, overwritten),
 * on the tensor cores (BF16 products, FP32 sums; the order of the sums varies
 * from run to run).  Same channel rules as mg_nn_conv3d; dy, x1 and x2 must be
 * 16-byte aligned. */
mg_status mg_nn_conv3d_wgrad(const void* dy, int cout, const void* x1, int c1, const void* x2,
                             int c2, int n, int d, int h, int w, float* dw, float* db,
                             void* cuda_stream);

/* Attach a network to a context (not owned; NULL detaches), or load one from
 * a file (owned by the context). */
mg_status mg_warmstart_attach(mg_ctx* ctx, mg_unet* net);
mg_status mg_warmstart_load(mg_ctx* ctx, const char* weights_path);
/* r = b - A phi (FP64, device arrays of the grid) for the Poisson problem of
 * rho (C/m^3): b = rho/eps0 + boundary lifts.  Electrode cells of phi are set
 * to their values first.  Enqueued on the context's stream. */
mg_status mg_poisson_residual(mg_ctx* ctx, const double* rho, double* phi, double* r);

/*
 * mg_residual_norms -- the norms of the stopping test of a solve, in plain
 * FP64 arithmetic on the natural layout (a check of an answer that does not
 * reuse the double-float refinement pass): norms[0] = ||b - A u||_2 and
 * norms[1] = ||b||_2 (the residual of the guess that is 0 on free cells and
 * keeps the electrode values), both over the free cells, for the problem of
 * the discretisation of Sec. 2 items (ii)-(iii) on the context's grid,
 * coefficients, electrodes and boundary conditions.
 *   kind   MG_PROBLEM_POISSON (Eq. 2, rhs = rho, b = rho/eps0 + lifts, param
 *          unused), MG_PROBLEM_HELMHOLTZ (Eq. 3, param = kappa > 0, rhs = S)
 *          or MG_PROBLEM_SCREENED (param = alpha >= 0, rhs = f).
 *   u      device, nx*ny*nz FP64 iterate whose electrode cells hold their
 *          values (as every solve leaves them).
 *   norms  host, two FP64 (output).
 * Uses the context's stream and work slot 0; synchronises.
 */
mg_status mg_residual_norms(mg_ctx* ctx, int kind, double param, const double* rhs,
                            const double* u, double norms[2]);

/*
 * mg_warmstart_predict -- guess for the Poisson solve of rho from the
 * previous potential.  The network is applied to the residual of the
 * previous potential, r = b_n - A phi_prev = A (phi_n - phi_prev) (its first
 * input channel), and phi_prev (second channel), giving the candidate
 * phi_prev + U(r s_rho, phi_prev s_phi) / s_out.  Plain multigrid judges it:
 * the candidate and phi_prev each get nu1 FP64 red-black Gauss-Seidel sweeps
 * (which remove the high-frequency part of the network's BF16 rounding), and
 * the smoothed candidate is the guess unless its FP64 residual ||b - A phi||
 * is larger than that of the smoothed phi_prev, which is then the guess.
 * *used_net (nullable) tells which.  Synchronises the context's stream.
 */
mg_status mg_warmstart_predict(mg_ctx* ctx, const double* rho, const double* phi_prev,
                               double* phi_guess, int* used_net);

/* ---- instrumentation ------------------------------------------------------
 * Kernel classes of the fine (finest-level) launches: red-black smoothing,
 * fused residual + restriction, prolongation + correction, the FP64
 * refinement residual (with the solution update), and everything on coarser
 * levels (coarse).  With profiling enabled every fine-level launch is
 * bracketed by CUDA events on the context's stream; `bytes` accumulates the
 * algorithmic bytes of each launch (each operand read once, each result
 * written once).  This is instrumentation of the solver, not part of the
 * method. */
typedef enum {
  MG_KCLASS_SMOOTH = 0,
  MG_KCLASS_RESTRICT = 1,
  MG_KCLASS_PROLONG = 2,
  MG_KCLASS_RESID64 = 3,
  MG_KCLASS_COARSE = 4,
  MG_KCLASS_COUNT = 5
} mg_kclass;

typedef struct {
  long long launches; /* kernel launches of this class */
  double ms;          /* summed event-timed duration (fine-level classes) */
  double bytes;       /* summed algorithmic bytes (fine-level classes) */
} mg_kprof;

/* Turn per-launch event timing on (1) or off (0); resets the counters. */
mg_status mg_profile_enable(mg_ctx* ctx, int enable);

/* Copy the per-class counters (MG_KCLASS_COUNT entries) into out; reset them
 * if reset != 0. */
mg_status mg_profile_read(mg_ctx* ctx, mg_kprof* out, int reset);

/* Process-wide number of kernel launches issued by libmg so far. */
long long mg_launch_count(void);

/*
 * mg_residual_norm_noalloc -- ||b - A u||_2 over free cells for a
 * constant-coefficient problem (beta = 1: the Helmholtz operator, or the
 * Poisson operator with eps_r = 1), computed without allocating any device
 * memory.  The paper has no counterpart; this is a service entry point for
 * callers that cannot call cudaMalloc during the call: codes whose device
 * memory is already owned by their own pool allocator, and time-stepping
 * loops that cannot take the device-wide synchronisation cudaMalloc/cudaFree
 * may cause.
 *   grid, bc   the box and its boundary conditions (Dirichlet values lift b).
 *   alpha      zeroth-order coefficient (0 for Poisson, kappa^2 for Helmholtz).
 *   rhs        device, nx*ny*nz FP64; b = rhs * rhs_scale + Dirichlet lifts
 *              (rhs_scale = 1/eps0 turns a charge density into rho/eps0).
 *   mask       device, nx*ny*nz uint8 electrode cells, or NULL.
 *   u          device, nx*ny*nz FP64 iterate (electrode cells hold their values).
 *   norm_out   device, one FP64: receives ||b - A u||_2.
 *   cuda_stream  stream to enqueue on (NULL = legacy default stream).
 * Work is enqueued and the call returns without synchronising.  Scratch: a
 * library-owned static device array of 16384 FP64 partial sums (128 KiB per
 * GPU, held until the process exits), one per thread block of the residual
 * kernel: ceil(nx/30) * ceil(ny/14) * (z-chunks of its automatic tile), which
 * the tile keeps at most max(ceil(nx/30) * ceil(ny/14), 10944).  So every
 * grid with ceil(nx/30) * ceil(ny/14) <= 16384 fits (every grid up to 2048 x
 * 2048 in x and y); nz and ceil(ny/14) must not exceed 65535.  Larger grids
 * are rejected with MG_ERR_UNSUPPORTED before anything is launched.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current, so make that first
 * call before capturing work into a CUDA graph on that device.  Every call
 * shares the array: calls that overlap on the GPU (other streams or host
 * threads) race and must be serialised by the caller.
 */
mg_status mg_residual_norm_noalloc(const mg_grid* grid, const mg_bc* bc, double alpha,
                                   const double* rhs, double rhs_scale, const uint8_t* mask,
                                   const double* u, double* norm_out, void* cuda_stream);

/* Rebind the context to another CUDA stream (cudaStream_t, NULL = legacy). */
mg_status mg_set_stream(mg_ctx* ctx, void* cuda_stream);

/* Number of multigrid levels and the dimensions of level l (for tests). */
mg_status mg_level_info(const mg_ctx* ctx, int level, int* nlevels, int dims[3]);

/* Free the context and all library-owned device memory.  NULL is a no-op. */
void mg_destroy(mg_ctx* ctx);

/* Static description of a status code. */
const char* mg_error_string(mg_status status);

/* Message of the last error raised on the calling thread ("" if none). */
const char* mg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MG_H */
