// Internal declarations of libmg: operator views handed to the kernels and
// the launch wrappers.  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace mg {

// Message returned by mg_last_error() on the calling thread.
void set_last_error(const std::string& msg);

// Process-wide count of kernel launches issued by the launch wrappers.
long long launch_count();
void add_launches(long long k);

// Face order -x,+x,-y,+y,-z,+z.
struct Box {
  int nx, ny, nz;
  __host__ __device__ long long n() const { return (long long)nx * ny * nz; }
};

// Packed per-face data of a box: faces -x, +x (ny*nz each, index k*ny + j),
// -y, +y (nx*nz, index k*nx + i), -z, +z (nx*ny, index j*nx + i).
__host__ __device__ inline long long face_offset(const Box& b, int f) {
  const long long ax = (long long)b.ny * b.nz, ay = (long long)b.nx * b.nz,
                  az = (long long)b.nx * b.ny;
  const long long off[6] = {0, ax, 2 * ax, 2 * ax + ay, 2 * ax + 2 * ay, 2 * ax + 2 * ay + az};
  return off[f];
}
// Entries of the packed face data of a box (2 (ny nz + nx nz + nx ny)).
__host__ __device__ inline long long face_count(const Box& b) {
  return face_offset(b, 5) + (long long)b.nx * b.ny;
}

// Small fixed arrays passed to kernels by value.
struct Dir6 {
  uint8_t d[6];
};
struct Val6 {
  double v[6];
};

// FP64 view of the level operator
//   (A u)_c = (alpha + D_c) u_c - sum_{free in-box nb} w_f u_nb
// with w_f already divided by h^2.  cx[c] holds the weight of the face
// between c and c - e_x (likewise cy, cz); D_c is the sum of all six face
// weights of c, including Dirichlet domain faces (2 beta_c / h^2) and faces
// towards electrode cells (beta_c / h^2); D_c < 0 marks an electrode cell.
// With cx == nullptr the operator has beta = 1: interior weights ih2, domain
// Dirichlet faces 2 ih2, and electrode cells come from `mask`.
struct Op64 {
  const double* cx;
  const double* cy;
  const double* cz;
  const double* D;
  // the same four level-0 arrays as double-floats (hi, lo) for the
  // refinement step (nullable: beta = 1)
  const float2* cxd;
  const float2* cyd;
  const float2* czd;
  const float2* Dd;
  const uint8_t* mask;
  Box b;
  double ih2;
  // per domain face (-x,+x,-y,+y,-z,+z): the face adds 2 beta_c rho / h^2 to
  // the diagonal and its homogeneous ghost is (1 - 2 rho) u_c: rho = 1
  // Dirichlet, 0 Neumann, (ah/2)/(1 + ah/2) Robin n.grad u + a u = 0
  double rho[6];
};

// FP32 view of a level in red/black split storage: colour c = (i+j+k)&1,
// packed row width W = (nx+1)/2, cell (i,j,k) at ((k*ny + j)*W + (i>>1)) of
// colour c.  beta[c] (nullable => beta = 1 everywhere, no electrode cells)
// holds the cell coefficient, with beta < 0 marking an electrode cell.
struct Split32 {
  const float* beta[2];
  Box b;
  int W;
  float ih2;
  float rho[6];  // face factors as in Op64 (this level's h)
  // Face-rule coarse levels (see mg_faces32.cu; dg[0] == nullptr otherwise):
  // per colour, the weights (already / h^2) of the faces towards -x, -y, -z
  // and the diagonal (sum of all six, < 0 on electrode cells).
  const float* fx[2];
  const float* fy[2];
  const float* fz[2];
  const float* dg[2];
};

// A stack of nb > 1 constant-coefficient problems on one grid (the stacked
// V-cycle of the Helmholtz problems): with it a Split32 level holds the
// problems one after another along z, b.nz = nb nzp; problem q owns planes
// [q nzp, (q+1) nzp) of every array, has its own alpha pa[q] and takes part
// only while bit q of `active` is set.  Its domain faces at z are those of
// its own planes; nzp is even on every level, so that a cell's colour is the
// same counted in its problem or in the stack.  (Kept out of Split32: a
// larger Split32 changed the register allocation, and the speed, of the
// one-problem kernels.)
struct Stk32 {
  int nb;
  int nzp;
  float pa[4];
  unsigned active;
};

constexpr int kMaxStack = 4;  // problems in one stacked V-cycle

struct Ptr2 {
  const float* p[2];
};
struct MPtr2 {
  float* p[2];
};

// Arguments of the fused refinement step (see mg_ir.cu).  The right-hand
// side comes as a double-float array (bdf), an FP64 array (rhs) or is formed
// on the fly from rhs * rhs_scale + lifts; the iterate comes as a
// double-float array (udf_in, plus the FP32 correction e) or as an FP64 array
// (u_in, split on load).
struct IrArgs {
  Op64 op;
  double alpha;
  const float2* bdf;   // b as double-floats (used when non-null)
  const double* rhs;   // b (lift == 0) or rhs with the lifts added here
  double rhs_scale;
  int lift;            // add Dirichlet-face lifts 2 beta_c g / h^2
  const double* beta0; // natural FP64 beta for the lifts (nullable = 1)
  Val6 bval;           // Dirichlet face values
  float2* bdf_out;     // b written as double-floats (nullable)
  const float2* udf_in;  // double-float iterate (used when non-null)
  const double* u_in;    // FP64 iterate otherwise
  float2* udf_out;     // u + e as double-floats (nullable: not written)
  const float* e[2];   // split FP32 correction (nullable: zero)
  float* r[2];         // split FP32 residual out (nullable)
  int W;               // packed row width of e and r
  double* partial;     // per-CTA sums of r^2
  double* partial_z;   // nullable: per-CTA sums of the squared residual of
                       // the guess that is 0 on free cells (FP64 guess only)
  int zchunk;          // z planes per CTA column, 0: automatic (the launcher
                       // replaces it by the planes used)
  double in_scale;     // FP64 inputs (u_in, rhs) times this power of two on
                       // load (1: as they are)
  // set by the launcher: 1/h^2, -alpha and the interior beta = 1 diagonal
  // 6/h^2 + alpha as double-floats; alpha != 0
  float2 ih2d, nalpha, dint;
  int has_alpha;
  // beta = 1: what a -z / +z domain face changes in the diagonal,
  // (2 rho - 1) / h^2, as double-floats
  float2 dzm, dzp;
};

// ---- setup ---------------------------------------------------------------
// out = in as double-floats (hi = in rounded to FP32, lo = in - hi rounded)
void launch_split_df(const double* in, float2* out, long long n, cudaStream_t s);
// Face weights / h^2 of a level; domain face f adds 2 beta_c rho[f] / h^2 to
// the diagonal (rho as in Op64).
void launch_faces64(const double* beta, const uint8_t* mask, Box b, double ih2,
                    const double rho[6], double* cx, double* cy, double* cz, double* D,
                    cudaStream_t s);
void launch_coarsen(const double* beta_f, const uint8_t* mask_f, Box fb, double* beta_c,
                    uint8_t* mask_c, cudaStream_t s);
// Face weights and diagonal of coarse level cb (layout of launch_faces64) from
// the fine level's face weights: between free coarse cells the mean over the 4
// crossing fine lines of the (1/4, 1/2, 1/4) series of the 3 fine faces
// between the coarse centres; towards a coarse electrode cell and on domain
// faces the cell rule on the coarse coefficient beta_c and mask mask_c.
void launch_coarsen_faces64(const double* fcx, const double* fcy, const double* fcz, Box fb,
                            const double* beta_c, const uint8_t* mask_c, Box cb, double ih2c,
                            const double rho[6], double* cx, double* cy, double* cz, double* D,
                            cudaStream_t s);
void launch_assemble_dense(Op64 op, double alpha, double* M, cudaStream_t s);
void launch_gj_invert(double* M, int n, double* rowp, double* colp, cudaStream_t s);

// ---- solve ---------------------------------------------------------------
// b = f * scale + Dirichlet-face lifts (2 beta_c g / h^2); 0 on electrode cells.
// g = bval[face], or the packed per-face-cell values when faces != nullptr.
void launch_rhs64(const double* f, double scale, const double* beta, const uint8_t* mask,
                  Box b, double ih2, const uint8_t dir[6], const double bval[6],
                  const double* faces, double* out, cudaStream_t s);
// Dirichlet face data of a ratio-2 sub-box at parent cell offset (ox,oy,oz)
// by trilinear interpolation of the parent solution.
void launch_subbox_bc(const double* parent_u, Box pb, int ox, int oy, int oz, Box sb,
                      double* faces, cudaStream_t s);
// u[c] = value[c] (or 0 if value == nullptr) on electrode cells.
void launch_set_masked(const uint8_t* mask, const double* value, long long n, double* u,
                       cudaStream_t s);
// Red-black Gauss-Seidel half-sweep of colour (i+j+k)&1 == color.
void launch_rbgs64(const Op64& op, double alpha, const double* f, double* u, int color,
                   cudaStream_t s);

// r = f - A u averaged over 8 children into fc; uc (nullable) zeroed.
void launch_resid_restrict64(const Op64& op, double alpha, const double* f, const double* u,
                             double* fc, double* uc, cudaStream_t s);

// uf += trilinear prolongation of ec (coarse box = fine/2); electrode fine
// cells untouched.  Coarse ghosts: (1 - 2 cop.rho) times the cell inside.
void launch_prolong64(const Op64& fop, const Op64& cop, const double* ec, double* uf,
                      cudaStream_t s);

// Residual r = f - A u of the level (no restriction); returns nothing.
void launch_resid64(const Op64& op, double alpha, const double* f, const double* u, double* r,
                    cudaStream_t s);

// u += Minv r over all n cells of the coarsest level (Minv FP64, rows of
// electrode cells zero).
void launch_dense_apply64(const double* Minv, int n, const double* r, double* u, cudaStream_t s);


// FP64 norms of the residual of u (plain FP64 on the natural layout): per
// block the sums over free cells of (f - A u)^2 into part[0..nblk) and of
// the zero guess's residual (electrode values kept) into part[nblk..2 nblk);
// nblk = resid_norms_blocks(b, capacity of each half).
int resid_norms_blocks(const Box& b, int cap);
void launch_resid_norms64(const Op64& op, double alpha, const double* f, const double* u,
                          double* part, int nblk, cudaStream_t s);

// sum of partial[0..n) into *out (single block, fixed order); out may be the
// device-side address of mapped pinned host memory.
void launch_sum_partials(const double* partial, int n, double* out, cudaStream_t s);

// ---- FP32 split-storage inner V-cycle (mg_split32.cu) -----------------------
// True (and cleared) if a staged half-sweep gave up waiting for a plane since
// the last call (synchronous read of a device flag).
bool sweep_timed_out();
// Sets the staged half-sweeps' shared-memory limits once; false if they
// cannot run (the register-fed half-sweep is used then).
bool sweep_kernels_ready();
// The same for the staged refinement step (mg_ir.cu).
bool ir_tma_ready();
bool ir_timed_out();
// zchunk: mg_options.sweep_zchunk (0 automatic, -1 register-fed only, or the
// staged form's z planes per CTA).
// stk: a stack of problems (op's planes span the stack; null: one problem).
void launch_half_sweep32(const Split32& op, float alpha, int col, const float* f, float* u,
                         const float* uo, bool zero_other, bool has_mask, int zchunk,
                         cudaStream_t s, const Stk32* stk = nullptr);
// Residual of the red cells only (needs nu1 >= 1: black residuals are 0).
// stk (nullable): the fine level's stack (its nzp; the coarse level has half)
void launch_resid_restrict32s(const Split32& op, const Split32& cop, float alpha, Ptr2 f, Ptr2 u,
                              MPtr2 fc, MPtr2 uc, cudaStream_t s, const Stk32* stk = nullptr);
// Corrects black cells only (needs nu2 >= 1: red cells are overwritten next).
void launch_prolong32s(const Split32& op, const Split32& cop, Ptr2 ec, MPtr2 u, cudaStream_t s,
                       const Stk32* stk = nullptr);
void launch_resid32s(const Split32& op, float alpha, Ptr2 f, Ptr2 u, MPtr2 r, cudaStream_t s);
void launch_dense_apply32s(const Split32& op, const double* Minv, Ptr2 r, MPtr2 u,
                           cudaStream_t s);
void launch_split_beta(const double* beta, const uint8_t* mask, const Split32& op, MPtr2 out,
                       cudaStream_t s);

// ---- face-rule coarse levels (mg_faces32.cu) ------------------------------
void launch_half_sweep32f(const Split32& op, float alpha, int col, const float* f, float* u,
                          const float* uo, bool zero_other, bool has_mask, cudaStream_t s);
void launch_resid_restrict32f(const Split32& op, const Split32& cop, float alpha, Ptr2 f, Ptr2 u,
                              MPtr2 fc, MPtr2 uc, cudaStream_t s);
void launch_resid32f(const Split32& op, float alpha, Ptr2 f, Ptr2 u, MPtr2 r, cudaStream_t s);
void launch_split_faces(const double* cx, const double* cy, const double* cz, const double* D,
                        Box b, int W, MPtr2 fx, MPtr2 fy, MPtr2 fz, MPtr2 dg, cudaStream_t s);

// ---- electric field and relaxation time (mg_efield.cu) --------------------
// E = -grad phi at cell centres (3 arrays of n, nullable) and, with J (3
// arrays of n) and dt_out (device double), min over free cells of
// eps0 |E| / |J| (+inf if J vanishes everywhere); min_bits is one device
// unsigned of scratch.  Grids need ny, nz <= 65535.
void launch_efield(const double* phi, const uint8_t* mask, Box b, double h, const uint8_t dir[6],
                   const double gval[6], const double* J, double* E, double eps0,
                   unsigned* min_bits, double* dt_out, cudaStream_t s);

// ---- fused refinement step (mg_ir.cu) --------------------------------------
// One pass: (u + e), r = b - A u, r -> FP32, per-CTA sums of r^2 (and of the
// squared residual of the zero guess when a.partial_z is set).
// Returns the thread blocks launched (= per-block partial sums written).
int launch_ir_fused(const IrArgs& a, cudaStream_t s);
// *flag (device address of mapped host memory) = 1.0 if any u[c] != 0.
void launch_nonzero(const double* u, long long n, double* flag, cudaStream_t s);
// The first pass for a zero guess on a grid without electrodes (pointwise:
// r = b); uses a.rhs, a.in_scale, a.bdf_out, a.udf_out, a.r, a.W, a.partial,
// a.partial_z; at most max_blocks blocks.  Returns the blocks launched.
int launch_first_zero(const IrArgs& a, int max_blocks, cudaStream_t s);
// out = (hi + lo) * scale in FP64 (the final iterate of a mixed-precision
// solve; scale a power of two); electrode cells (mask nonzero, nullable) are
// left as they are
void launch_df_to_f64(const float2* in, const uint8_t* mask, double* out, long long n,
                      double scale, cudaStream_t s);
// Most CTAs (= partial sums) the refinement pass can launch for z planes
// per CTA column zchunk (0: automatic), over its one- and two-cell kernels.
int ir_partials(const Box& b, int zchunk = 0);

// ---- composite AMR hierarchy (mg_amr.cu) ----------------------------------
// One box of a ratio-2 AMR hierarchy as the kernels see it.
struct AmrDev {
  Box b;
  int fo[3];            // level >= 1: footprint lower corner in the parent's cells
  int parent;           // index of the parent box, -1 for the base box
  int child0;           // first entry of this box's children in the child list
  double ih2;
  const double* u;      // iterate
  const double* beta;   // cell coefficient (nullable: 1)
  const double* ghost;  // level >= 1: coarse-fine ghost values, packed per face
  const uint8_t* cov;   // nullable (no children): 0 valid, k + 1 covered by child k
                        // (k < 254), 255 valid next to a covered cell
};

struct AmrResArgs {
  double alpha;
  // same-level face weights / h^2 as in Op64 (nullable: beta = 1, weight 1/h^2)
  const double* cx;
  const double* cy;
  const double* cz;
  const uint8_t* mask;  // electrode cells (base box only, nullable)
  double rho[6];        // base box: domain face factors (1 Dirichlet, 0 Neumann)
  const double* b;      // right-hand side with lifts
  double* r;            // composite residual (valid and electrode cells), or
  float* f32[2];        // (when f32[0] is set) its FP32 red/black split copy
  int W;                // packed row width of f32
  double* partial;      // nullable: per-block sums of r^2 over the valid cells
  double* partial_z;    // nullable: the same for the zero guess (electrode
                        // values kept)
  const unsigned* special;  // the box's valid boundary cells and the valid
  unsigned nspecial;        // cells next to a covered cell (general rows)
  // the interior rows in double-float arithmetic: the box's level-0 face
  // weights and diagonal as double-floats (nullable: beta = 1), 1/h^2,
  // 6/h^2 + alpha and -alpha as double-floats
  const float2* cxd;
  const float2* cyd;
  const float2* czd;
  const float2* Dd;
  float2 ih2d, dint, nalpha;
  int has_alpha;
};

// Ghost values of box q (level >= 1) from its own and its parent's iterate.
void launch_amr_ghost(const AmrDev* D, int q, const Box& b, double* ghost, cudaStream_t s);
// Composite residual of box q: the plain interior rows, then the listed
// special cells (grid-stride kernels, amr_resid_blocks(b, nspecial) partial
// sums in all); children's ghosts must be current.
void launch_amr_resid(const AmrDev* D, const int* child_list, int q, const Box& b,
                      const AmrResArgs& a, cudaStream_t s);
unsigned amr_resid_blocks(const Box& b, long long nspecial);
// dst (parent cells over the child's footprint fo) = mean of the 8 children;
// with dst0 set, into the parent's FP32 red/black split arrays (dst0, dst1,
// row width W) instead.
void launch_amr_average(const Box& cb, const int fo[3], const double* src, const Box& pb,
                        double* dst, float* dst0, float* dst1, int W, cudaStream_t s);
// FP32 red/black split copy of an FP64 field (packed row width W).
void launch_amr_split(const Box& b, int W, const double* r, float* f0, float* f1, cudaStream_t s);
// u += e on free cells (e split FP32 (e0, e1, width W) or FP64 e64); delta
// (nullable) = e.
void launch_amr_add(const Box& b, int W, const float* e0, const float* e1, const double* e64,
                    const uint8_t* mask, double* u, double* delta, cudaStream_t s);
// Child u += trilinear interpolation of the parent correction (as above);
// delta (nullable) = the increment.
void launch_amr_prolong(const Box& pb, int W, const float* e0, const float* e1, const double* e64,
                        const Box& cb, const int fo[3], double* u, double* delta, cudaStream_t s);

}  // namespace mg
