// Composite (AMR) kernels of libmg: coarse-fine ghost values, the composite
// residual with refluxing, averaging onto covered cells and the transfer of
// a box's correction to itself and to the boxes refining it.
//
// The paper solves its elliptic equations with second-order cell-centred
// finite volumes on patch-based AMR grids (Sec. 2 items (ii)-(iii); the
// Berger-Rigoutsos grids of Sec. 4).  It prints no coarse-fine treatment;
// the one built here is the standard conservative one for cell-centred AMR
// with refinement ratio 2:
//  * the ghost g of a fine cell f across the boundary of its box is the
//    quadratic along the face normal through u_f, the next cell inward u_f2
//    and a coarse value cc on the normal through the coarse cell C holding
//    the ghost: g = (8/15) cc + (2/3) u_f - (1/5) u_f2 (Lagrange weights of
//    the points h_f, -h_f/2, -3h_f/2 at h_f/2); cc is the 2D quadratic with
//    mixed term through the 3 x 3 cells of the parent around C in the face
//    plane, at the ghost's offset (+-1/4, +-1/4) parent cells;
//  * the fine face flux is hmean(beta_f, beta_C) (g - u_f) / h_f, and the
//    coarse cell next to a covered cell takes the mean of the four fine
//    fluxes through its face (refluxing), so every flux leaves one cell and
//    enters another exactly.
#include <algorithm>

#include "df.cuh"
#include "mg_internal.h"

namespace mg {

namespace {

constexpr int kT = 256;
constexpr int kResidBlocksMax = 152 * 8;  // grid of the residual pass (grid-stride)

inline unsigned blocks_for(long long n) { return (unsigned)((n + kT - 1) / kT); }

__device__ __forceinline__ long long lin(const Box& b, int i, int j, int k) {
  return ((long long)k * b.ny + j) * b.nx + i;
}

__device__ __forceinline__ long long lin3(const Box& b, const int* x) {
  return lin(b, x[0], x[1], x[2]);
}

__device__ __forceinline__ int dim(const Box& b, int a) { return a == 0 ? b.nx : a == 1 ? b.ny : b.nz; }

// Index of the boundary cell x within the packed data of face f.
__device__ __forceinline__ long long face_slot(const Box& b, int f, const int* x) {
  const int ax = f >> 1;
  const long long q = ax == 0   ? (long long)x[2] * b.ny + x[1]
                      : ax == 1 ? (long long)x[2] * b.nx + x[0]
                                : (long long)x[1] * b.nx + x[0];
  return face_offset(b, f) + q;
}

__device__ __forceinline__ double hmean(double a, double b) { return 2.0 * a * b / (a + b); }

__device__ __forceinline__ double coef(const double* beta, long long c) {
  return beta ? beta[c] : 1.0;
}

// Face-plane weight of the parent cell at offset (a, b) in {-1,0,1}^2 of the
// quadratic u_C + s1 d1 + s2 d2 + s1^2/2 d11 + s2^2/2 d22 + s1 s2 d12 (centred
// differences) at offset (s1, s2).
__device__ __forceinline__ double tangential_weight(int a, int b, double s1, double s2) {
  if (a == 0 && b == 0) return 1.0 - s1 * s1 - s2 * s2;
  if (b == 0) return 0.5 * s1 * a + 0.5 * s1 * s1;
  if (a == 0) return 0.5 * s2 * b + 0.5 * s2 * s2;
  return 0.25 * s1 * s2 * a * b;
}

constexpr double kWc = 8.0 / 15.0;  // coarse value
constexpr double kW1 = 2.0 / 3.0;   // first fine cell inward
constexpr double kW2 = -1.0 / 5.0;  // second fine cell inward
constexpr uint8_t kShell = 255;      // valid cell with a covered face neighbour

// One thread per boundary-face cell of box q: ghost value across that face.
__global__ void __launch_bounds__(kT) k_amr_ghost(const AmrDev* __restrict__ D, int q,
                                                   double* __restrict__ ghost) {
  const AmrDev B = D[q];
  const Box& b = B.b;
  const long long t = (long long)blockIdx.x * kT + threadIdx.x;
  if (t >= face_count(b)) return;
  int f = 0;
  while (f < 5 && t >= face_offset(b, f + 1)) ++f;
  const long long s = t - face_offset(b, f);
  const int ax = f >> 1, side = (f & 1) ? 1 : -1;
  const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;  // face-plane axes (increasing)
  int x[3];
  const int m1 = dim(b, t1);
  x[t1] = (int)(s % m1);
  x[t2] = (int)(s / m1);
  x[ax] = side < 0 ? 0 : dim(b, ax) - 1;
  const double u1 = B.u[lin3(b, x)];
  x[ax] -= side;
  const double u2 = B.u[lin3(b, x)];
  x[ax] += side;
  // parent cell C holding the ghost (parent-local), offsets of the ghost
  const AmrDev P = D[B.parent];
  int C[3];
  for (int a = 0; a < 3; ++a) C[a] = B.fo[a] + (x[a] >> 1);
  C[ax] = side < 0 ? B.fo[ax] - 1 : B.fo[ax] + dim(b, ax) / 2;
  const double s1 = (x[t1] & 1) ? 0.25 : -0.25;
  const double s2 = (x[t2] & 1) ? 0.25 : -0.25;
  double cc = 0.0;
#pragma unroll
  for (int a = -1; a <= 1; ++a)
#pragma unroll
    for (int bb = -1; bb <= 1; ++bb) {
      int y[3] = {C[0], C[1], C[2]};
      y[t1] += a;
      y[t2] += bb;
      cc += tangential_weight(a, bb, s1, s2) * P.u[lin3(P.b, y)];
    }
  ghost[t] = kWc * cc + kW1 * u1 + kW2 * u2;
}

// Block sum of v into *out (all threads participate).
__device__ __forceinline__ void block_sum(double v, double* out) {
  __shared__ double w[kT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < kT / 32 ? w[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) *out = v;
  }
}

// Output of the residual pass: FP64 natural, or (Split) the FP32 red/black
// split right-hand side of the box's correction solve.
template <bool Split>
__device__ __forceinline__ void store_r(const AmrResArgs& a, unsigned c, unsigned i, unsigned jk,
                                        unsigned j, unsigned k, double r) {
  if (Split)
    a.f32[(i + j + k) & 1][(size_t)jk * a.W + (i >> 1)] = (float)r;
  else
    a.r[c] = r;
}

// Contribution of face F of valid cell (i, j, k) to (A u)_c (acc) and to the
// zero-guess row (accz) on the general path: domain face, coarse-fine ghost,
// refluxed face next to a covered cell, or a same-level face.
template <int F>
__device__ __forceinline__ void face_general(const AmrDev* __restrict__ D,
                                             const int* __restrict__ child_list,
                                             const AmrDev* __restrict__ Bp, const AmrResArgs& a,
                                             int i, int j, int k, long long c, double uc,
                                             double bc, double& acc, double& accz) {
  constexpr int ax = F >> 1, side = (F & 1) ? 1 : -1;
  constexpr int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
  const Box b = Bp->b;
  const int x[3] = {i, j, k};
  const int dims[3] = {b.nx, b.ny, b.nz};
  const long long stride = ax == 0 ? 1 : ax == 1 ? (long long)b.nx : (long long)b.nx * b.ny;
  const double* cw = ax == 0 ? a.cx : ax == 1 ? a.cy : a.cz;
  const int xn = x[ax] + side;
  if (xn >= 0 && xn < dims[ax]) {
    const long long n = c + side * stride;
    const uint8_t kn = Bp->cov ? Bp->cov[n] : 0;
    if (kn != 0 && kn != kShell) {
      // refluxing: mean of the four fine fluxes through this face
      const AmrDev* __restrict__ Kp = D + child_list[Bp->child0 + kn - 1];
      const Box kb = Kp->b;
      const int kdims[3] = {kb.nx, kb.ny, kb.nz};
      constexpr int kf = side > 0 ? 2 * ax : 2 * ax + 1;  // the child's face
      double sum = 0.0;
#pragma unroll
      for (int d1 = 0; d1 < 2; ++d1)
#pragma unroll
        for (int d2 = 0; d2 < 2; ++d2) {
          int y[3];
          y[ax] = side > 0 ? 0 : kdims[ax] - 1;
          y[t1] = 2 * (x[t1] - Kp->fo[t1]) + d1;
          y[t2] = 2 * (x[t2] - Kp->fo[t2]) + d2;
          const long long fc = lin3(kb, y);
          const double g = Kp->ghost[face_slot(kb, kf, y)];
          const double w = (Kp->beta || Bp->beta) ? hmean(coef(Kp->beta, fc), bc) : 1.0;
          sum += w * (g - Kp->u[fc]);
        }
      acc += 0.5 * Bp->ih2 * sum;
    } else {
      // same-level face (the weight of the face between a cell and its lower
      // neighbour is stored at the cell)
      const double w = cw ? cw[side > 0 ? n : c] : Bp->ih2;
      const double un = Bp->u[n];
      acc += w * (uc - un);
      if (a.mask && a.mask[n]) accz -= w * un;
    }
  } else if (Bp->parent < 0) {
    // domain face: Dirichlet (value lifted into b) or Neumann
    acc += 2.0 * bc * a.rho[F] * Bp->ih2 * uc;
  } else {
    // coarse-fine face: the ghost
    const AmrDev* __restrict__ Pp = D + Bp->parent;
    int C[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) C[e] = Bp->fo[e] + (x[e] >> 1);
    C[ax] = side < 0 ? Bp->fo[ax] - 1 : Bp->fo[ax] + dims[ax] / 2;
    const double w = (Bp->beta || Pp->beta) ? hmean(bc, coef(Pp->beta, lin3(Pp->b, C))) : 1.0;
    acc += w * Bp->ih2 * (uc - Bp->ghost[face_slot(b, F, x)]);
  }
}

// (A u)_c of a boundary or shell cell (general path, out of line so that it
// does not weigh on the registers of the interior path); accz: the row of
// the zero guess (electrode neighbours only).
__device__ __noinline__ double general_row(const AmrDev* __restrict__ D,
                                           const int* __restrict__ child_list,
                                           const AmrDev* __restrict__ Bp, const AmrResArgs& a,
                                           int i, int j, int k, long long c, double uc,
                                           double* accz_out) {
  const double bc = coef(Bp->beta, c);
  double acc = a.alpha * uc, accz = 0.0;
  face_general<0>(D, child_list, Bp, a, i, j, k, c, uc, bc, acc, accz);
  face_general<1>(D, child_list, Bp, a, i, j, k, c, uc, bc, acc, accz);
  face_general<2>(D, child_list, Bp, a, i, j, k, c, uc, bc, acc, accz);
  face_general<3>(D, child_list, Bp, a, i, j, k, c, uc, bc, acc, accz);
  face_general<4>(D, child_list, Bp, a, i, j, k, c, uc, bc, acc, accz);
  face_general<5>(D, child_list, Bp, a, i, j, k, c, uc, bc, acc, accz);
  *accz_out = accz;
  return acc;
}

// Composite residual r = b - A u of the interior cells of box q (every
// neighbour in the box) that are valid and have no covered neighbour: the
// plain seven-point row.  Electrode cells get 0; covered and shell cells are
// left to k_amr_average and k_amr_resid_special.  Grid-stride; r^2 (and the
// zero-guess row's square) summed per block.
//
// The row is evaluated in double-float arithmetic (FP32 pairs, 48 bits)
// from the FP64 data, split on load on the integer pipe, with the box's
// double-float face weights and diagonal: GB300's FP64 pipe (about 2 DFMA
// per clock per SM) would otherwise bound the pass.  The error stays near
// 2^-48 of the largest term of the row, far below the 1e-10 tolerance.
template <bool Split>
__global__ void __launch_bounds__(kT) k_amr_resid_interior(const AmrDev* __restrict__ D, int q,
                                                           const __grid_constant__ AmrResArgs a) {
  using namespace df;
  const AmrDev* __restrict__ Bp = D + q;
  const int nx = Bp->b.nx, ny = Bp->b.ny, nz = Bp->b.nz;
  const unsigned mx = nx - 2, my = ny - 2;
  const unsigned m = mx * my * (unsigned)(nz - 2);
  const unsigned sy = nx, sz = (unsigned)nx * ny;
  const double* __restrict__ u = Bp->u;
  const uint8_t* __restrict__ cov = Bp->cov;
  float rr = 0.0f, rz = 0.0f;
  for (unsigned t = blockIdx.x * kT + threadIdx.x; t < m; t += gridDim.x * kT) {
    const unsigned i = t % mx + 1, t2 = t / mx;
    const unsigned j = t2 % my + 1, k = t2 / my + 1;
    const unsigned jk = k * ny + j;
    const unsigned c = jk * nx + i;
    if (cov && cov[c]) continue;
    if (a.mask && a.mask[c]) {
      store_r<Split>(a, c, i, jk, j, k, 0.0);
      continue;
    }
    const float2 uc = split_df(u[c]);
    const float2 uxm = split_df(u[c - 1]), uxp = split_df(u[c + 1]),
                 uym = split_df(u[c - sy]), uyp = split_df(u[c + sy]),
                 uzm = split_df(u[c - sz]), uzp = split_df(u[c + sz]);
    float2 wxm = a.ih2d, wxp = a.ih2d, wym = a.ih2d, wyp = a.ih2d, wzm = a.ih2d, wzp = a.ih2d;
    float2 dg = a.dint;  // beta = 1: 6/h^2 + alpha
    const float2 bb = split_df(a.b[c]);
    DfAcc acc{bb.x, bb.y};
    if (a.cxd) {
      wxm = a.cxd[c];
      wxp = a.cxd[c + 1];
      wym = a.cyd[c];
      wyp = a.cyd[c + sy];
      wzm = a.czd[c];
      wzp = a.czd[c + sz];
      dg = a.Dd[c];
      if (a.has_alpha) acc.add(a.nalpha, uc);
    }
    acc.add(make_float2(-dg.x, -dg.y), uc);
    acc.add(wxm, uxm);
    acc.add(wxp, uxp);
    acc.add(wym, uym);
    acc.add(wyp, uyp);
    acc.add(wzm, uzm);
    acc.add(wzp, uzp);
    if (Split)
      a.f32[(i + j + k) & 1][(size_t)jk * a.W + (i >> 1)] = acc.value();
    else
      a.r[c] = widen(acc.s) + widen(acc.e);
    const float rv = acc.value();
    rr = fmaf(rv, rv, rr);
    if (a.partial_z) {
      DfAcc az{bb.x, bb.y};
      if (a.mask) {
        if (a.mask[c - 1]) az.add(wxm, uxm);
        if (a.mask[c + 1]) az.add(wxp, uxp);
        if (a.mask[c - sy]) az.add(wym, uym);
        if (a.mask[c + sy]) az.add(wyp, uyp);
        if (a.mask[c - sz]) az.add(wzm, uzm);
        if (a.mask[c + sz]) az.add(wzp, uzp);
      }
      const float zv = az.value();
      rz = fmaf(zv, zv, rz);
    }
  }
  if (a.partial) block_sum((double)rr, a.partial + blockIdx.x);
  if (a.partial_z) block_sum((double)rz, a.partial_z + blockIdx.x);
}

// The same for the listed cells of box q (its valid boundary cells and the
// cells next to a covered cell): the general row with domain faces,
// coarse-fine ghosts and refluxed faces.
template <bool Split>
__global__ void __launch_bounds__(kT) k_amr_resid_special(const AmrDev* __restrict__ D,
                                                          const int* __restrict__ child_list,
                                                          int q, const __grid_constant__ AmrResArgs a) {
  const AmrDev* __restrict__ Bp = D + q;
  const int nx = Bp->b.nx, ny = Bp->b.ny;
  double rr = 0.0, rz = 0.0;
  for (unsigned t = blockIdx.x * kT + threadIdx.x; t < a.nspecial; t += gridDim.x * kT) {
    const unsigned c = a.special[t];
    const unsigned i = c % nx, jk = c / nx;
    const unsigned j = jk % ny, k = jk / ny;
    if (a.mask && a.mask[c]) {
      store_r<Split>(a, c, i, jk, j, k, 0.0);
      continue;
    }
    double accz;
    const double acc = general_row(D, child_list, Bp, a, i, j, k, c, Bp->u[c], &accz);
    const double bb = a.b[c];
    const double r = bb - acc;
    store_r<Split>(a, c, i, jk, j, k, r);
    rr = fma(r, r, rr);
    const double z = bb - accz;
    rz = fma(z, z, rz);
  }
  if (a.partial) block_sum(rr, a.partial + blockIdx.x);
  if (a.partial_z) block_sum(rz, a.partial_z + blockIdx.x);
}

// dst (parent box) = mean of the 8 children in src (child box) over the
// child's footprint; one thread per footprint cell.  With Split the parent's
// values go to its FP32 red/black split arrays (dst0, dst1, row width W).
template <bool Split>
__global__ void __launch_bounds__(kT) k_amr_average(Box cb, int fx, int fy, int fz,
                                                     const double* __restrict__ src, Box pb,
                                                     double* __restrict__ dst, float* dst0,
                                                     float* dst1, int W) {
  const Box fb{cb.nx / 2, cb.ny / 2, cb.nz / 2};
  const long long t = (long long)blockIdx.x * kT + threadIdx.x;
  if (t >= fb.n()) return;
  const int I = (int)(t % fb.nx);
  const long long JK = t / fb.nx;
  const int J = (int)(JK % fb.ny), K = (int)(JK / fb.ny);
  double s = 0.0;
  for (int dk = 0; dk < 2; ++dk)
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) s += src[lin(cb, 2 * I + di, 2 * J + dj, 2 * K + dk)];
  const int i = fx + I, j = fy + J, k = fz + K;
  if (Split)
    (((i + j + k) & 1) ? dst1 : dst0)[((long long)k * pb.ny + j) * W + (i >> 1)] =
        (float)(0.125 * s);
  else
    dst[lin(pb, i, j, k)] = 0.125 * s;
}

// FP32 red/black split copy of r: colour (i+j+k)&1, packed row width W.
__global__ void __launch_bounds__(kT) k_amr_split(Box b, int W, const double* __restrict__ r,
                                                   float* __restrict__ f0, float* __restrict__ f1) {
  const long long c = (long long)blockIdx.x * kT + threadIdx.x;
  if (c >= b.n()) return;
  const int i = (int)(c % b.nx);
  const long long jk = c / b.nx;
  const int j = (int)(jk % b.ny), k = (int)(jk / b.ny);
  const long long p = jk * W + (i >> 1);
  ((i + j + k) & 1 ? f1 : f0)[p] = (float)r[c];
}

// Value of a correction at cell (i, j, k): split FP32 or natural FP64.
struct CorrSrc {
  Box b;
  int W;
  const float* e[2];
  const double* e64;
  __device__ __forceinline__ double at(int i, int j, int k) const {
    if (e64) return e64[lin(b, i, j, k)];
    return (double)e[(i + j + k) & 1][((long long)k * b.ny + j) * W + (i >> 1)];
  }
};

// u += e on the free cells of a box; delta (nullable) = e.
__global__ void __launch_bounds__(kT) k_amr_add(CorrSrc e, const uint8_t* __restrict__ mask,
                                                 double* __restrict__ u, double* __restrict__ delta) {
  const Box& b = e.b;
  const long long c = (long long)blockIdx.x * kT + threadIdx.x;
  if (c >= b.n()) return;
  const int i = (int)(c % b.nx);
  const long long jk = c / b.nx;
  const int j = (int)(jk % b.ny), k = (int)(jk / b.ny);
  const double v = (mask && mask[c]) ? 0.0 : e.at(i, j, k);
  u[c] += v;
  if (delta) delta[c] = v;
}

// Child box cells: u += trilinear interpolation of the parent correction
// (cell-centred weights 3/4, 1/4 per axis towards the fine cell); delta
// (nullable) = that increment.
__global__ void __launch_bounds__(kT) k_amr_prolong(CorrSrc e, Box cb, int fx, int fy, int fz,
                                                     double* __restrict__ u,
                                                     double* __restrict__ delta) {
  const long long c = (long long)blockIdx.x * kT + threadIdx.x;
  if (c >= cb.n()) return;
  const int i = (int)(c % cb.nx);
  const long long jk = c / cb.nx;
  const int j = (int)(jk % cb.ny), k = (int)(jk / cb.ny);
  const int I = fx + (i >> 1), J = fy + (j >> 1), K = fz + (k >> 1);
  const int si = (i & 1) ? 1 : -1, sj = (j & 1) ? 1 : -1, sk = (k & 1) ? 1 : -1;
  double v = 0.0;
  for (int dk = 0; dk < 2; ++dk)
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) {
        const double w = (di ? 0.25 : 0.75) * (dj ? 0.25 : 0.75) * (dk ? 0.25 : 0.75);
        v += w * e.at(I + di * si, J + dj * sj, K + dk * sk);
      }
  u[c] += v;
  if (delta) delta[c] = v;
}

}  // namespace

void launch_amr_ghost(const AmrDev* D, int q, const Box& b, double* ghost, cudaStream_t s) {
  k_amr_ghost<<<blocks_for(face_count(b)), kT, 0, s>>>(D, q, ghost);
  add_launches(1);
}

static unsigned capped_blocks(long long n) {
  return (unsigned)std::min<long long>(blocks_for(n), kResidBlocksMax);
}

unsigned amr_resid_blocks(const Box& b, long long nspecial) {
  const long long m = (long long)std::max(b.nx - 2, 0) * std::max(b.ny - 2, 0) *
                      std::max(b.nz - 2, 0);
  return capped_blocks(m) + capped_blocks(nspecial);
}

void launch_amr_resid(const AmrDev* D, const int* child_list, int q, const Box& b,
                      const AmrResArgs& a, cudaStream_t s) {
  const long long m = (long long)std::max(b.nx - 2, 0) * std::max(b.ny - 2, 0) *
                      std::max(b.nz - 2, 0);
  const unsigned gi = capped_blocks(m), gs = capped_blocks(a.nspecial);
  AmrResArgs as = a;  // the list kernel's partial sums follow the interior ones
  if (a.partial) as.partial = a.partial + gi;
  if (a.partial_z) as.partial_z = a.partial_z + gi;
  if (gi) {
    if (a.f32[0])
      k_amr_resid_interior<true><<<gi, kT, 0, s>>>(D, q, a);
    else
      k_amr_resid_interior<false><<<gi, kT, 0, s>>>(D, q, a);
    add_launches(1);
  }
  if (gs) {
    if (a.f32[0])
      k_amr_resid_special<true><<<gs, kT, 0, s>>>(D, child_list, q, as);
    else
      k_amr_resid_special<false><<<gs, kT, 0, s>>>(D, child_list, q, as);
    add_launches(1);
  }
}

void launch_amr_average(const Box& cb, const int fo[3], const double* src, const Box& pb,
                        double* dst, float* dst0, float* dst1, int W, cudaStream_t s) {
  const Box fb{cb.nx / 2, cb.ny / 2, cb.nz / 2};
  if (dst0)
    k_amr_average<true><<<blocks_for(fb.n()), kT, 0, s>>>(cb, fo[0], fo[1], fo[2], src, pb,
                                                          nullptr, dst0, dst1, W);
  else
    k_amr_average<false><<<blocks_for(fb.n()), kT, 0, s>>>(cb, fo[0], fo[1], fo[2], src, pb,
                                                           dst, nullptr, nullptr, 0);
  add_launches(1);
}

void launch_amr_split(const Box& b, int W, const double* r, float* f0, float* f1,
                      cudaStream_t s) {
  k_amr_split<<<blocks_for(b.n()), kT, 0, s>>>(b, W, r, f0, f1);
  add_launches(1);
}

static CorrSrc corr(const Box& b, int W, const float* e0, const float* e1, const double* e64) {
  CorrSrc e;
  e.b = b;
  e.W = W;
  e.e[0] = e0;
  e.e[1] = e1;
  e.e64 = e64;
  return e;
}

void launch_amr_add(const Box& b, int W, const float* e0, const float* e1, const double* e64,
                    const uint8_t* mask, double* u, double* delta, cudaStream_t s) {
  k_amr_add<<<blocks_for(b.n()), kT, 0, s>>>(corr(b, W, e0, e1, e64), mask, u, delta);
  add_launches(1);
}

void launch_amr_prolong(const Box& pb, int W, const float* e0, const float* e1, const double* e64,
                        const Box& cb, const int fo[3], double* u, double* delta, cudaStream_t s) {
  k_amr_prolong<<<blocks_for(cb.n()), kT, 0, s>>>(corr(pb, W, e0, e1, e64), cb, fo[0], fo[1],
                                                   fo[2], u, delta);
  add_launches(1);
}

}  // namespace mg
