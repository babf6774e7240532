// FP32 kernels of the inner V-cycle on red/black split storage.
//
// Each grid level keeps its FP32 unknowns, right-hand sides and coefficients
// as two arrays, one per colour ((i+j+k)&1), each packed along x with
// W = (nx+1)/2 entries per row: cell (i,j,k) lives at row (k*ny + j), packed
// index i>>1 of colour (i+j+k)&1.  A red-black Gauss-Seidel half-sweep
// (Sec. 2 item (ii) of arXiv:1809.08857) then reads the other colour and
// writes its own colour with unit-stride, fully coalesced accesses and no
// wasted sectors, in place.
//
// Operator (Sec. 2 items (ii)-(iii)): (A u)_c = alpha u_c + sum_f w_f (u_c -
// u_nb)/h^2 with w_f the harmonic mean of the two cells' beta, beta_c towards
// an electrode cell (beta < 0 marks one) and 2 beta_c on a Dirichlet face.
#include "mg_internal.h"

namespace mg {

namespace {

constexpr int kT = 256;

inline unsigned nblk(long long n) { return (unsigned)((n + kT - 1) / kT); }

// Colour selection by value (a runtime index into a by-value parameter
// array would force it into local memory).
__device__ __forceinline__ const float* sel(const Ptr2& a, int c) { return c ? a.p[1] : a.p[0]; }
__device__ __forceinline__ float* sel(const MPtr2& a, int c) { return c ? a.p[1] : a.p[0]; }
__device__ __forceinline__ const float* bsel(const Split32& op, int c) {
  return c ? op.beta[1] : op.beta[0];
}

__device__ __forceinline__ float wface(float bc, float bn) {
  return bn < 0.0f ? bc : __fdividef(2.0f * bc * bn, bc + bn);
}

// Row of the operator at a cell of colour `col`, packed position t (row
// offset + p), coordinates (i, j, k), s = i & 1.  Returns the residual
// f - A u; u_c is the cell's own value.
template <bool VB>
__device__ __forceinline__ void row32(const Split32& op, int col, long long t, int i, int j,
                                      int k, const float* __restrict__ uo, float& diag,
                                      float& off) {
  const int W = op.W;
  const long long rowo = t - (i >> 1);
  const int s = i & 1;
  const float* bt = bsel(op, col ^ 1);
  const float bc = VB ? bsel(op, col)[t] : 1.0f;
  float d = 0.0f, o = 0.0f, w;
  if (i > 0) {
    const long long q = rowo + (i >> 1) - 1 + s;
    w = VB ? wface(bc, bt[q]) : 1.0f;
    d += w;
    o += w * uo[q];
  } else if (op.dir[0]) {
    d += 2.0f * bc;
  }
  if (i + 1 < op.b.nx) {
    const long long q = rowo + (i >> 1) + s;
    w = VB ? wface(bc, bt[q]) : 1.0f;
    d += w;
    o += w * uo[q];
  } else if (op.dir[1]) {
    d += 2.0f * bc;
  }
  if (j > 0) {
    const long long q = t - W;
    w = VB ? wface(bc, bt[q]) : 1.0f;
    d += w;
    o += w * uo[q];
  } else if (op.dir[2]) {
    d += 2.0f * bc;
  }
  if (j + 1 < op.b.ny) {
    const long long q = t + W;
    w = VB ? wface(bc, bt[q]) : 1.0f;
    d += w;
    o += w * uo[q];
  } else if (op.dir[3]) {
    d += 2.0f * bc;
  }
  const long long sz = (long long)W * op.b.ny;
  if (k > 0) {
    const long long q = t - sz;
    w = VB ? wface(bc, bt[q]) : 1.0f;
    d += w;
    o += w * uo[q];
  } else if (op.dir[4]) {
    d += 2.0f * bc;
  }
  if (k + 1 < op.b.nz) {
    const long long q = t + sz;
    w = VB ? wface(bc, bt[q]) : 1.0f;
    d += w;
    o += w * uo[q];
  } else if (op.dir[5]) {
    d += 2.0f * bc;
  }
  diag = d * op.ih2;
  off = o * op.ih2;
}

// One colour of a red-black sweep: u_own <- (f + off) / (alpha + diag).
// zero_other: the other colour is known to be zero (first half-sweep from a
// zero guess), so it is not read.
template <bool VB, bool ZeroOther>
__global__ void __launch_bounds__(kT) k_half_sweep(Split32 op, float alpha, int col,
                                                   const float* __restrict__ f,
                                                   float* __restrict__ u,
                                                   const float* __restrict__ uo) {
  const long long t = (long long)blockIdx.x * kT + threadIdx.x;
  const int W = op.W;
  if (t >= (long long)W * op.b.ny * op.b.nz) return;
  const int p = (int)(t % W);
  const long long jk = t / W;
  const int j = (int)(jk % op.b.ny), k = (int)(jk / op.b.ny);
  const int i = 2 * p + ((j + k + col) & 1);
  if (i >= op.b.nx) return;
  if (VB && bsel(op, col)[t] < 0.0f) return;
  float diag, off;
  if (ZeroOther) {
    row32<VB>(op, col, t, i, j, k, uo, diag, off);  // off unused
    u[t] = __fdividef(f[t], diag + alpha);
  } else {
    row32<VB>(op, col, t, i, j, k, uo, diag, off);
    u[t] = __fdividef(f[t] + off, diag + alpha);
  }
}

__device__ __forceinline__ long long spos(const Split32& op, int i, int j, int k) {
  return ((long long)k * op.b.ny + j) * op.W + (i >> 1);
}

// Residual of the 8 fine children of each coarse cell, averaged into the
// coarse right-hand side; the coarse unknown is zeroed.  Children of coarse
// cell (I,J,K) sit at packed index I of fine rows (2J+b, 2K+c).
template <bool VB>
__global__ void __launch_bounds__(kT) k_resid_restrict(Split32 op, Split32 cop, float alpha,
                                                       Ptr2 f, Ptr2 u, MPtr2 fc, MPtr2 uc) {
  const long long C = (long long)blockIdx.x * kT + threadIdx.x;
  if (C >= cop.b.n()) return;
  const int I = (int)(C % cop.b.nx);
  const long long JK = C / cop.b.nx;
  const int J = (int)(JK % cop.b.ny), K = (int)(JK / cop.b.ny);
  float sum = 0.0f;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int a = q & 1, b = (q >> 1) & 1, c = q >> 2;
    const int i = 2 * I + a, j = 2 * J + b, k = 2 * K + c;
    const int col = (a + b + c) & 1;
    const long long t = spos(op, i, j, k);
    if (VB && bsel(op, col)[t] < 0.0f) continue;
    float diag, off;
    row32<VB>(op, col, t, i, j, k, sel(u, col ^ 1), diag, off);
    sum += sel(f, col)[t] - ((diag + alpha) * sel(u, col)[t] - off);
  }
  const int ccol = (I + J + K) & 1;
  const long long ct = spos(cop, I, J, K);
  sel(fc, ccol)[ct] = 0.125f * sum;
  sel(uc, ccol)[ct] = 0.0f;
}

// coarse correction at a possibly out-of-box coarse index (homogeneous
// reflection: -1 across Dirichlet faces, +1 across Neumann faces)
__device__ __forceinline__ float cval(const Split32& cop, const Ptr2& ec, int I, int J, int K) {
  float s = 1.0f;
  if (I < 0) { I = 0; if (cop.dir[0]) s = -s; }
  if (I >= cop.b.nx) { I = cop.b.nx - 1; if (cop.dir[1]) s = -s; }
  if (J < 0) { J = 0; if (cop.dir[2]) s = -s; }
  if (J >= cop.b.ny) { J = cop.b.ny - 1; if (cop.dir[3]) s = -s; }
  if (K < 0) { K = 0; if (cop.dir[4]) s = -s; }
  if (K >= cop.b.nz) { K = cop.b.nz - 1; if (cop.dir[5]) s = -s; }
  return s * sel(ec, (I + J + K) & 1)[spos(cop, I, J, K)];
}

// u_fine += trilinear (27, 9, 3, 1)/64 interpolation of the coarse
// correction; electrode cells untouched.  blockIdx.y = fine colour.
template <bool VB>
__global__ void __launch_bounds__(kT) k_prolong(Split32 op, Split32 cop, Ptr2 ec, MPtr2 u) {
  const int col = blockIdx.y;
  const long long t = (long long)blockIdx.x * kT + threadIdx.x;
  const int W = op.W;
  if (t >= (long long)W * op.b.ny * op.b.nz) return;
  const int p = (int)(t % W);
  const long long jk = t / W;
  const int j = (int)(jk % op.b.ny), k = (int)(jk / op.b.ny);
  const int i = 2 * p + ((j + k + col) & 1);
  if (i >= op.b.nx) return;
  if (VB && bsel(op, col)[t] < 0.0f) return;
  const int I = i >> 1, J = j >> 1, K = k >> 1;
  const int si = (i & 1) ? 1 : -1, sj = (j & 1) ? 1 : -1, sk = (k & 1) ? 1 : -1;
  const float c000 = cval(cop, ec, I, J, K);
  const float c100 = cval(cop, ec, I + si, J, K);
  const float c010 = cval(cop, ec, I, J + sj, K);
  const float c110 = cval(cop, ec, I + si, J + sj, K);
  const float c001 = cval(cop, ec, I, J, K + sk);
  const float c101 = cval(cop, ec, I + si, J, K + sk);
  const float c011 = cval(cop, ec, I, J + sj, K + sk);
  const float c111 = cval(cop, ec, I + si, J + sj, K + sk);
  const float v = (27.0f * c000 + 9.0f * (c100 + c010 + c001) + 3.0f * (c110 + c101 + c011) +
                   c111) *
                  (1.0f / 64.0f);
  sel(u, col)[t] += v;
}

// r = f - A u at every cell of the level (electrode and padding cells: 0).
template <bool VB>
__global__ void __launch_bounds__(kT) k_resid(Split32 op, float alpha, Ptr2 f, Ptr2 u, MPtr2 r) {
  const int col = blockIdx.y;
  const long long t = (long long)blockIdx.x * kT + threadIdx.x;
  const int W = op.W;
  if (t >= (long long)W * op.b.ny * op.b.nz) return;
  const int p = (int)(t % W);
  const long long jk = t / W;
  const int j = (int)(jk % op.b.ny), k = (int)(jk / op.b.ny);
  const int i = 2 * p + ((j + k + col) & 1);
  float res = 0.0f;
  if (i < op.b.nx && !(VB && bsel(op, col)[t] < 0.0f)) {
    float diag, off;
    row32<VB>(op, col, t, i, j, k, sel(u, col ^ 1), diag, off);
    res = sel(f, col)[t] - ((diag + alpha) * sel(u, col)[t] - off);
  }
  sel(r, col)[t] = res;
}

// u += Minv r on the coarsest level; Minv is indexed by natural cell order.
__global__ void k_dense_apply(Split32 op, const double* __restrict__ Minv, Ptr2 r, MPtr2 u) {
  const int n = (int)op.b.n();
  const int row = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  double s = 0.0;
  for (int c = lane; c < n; c += 32) {
    const int i = c % op.b.nx, j = (c / op.b.nx) % op.b.ny, k = c / (op.b.nx * op.b.ny);
    s += Minv[(size_t)row * n + c] * (double)sel(r, (i + j + k) & 1)[spos(op, i, j, k)];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const int i = row % op.b.nx, j = (row / op.b.nx) % op.b.ny, k = row / (op.b.nx * op.b.ny);
    sel(u, (i + j + k) & 1)[spos(op, i, j, k)] += (float)s;
  }
}

// FP32 split beta of one level from the natural FP64 beta (nullable = 1) and
// mask (nullable): electrode cells get -1.
__global__ void k_split_beta(const double* beta, const uint8_t* mask, Split32 op, MPtr2 out) {
  const long long c = (long long)blockIdx.x * kT + threadIdx.x;
  if (c >= op.b.n()) return;
  const int i = (int)(c % op.b.nx);
  const long long jk = c / op.b.nx;
  const int j = (int)(jk % op.b.ny), k = (int)(jk / op.b.ny);
  const float v = (mask && mask[c]) ? -1.0f : (beta ? (float)beta[c] : 1.0f);
  sel(out, (i + j + k) & 1)[spos(op, i, j, k)] = v;
}

}  // namespace

void launch_half_sweep32(const Split32& op, float alpha, int col, const float* f, float* u,
                         const float* uo, bool zero_other, cudaStream_t s) {
  const long long t = (long long)op.W * op.b.ny * op.b.nz;
  const bool vb = op.beta[0] != nullptr;
  if (vb) {
    if (zero_other) k_half_sweep<true, true><<<nblk(t), kT, 0, s>>>(op, alpha, col, f, u, uo);
    else k_half_sweep<true, false><<<nblk(t), kT, 0, s>>>(op, alpha, col, f, u, uo);
  } else {
    if (zero_other) k_half_sweep<false, true><<<nblk(t), kT, 0, s>>>(op, alpha, col, f, u, uo);
    else k_half_sweep<false, false><<<nblk(t), kT, 0, s>>>(op, alpha, col, f, u, uo);
  }
  add_launches(1);
}

void launch_resid_restrict32s(const Split32& op, const Split32& cop, float alpha, Ptr2 f, Ptr2 u,
                              MPtr2 fc, MPtr2 uc, cudaStream_t s) {
  if (op.beta[0]) k_resid_restrict<true><<<nblk(cop.b.n()), kT, 0, s>>>(op, cop, alpha, f, u, fc, uc);
  else k_resid_restrict<false><<<nblk(cop.b.n()), kT, 0, s>>>(op, cop, alpha, f, u, fc, uc);
  add_launches(1);
}

void launch_prolong32s(const Split32& op, const Split32& cop, Ptr2 ec, MPtr2 u, cudaStream_t s) {
  const long long t = (long long)op.W * op.b.ny * op.b.nz;
  dim3 g(nblk(t), 2);
  if (op.beta[0]) k_prolong<true><<<g, kT, 0, s>>>(op, cop, ec, u);
  else k_prolong<false><<<g, kT, 0, s>>>(op, cop, ec, u);
  add_launches(1);
}

void launch_resid32s(const Split32& op, float alpha, Ptr2 f, Ptr2 u, MPtr2 r, cudaStream_t s) {
  const long long t = (long long)op.W * op.b.ny * op.b.nz;
  dim3 g(nblk(t), 2);
  if (op.beta[0]) k_resid<true><<<g, kT, 0, s>>>(op, alpha, f, u, r);
  else k_resid<false><<<g, kT, 0, s>>>(op, alpha, f, u, r);
  add_launches(1);
}

void launch_dense_apply32s(const Split32& op, const double* Minv, Ptr2 r, MPtr2 u,
                           cudaStream_t s) {
  const long long n = op.b.n();
  k_dense_apply<<<nblk(n * 32), kT, 0, s>>>(op, Minv, r, u);
  add_launches(1);
}

void launch_split_beta(const double* beta, const uint8_t* mask, const Split32& op, MPtr2 out,
                       cudaStream_t s) {
  k_split_beta<<<nblk(op.b.n()), kT, 0, s>>>(beta, mask, op, out);
  add_launches(1);
}

}  // namespace mg
