// FP32 kernels of the inner V-cycle on the coarse levels of a
// variable-coefficient Poisson problem whose coarse operators are built face
// by face (launch_coarsen_faces64): red/black split storage as in
// mg_split32.cu, but the operator is given by per-cell face weights instead
// of a cell coefficient:
//
//     (A u)_c = (alpha + D_c) u_c - sum_{in-box nb} w_f u_nb
//
// with fx[c], fy[c], fz[c] the weights (already / h^2) of the faces between c
// and c - e_x, c - e_y, c - e_z, the +x/+y/+z faces of c being the -x/-y/-z
// faces of its neighbours (the other colour), and D_c the sum of all six face
// weights including domain and electrode faces (D_c < 0 marks an electrode
// cell, which keeps its value).  A domain face holds its weight in D_c only:
// it has no neighbour value (the correction's boundary data are homogeneous).
// Smoothing is red-black Gauss-Seidel (Sec. 2 item (ii) of arXiv:1809.08857).
#include "mg_internal.h"

namespace mg {

namespace {

constexpr int kT = 256;

__device__ __forceinline__ const float* csel(const float* const* a, int c) {
  return c ? a[1] : a[0];
}
__device__ __forceinline__ const float* ps(const Ptr2& a, int c) { return c ? a.p[1] : a.p[0]; }
__device__ __forceinline__ float* ps(const MPtr2& a, int c) { return c ? a.p[1] : a.p[0]; }

__device__ __forceinline__ float4 ld4(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}
__device__ __forceinline__ float el(const float4& v, int e) {
  return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}

// Residual row at cell (i, j, k) of colour col, packed position t: returns
// (diag without alpha, off-diagonal sum) with the other colour's values uo.
__device__ __forceinline__ void frow(const Split32& op, int col, long long t, int i, int j,
                                     int k, const float* __restrict__ uo, float& diag,
                                     float& off) {
  const int W = op.W;
  const int o = col ^ 1;
  const long long rowo = t - (i >> 1);
  const long long sz = (long long)W * op.b.ny;
  const float* fxo = csel(op.fx, o);
  const float* fyo = csel(op.fy, o);
  const float* fzo = csel(op.fz, o);
  float s = 0.0f;
  if (i > 0) s = fmaf(csel(op.fx, col)[t], uo[rowo + ((i - 1) >> 1)], s);
  if (i + 1 < op.b.nx) {
    const long long q = rowo + ((i + 1) >> 1);
    s = fmaf(fxo[q], uo[q], s);
  }
  if (j > 0) s = fmaf(csel(op.fy, col)[t], uo[t - W], s);
  if (j + 1 < op.b.ny) s = fmaf(fyo[t + W], uo[t + W], s);
  if (k > 0) s = fmaf(csel(op.fz, col)[t], uo[t - sz], s);
  if (k + 1 < op.b.nz) s = fmaf(fzo[t + sz], uo[t + sz], s);
  diag = csel(op.dg, col)[t];
  off = s;
}

// One colour of a red-black sweep, one cell per thread (any nx).  Block
// (32, 8) over (packed x, y), one z plane per blockIdx.z.
template <bool ZeroOther>
__global__ void __launch_bounds__(kT) k_half_sweep_f(Split32 op, float alpha, int col,
                                                     const float* __restrict__ f,
                                                     float* __restrict__ u,
                                                     const float* __restrict__ uo) {
  const int p = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
  if (p >= op.W || j >= op.b.ny) return;
  const int i = 2 * p + ((j + k + col) & 1);
  if (i >= op.b.nx) return;
  const long long t = ((long long)k * op.b.ny + j) * op.W + p;
  float diag, off = 0.0f;
  if (ZeroOther) diag = csel(op.dg, col)[t];
  else frow(op, col, t, i, j, k, uo, diag, off);
  if (diag < 0.0f) return;  // electrode cell
  u[t] = __fdividef(f[t] + off, diag + alpha);
}

// Four packed cells per thread (float4), x-neighbours across quads by warp
// shuffles; needs nx % 8 == 0.  Row parity S (warp-uniform) as in
// k_half_sweep_v4 of mg_split32.cu: the other-colour x-neighbours of own
// packed cell p sit at packed p - 1 + S and p + S.
template <bool ZeroOther, bool HasMask, int S>
__device__ __forceinline__ float4 fquad(const Split32& op, float alpha, int pp, const float4& F,
                                        const float4& Dg, const float4& WX, const float4& WY,
                                        const float4& WZ, const float* ux, const float* wxo,
                                        const float4& WYp, const float4& WZp, const float4& UYm,
                                        const float4& UYp, const float4& UZm, const float4& UZp,
                                        const float4& U, bool ym, bool yp, bool zm, bool zp) {
  float out[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int p = pp + e;
    float o = 0.0f;
    if (!ZeroOther) {
      if (!(S == 0 && p == 0)) o = fmaf(el(WX, e), ux[e + S], o);
      if (!(S == 1 && p == op.W - 1)) o = fmaf(wxo[e + S + 1], ux[e + S + 1], o);
      if (ym) o = fmaf(el(WY, e), el(UYm, e), o);
      if (yp) o = fmaf(el(WYp, e), el(UYp, e), o);
      if (zm) o = fmaf(el(WZ, e), el(UZm, e), o);
      if (zp) o = fmaf(el(WZp, e), el(UZp, e), o);
    }
    const float d = el(Dg, e);
    float v = __fdividef(el(F, e) + o, d + alpha);
    if (HasMask && d < 0.0f) v = el(U, e);
    out[e] = v;
  }
  return make_float4(out[0], out[1], out[2], out[3]);
}

template <bool ZeroOther, bool HasMask>
__global__ void __launch_bounds__(kT, 3) k_half_sweep_f4(Split32 op, float alpha, int col,
                                                         const float* __restrict__ f,
                                                         float* __restrict__ u,
                                                         const float* __restrict__ uo) {
  const unsigned FULL = 0xffffffffu;
  const int W = op.W, ny = op.b.ny, nz = op.b.nz;
  const int lane = threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
  const int p0 = 4 * (blockIdx.x * 32 + lane);
  const bool active = j < ny && p0 < W;
  const int jj = min(j, ny - 1);
  const int pp = min(p0, W - 4);
  const long long t0 = ((long long)k * ny + jj) * W + pp;
  const long long sz = (long long)W * ny;
  const int o = col ^ 1;
  const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const bool ym = jj > 0, yp = jj < ny - 1, zm = k > 0, zp = k < nz - 1;
  const float4 F = ld4(f + t0);
  const float4 Dg = ld4(csel(op.dg, col) + t0);
  float4 WX = zero, WY = zero, WZ = zero, WYp = zero, WZp = zero, WXO = zero, UO = zero;
  float4 UYm = zero, UYp = zero, UZm = zero, UZp = zero;
  if (!ZeroOther) {
    WX = ld4(csel(op.fx, col) + t0);
    WY = ld4(csel(op.fy, col) + t0);
    WZ = ld4(csel(op.fz, col) + t0);
    WXO = ld4(csel(op.fx, o) + t0);
    UO = ld4(uo + t0);
    if (ym) UYm = ld4(uo + t0 - W);
    if (yp) {
      UYp = ld4(uo + t0 + W);
      WYp = ld4(csel(op.fy, o) + t0 + W);
    }
    if (zm) UZm = ld4(uo + t0 - sz);
    if (zp) {
      UZp = ld4(uo + t0 + sz);
      WZp = ld4(csel(op.fz, o) + t0 + sz);
    }
  }
  const float4 U = HasMask ? ld4(u + t0) : zero;
  float uprev = __shfl_up_sync(FULL, UO.w, 1), unext = __shfl_down_sync(FULL, UO.x, 1);
  float wnext = __shfl_down_sync(FULL, WXO.x, 1);
  if (!ZeroOther) {
    if (lane == 0 && pp > 0) uprev = uo[t0 - 1];
    if (lane == 31 && pp + 4 < W) {
      unext = uo[t0 + 4];
      wnext = csel(op.fx, o)[t0 + 4];
    }
  }
  // other colour at packed pp-1 .. pp+4; the -x face weight of the other
  // colour's cell at packed q is wxo[q - pp + 1] (entry 0 is never used: it
  // is the face of a cell to the left of every own cell)
  const float ux[6] = {uprev, UO.x, UO.y, UO.z, UO.w, unext};
  const float wxo[6] = {0.0f, WXO.x, WXO.y, WXO.z, WXO.w, wnext};
  const int s = (jj + k + col) & 1;  // warp-uniform
  const float4 v =
      s ? fquad<ZeroOther, HasMask, 1>(op, alpha, pp, F, Dg, WX, WY, WZ, ux, wxo, WYp, WZp, UYm,
                                       UYp, UZm, UZp, U, ym, yp, zm, zp)
        : fquad<ZeroOther, HasMask, 0>(op, alpha, pp, F, Dg, WX, WY, WZ, ux, wxo, WYp, WZp, UYm,
                                       UYp, UZm, UZp, U, ym, yp, zm, zp);
  if (active) *reinterpret_cast<float4*>(u + t0) = v;
}

// Residual of the red fine children of each coarse cell, averaged (1/8)
// into the coarse right-hand side (the black children carry no residual
// after a pre-smoothing that ends with a black half-sweep); the coarse
// unknown is zeroed.  One thread per coarse cell.
__global__ void __launch_bounds__(kT) k_resid_restrict_f(Split32 op, Split32 cop, float alpha,
                                                         Ptr2 f, Ptr2 u, MPtr2 fc, MPtr2 uc) {
  const int I = blockIdx.x * 32 + threadIdx.x;
  const int J = blockIdx.y * 8 + threadIdx.y, K = blockIdx.z;
  if (I >= cop.b.nx || J >= cop.b.ny) return;
  const int ny = op.b.ny, W = op.W;
  float acc = 0.0f;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int a = q & 1, b = (q >> 1) & 1, c = q >> 2;
    if ((a + b + c) & 1) continue;  // black child (2I, 2J, 2K parities are even)
    const int i = 2 * I + a, j = 2 * J + b, k = 2 * K + c;
    const long long t = ((long long)k * ny + j) * W + (i >> 1);
    float diag, off;
    frow(op, 0, t, i, j, k, u.p[1], diag, off);
    if (diag < 0.0f) continue;
    acc += f.p[0][t] - fmaf(diag + alpha, u.p[0][t], -off);
  }
  const int ccol = (I + J + K) & 1;
  const long long ct = ((long long)K * cop.b.ny + J) * cop.W + (I >> 1);
  ps(fc, ccol)[ct] = 0.125f * acc;
  ps(uc, ccol)[ct] = 0.0f;
}

// r = f - A u at every cell of the level (electrode and padding cells: 0).
__global__ void __launch_bounds__(kT) k_resid_f(Split32 op, float alpha, Ptr2 f, Ptr2 u,
                                                MPtr2 r) {
  const int col = blockIdx.y;
  const long long t = (long long)blockIdx.x * kT + threadIdx.x;
  const int W = op.W;
  if (t >= (long long)W * op.b.ny * op.b.nz) return;
  const int p = (int)(t % W);
  const long long jk = t / W;
  const int j = (int)(jk % op.b.ny), k = (int)(jk / op.b.ny);
  const int i = 2 * p + ((j + k + col) & 1);
  float res = 0.0f;
  if (i < op.b.nx) {
    float diag, off;
    frow(op, col, t, i, j, k, ps(u, col ^ 1), diag, off);
    if (diag >= 0.0f) res = ps(f, col)[t] - fmaf(diag + alpha, ps(u, col)[t], -off);
  }
  ps(r, col)[t] = res;
}

// FP32 split copies of a level's FP64 face weights and diagonal.
__global__ void k_split_faces(const double* __restrict__ cx, const double* __restrict__ cy,
                              const double* __restrict__ cz, const double* __restrict__ D, Box b,
                              int W, MPtr2 fx, MPtr2 fy, MPtr2 fz, MPtr2 dg) {
  const long long c = (long long)blockIdx.x * kT + threadIdx.x;
  if (c >= b.n()) return;
  const int i = (int)(c % b.nx);
  const long long jk = c / b.nx;
  const int j = (int)(jk % b.ny), k = (int)(jk / b.ny);
  const int col = (i + j + k) & 1;
  const long long t = ((long long)k * b.ny + j) * W + (i >> 1);
  ps(fx, col)[t] = (float)cx[c];
  ps(fy, col)[t] = (float)cy[c];
  ps(fz, col)[t] = (float)cz[c];
  ps(dg, col)[t] = (float)D[c];
}

}  // namespace

void launch_half_sweep32f(const Split32& op, float alpha, int col, const float* f, float* u,
                          const float* uo, bool zero_other, bool has_mask, cudaStream_t s) {
  dim3 blk(32, 8);
  if (op.b.nx % 8 == 0) {
    dim3 g((op.W / 4 + 31) / 32, (op.b.ny + 7) / 8, op.b.nz);
    if (zero_other) {
      if (has_mask) k_half_sweep_f4<true, true><<<g, blk, 0, s>>>(op, alpha, col, f, u, uo);
      else k_half_sweep_f4<true, false><<<g, blk, 0, s>>>(op, alpha, col, f, u, uo);
    } else {
      if (has_mask) k_half_sweep_f4<false, true><<<g, blk, 0, s>>>(op, alpha, col, f, u, uo);
      else k_half_sweep_f4<false, false><<<g, blk, 0, s>>>(op, alpha, col, f, u, uo);
    }
  } else {
    dim3 g((op.W + 31) / 32, (op.b.ny + 7) / 8, op.b.nz);
    if (zero_other) k_half_sweep_f<true><<<g, blk, 0, s>>>(op, alpha, col, f, u, uo);
    else k_half_sweep_f<false><<<g, blk, 0, s>>>(op, alpha, col, f, u, uo);
  }
  add_launches(1);
}

void launch_resid_restrict32f(const Split32& op, const Split32& cop, float alpha, Ptr2 f, Ptr2 u,
                              MPtr2 fc, MPtr2 uc, cudaStream_t s) {
  dim3 blk(32, 8), g((cop.b.nx + 31) / 32, (cop.b.ny + 7) / 8, cop.b.nz);
  k_resid_restrict_f<<<g, blk, 0, s>>>(op, cop, alpha, f, u, fc, uc);
  add_launches(1);
}

void launch_resid32f(const Split32& op, float alpha, Ptr2 f, Ptr2 u, MPtr2 r, cudaStream_t s) {
  const long long t = (long long)op.W * op.b.ny * op.b.nz;
  dim3 g((unsigned)((t + kT - 1) / kT), 2);
  k_resid_f<<<g, kT, 0, s>>>(op, alpha, f, u, r);
  add_launches(1);
}

void launch_split_faces(const double* cx, const double* cy, const double* cz, const double* D,
                        Box b, int W, MPtr2 fx, MPtr2 fy, MPtr2 fz, MPtr2 dg, cudaStream_t s) {
  k_split_faces<<<(unsigned)((b.n() + kT - 1) / kT), kT, 0, s>>>(cx, cy, cz, D, b, W, fx, fy, fz,
                                                                  dg);
  add_launches(1);
}

}  // namespace mg
