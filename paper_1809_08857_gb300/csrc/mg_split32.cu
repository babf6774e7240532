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
// an electrode cell and 2 beta_c on a Dirichlet face.  Each level stores
// hb = 1/(2 beta) per cell (hb < 0 marks an electrode cell), so the harmonic
// mean 2 b_c b_n / (b_c + b_n) is one add and one reciprocal:
// w = 1 / (hb_c + hb_n); towards an electrode w = 1 / (2 hb_c); on a
// Dirichlet face w = 1 / hb_c.
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

// face weight between a free cell (hb = hc) and an in-box neighbour (hn)
__device__ __forceinline__ float wface(float hc, float hn) {
  return __fdividef(1.0f, hn < 0.0f ? hc + hc : hc + hn);
}
// Dirichlet domain face: 2 beta_c
__device__ __forceinline__ float wdir(float hc) { return __fdividef(1.0f, hc); }

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
  const float bc = VB ? bsel(op, col)[t] : 0.5f;  // hb of the cell
  const float wd = VB ? wdir(bc) : 2.0f;           // Dirichlet face weight
  float d = 0.0f, o = 0.0f, w;
  if (i > 0) {
    const long long q = rowo + (i >> 1) - 1 + s;
    w = VB ? wface(bc, bt[q]) : 1.0f;
    d += w;
    o += w * uo[q];
  } else if (op.dir[0]) {
    d += wd;
  }
  if (i + 1 < op.b.nx) {
    const long long q = rowo + (i >> 1) + s;
    w = VB ? wface(bc, bt[q]) : 1.0f;
    d += w;
    o += w * uo[q];
  } else if (op.dir[1]) {
    d += wd;
  }
  if (j > 0) {
    const long long q = t - W;
    w = VB ? wface(bc, bt[q]) : 1.0f;
    d += w;
    o += w * uo[q];
  } else if (op.dir[2]) {
    d += wd;
  }
  if (j + 1 < op.b.ny) {
    const long long q = t + W;
    w = VB ? wface(bc, bt[q]) : 1.0f;
    d += w;
    o += w * uo[q];
  } else if (op.dir[3]) {
    d += wd;
  }
  const long long sz = (long long)W * op.b.ny;
  if (k > 0) {
    const long long q = t - sz;
    w = VB ? wface(bc, bt[q]) : 1.0f;
    d += w;
    o += w * uo[q];
  } else if (op.dir[4]) {
    d += wd;
  }
  if (k + 1 < op.b.nz) {
    const long long q = t + sz;
    w = VB ? wface(bc, bt[q]) : 1.0f;
    d += w;
    o += w * uo[q];
  } else if (op.dir[5]) {
    d += wd;
  }
  diag = d * op.ih2;
  off = o * op.ih2;
}

// One colour of a red-black sweep: u_own <- (f + off) / (alpha + diag).
// ZeroOther: the other colour is known to be zero (first half-sweep from a
// zero guess), so it is not read.  Block (32, 8) over (packed x, y), one z
// plane per blockIdx.z: no integer division in the index math.
template <bool VB, bool ZeroOther>
__global__ void __launch_bounds__(kT) k_half_sweep(Split32 op, float alpha, int col,
                                                   const float* __restrict__ f,
                                                   float* __restrict__ u,
                                                   const float* __restrict__ uo) {
  const int p = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
  if (p >= op.W || j >= op.b.ny) return;
  const int i = 2 * p + ((j + k + col) & 1);
  if (i >= op.b.nx) return;
  const long long t = ((long long)k * op.b.ny + j) * op.W + p;
  if (VB && bsel(op, col)[t] < 0.0f) return;
  float diag, off;
  row32<VB>(op, col, t, i, j, k, uo, diag, off);
  u[t] = __fdividef(ZeroOther ? f[t] : f[t] + off, diag + alpha);
}

__device__ __forceinline__ float4 ld4(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}
__device__ __forceinline__ float el(const float4& v, int e) {
  return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}

// Vectorised half-sweep: four packed cells per thread (float4 loads and
// store), x-neighbours across quad edges exchanged by warp shuffles.  Needs
// nx % 8 == 0 (W % 4 == 0, no padding).  Block (32, 8): a warp covers 128
// packed cells of one row, so the row parity S (which decides whether a
// cell's x-neighbours in the other colour sit at packed p-1, p or p, p+1) is
// warp-uniform and the quad update is compiled once per parity.
struct Quad {
  float4 F, BO, U;                   // own rhs, own hb, own old value (electrodes)
  float ux[6], bx[6];                // other colour at packed pp-1 .. pp+4
  float4 UYm, UYp, UZm, UZp;         // other colour, y/z neighbours
  float4 BYm, BYp, BZm, BZp;
};

template <bool VB, bool ZeroOther, bool HasMask, int S>
__device__ __forceinline__ float4 quad_update(const Split32& op, float alpha, const Quad& q,
                                              int pp, bool ym, bool yp, bool zm, bool zp) {
  float out[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int p = pp + e;
    const float hc = VB ? el(q.BO, e) : 0.5f;
    float d = 0.0f, o = 0.0f;
    auto face = [&](float hn, float un) {
      float w = 1.0f;
      if (VB) w = HasMask ? wface(hc, hn) : __fdividef(1.0f, hc + hn);
      d += w;
      if (!ZeroOther) o = fmaf(w, un, o);
    };
    auto dface = [&](bool dir) {
      if (dir) d += VB ? wdir(hc) : 2.0f;
    };
    // x: other-colour neighbours at packed p - 1 + S and p + S
    if (!(S == 0 && p == 0)) face(q.bx[e + S], q.ux[e + S]);
    else dface(op.dir[0]);
    if (!(S == 1 && p == op.W - 1)) face(q.bx[e + S + 1], q.ux[e + S + 1]);
    else dface(op.dir[1]);
    if (ym) face(el(q.BYm, e), el(q.UYm, e)); else dface(op.dir[2]);
    if (yp) face(el(q.BYp, e), el(q.UYp, e)); else dface(op.dir[3]);
    if (zm) face(el(q.BZm, e), el(q.UZm, e)); else dface(op.dir[4]);
    if (zp) face(el(q.BZp, e), el(q.UZp, e)); else dface(op.dir[5]);
    float v = __fdividef(fmaf(o, op.ih2, el(q.F, e)), fmaf(d, op.ih2, alpha));
    if (HasMask && hc < 0.0f) v = el(q.U, e);
    out[e] = v;
  }
  return make_float4(out[0], out[1], out[2], out[3]);
}

template <bool VB, bool ZeroOther, bool HasMask>
__global__ void __launch_bounds__(kT, 4) k_half_sweep_v4(Split32 op, float alpha, int col,
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
  const float* bo = bsel(op, col);
  const float* bt = bsel(op, col ^ 1);
  const float4 half = make_float4(0.5f, 0.5f, 0.5f, 0.5f);
  const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const bool ym = jj > 0, yp = jj < ny - 1, zm = k > 0, zp = k < nz - 1;
  Quad q;
  q.F = ld4(f + t0);
  q.BO = VB ? ld4(bo + t0) : half;
  const float4 UO = ZeroOther ? zero : ld4(uo + t0);
  const float4 BT = VB ? ld4(bt + t0) : half;
  q.UYm = (!ZeroOther && ym) ? ld4(uo + t0 - W) : zero;
  q.UYp = (!ZeroOther && yp) ? ld4(uo + t0 + W) : zero;
  q.UZm = (!ZeroOther && zm) ? ld4(uo + t0 - sz) : zero;
  q.UZp = (!ZeroOther && zp) ? ld4(uo + t0 + sz) : zero;
  q.BYm = (VB && ym) ? ld4(bt + t0 - W) : half;
  q.BYp = (VB && yp) ? ld4(bt + t0 + W) : half;
  q.BZm = (VB && zm) ? ld4(bt + t0 - sz) : half;
  q.BZp = (VB && zp) ? ld4(bt + t0 + sz) : half;
  q.U = HasMask ? ld4(u + t0) : zero;
  float uprev = __shfl_up_sync(FULL, UO.w, 1), unext = __shfl_down_sync(FULL, UO.x, 1);
  float bprev = __shfl_up_sync(FULL, BT.w, 1), bnext = __shfl_down_sync(FULL, BT.x, 1);
  if (lane == 0 && pp > 0) {
    if (!ZeroOther) uprev = uo[t0 - 1];
    if (VB) bprev = bt[t0 - 1];
  }
  if (lane == 31 && pp + 4 < W) {
    if (!ZeroOther) unext = uo[t0 + 4];
    if (VB) bnext = bt[t0 + 4];
  }
  q.ux[0] = uprev; q.ux[1] = UO.x; q.ux[2] = UO.y; q.ux[3] = UO.z; q.ux[4] = UO.w; q.ux[5] = unext;
  q.bx[0] = bprev; q.bx[1] = BT.x; q.bx[2] = BT.y; q.bx[3] = BT.z; q.bx[4] = BT.w; q.bx[5] = bnext;
  const int s = (jj + k + col) & 1;  // warp-uniform
  const float4 v = s ? quad_update<VB, ZeroOther, HasMask, 1>(op, alpha, q, pp, ym, yp, zm, zp)
                     : quad_update<VB, ZeroOther, HasMask, 0>(op, alpha, q, pp, ym, yp, zm, zp);
  if (active) *reinterpret_cast<float4*>(u + t0) = v;
}

__device__ __forceinline__ long long spos(const Split32& op, int i, int j, int k) {
  return ((long long)k * op.b.ny + j) * op.W + (i >> 1);
}

// Residual of the 8 fine children of each coarse cell, averaged into the
// coarse right-hand side; the coarse unknown is zeroed.  Children of coarse
// cell (I,J,K) sit at packed index I of fine rows (2J+b, 2K+c).
// RedOnly: the pre-smoothing ended with a black half-sweep, after which every
// black cell satisfies its own equation (Gauss-Seidel), so only the four red
// children carry a residual.
template <bool VB, bool RedOnly>
__global__ void __launch_bounds__(kT) k_resid_restrict(Split32 op, Split32 cop, float alpha,
                                                       Ptr2 f, Ptr2 u, MPtr2 fc, MPtr2 uc) {
  const int I = blockIdx.x * 32 + threadIdx.x;
  const int J = blockIdx.y * 8 + threadIdx.y, K = blockIdx.z;
  if (I >= cop.b.nx || J >= cop.b.ny) return;
  float sum = 0.0f;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int a = q & 1, b = (q >> 1) & 1, c = q >> 2;
    const int i = 2 * I + a, j = 2 * J + b, k = 2 * K + c;
    const int col = (a + b + c) & 1;
    if (RedOnly && col == 1) continue;
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


// u_fine += trilinear (27, 9, 3, 1)/64 interpolation of the coarse
// correction; electrode cells untouched.  One thread per fine x-pair
// (2p, 2p+1): both cells sit at packed index p (one in each colour) and share
// the coarse parent I = p, so the 8-point stencils of the pair need 12
// coarse values.  Block (32, 8) over (p, j), blockIdx.z = k.
// BlackOnly: post-smoothing starts with a red half-sweep, which overwrites
// every red cell without reading it, so only black cells are corrected.
template <bool VB, bool BlackOnly>
__global__ void __launch_bounds__(kT) k_prolong(Split32 op, Split32 cop, Ptr2 ec, MPtr2 u) {
  const int p = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
  if (p >= op.W || j >= op.b.ny) return;
  const long long t = ((long long)k * op.b.ny + j) * op.W + p;
  const int c0 = (j + k) & 1;  // colour of cell 2p
  const bool do0 = !BlackOnly || c0 == 1;
  const bool do1 = (!BlackOnly || c0 == 0) && 2 * p + 1 < op.b.nx;
  const int cnx = cop.b.nx, cny = cop.b.ny, cnz = cop.b.nz, cW = cop.W;
  // coarse x positions I-1, I, I+1 (I = p) and the two y / z rows, reflected
  // at domain faces (sign -1 across Dirichlet faces, +1 across Neumann)
  const int I = p, J = j >> 1, K = k >> 1;
  const int Jn = J + ((j & 1) ? 1 : -1), Kn = K + ((k & 1) ? 1 : -1);
  int xi[3] = {I - 1, I, I + 1};
  float xs[3] = {1.0f, 1.0f, 1.0f};
  if (xi[0] < 0) { xi[0] = 0; xs[0] = cop.dir[0] ? -1.0f : 1.0f; }
  if (xi[2] >= cnx) { xi[2] = cnx - 1; xs[2] = cop.dir[1] ? -1.0f : 1.0f; }
  int yj[2] = {J, Jn};
  float ys = 1.0f;
  if (Jn < 0) { yj[1] = 0; ys = cop.dir[2] ? -1.0f : 1.0f; }
  if (Jn >= cny) { yj[1] = cny - 1; ys = cop.dir[3] ? -1.0f : 1.0f; }
  int zk[2] = {K, Kn};
  float zs = 1.0f;
  if (Kn < 0) { zk[1] = 0; zs = cop.dir[4] ? -1.0f : 1.0f; }
  if (Kn >= cnz) { zk[1] = cnz - 1; zs = cop.dir[5] ? -1.0f : 1.0f; }
  float x0 = 0.0f, x1 = 0.0f;  // interpolants of cells 2p and 2p+1
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int b = q & 1, c = q >> 1;
    const float wyz = (b ? 0.25f * ys : 0.75f) * (c ? 0.25f * zs : 0.75f);
    const int JJ = yj[b], KK = zk[c];
    const long long row = ((long long)KK * cny + JJ) * cW;
    const int par = (JJ + KK) & 1;
    // coarse cell (X, JJ, KK) has colour (X + JJ + KK) & 1, packed X >> 1
    const float B = sel(ec, (xi[1] + par) & 1)[row + (xi[1] >> 1)];
    if (do0) {
      const float A = xs[0] * sel(ec, (xi[0] + par) & 1)[row + (xi[0] >> 1)];
      x0 = fmaf(wyz, fmaf(0.75f, B, 0.25f * A), x0);
    }
    if (do1) {
      const float C = xs[2] * sel(ec, (xi[2] + par) & 1)[row + (xi[2] >> 1)];
      x1 = fmaf(wyz, fmaf(0.75f, B, 0.25f * C), x1);
    }
  }
  if (do0 && !(VB && bsel(op, c0)[t] < 0.0f)) sel(u, c0)[t] += x0;
  if (do1 && !(VB && bsel(op, c0 ^ 1)[t] < 0.0f)) sel(u, c0 ^ 1)[t] += x1;
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

// FP32 split coefficient hb = 1/(2 beta) of one level from the natural FP64
// beta (nullable = 1) and mask (nullable): electrode cells get -1.
__global__ void k_split_beta(const double* beta, const uint8_t* mask, Split32 op, MPtr2 out) {
  const long long c = (long long)blockIdx.x * kT + threadIdx.x;
  if (c >= op.b.n()) return;
  const int i = (int)(c % op.b.nx);
  const long long jk = c / op.b.nx;
  const int j = (int)(jk % op.b.ny), k = (int)(jk / op.b.ny);
  const float v = (mask && mask[c]) ? -1.0f : (beta ? (float)(0.5 / beta[c]) : 0.5f);
  sel(out, (i + j + k) & 1)[spos(op, i, j, k)] = v;
}

}  // namespace

void launch_half_sweep32(const Split32& op, float alpha, int col, const float* f, float* u,
                         const float* uo, bool zero_other, bool has_mask, cudaStream_t s) {
  const bool vb = op.beta[0] != nullptr;
  dim3 blk(32, 8);
  if (op.b.nx % 8 == 0) {
    dim3 g((op.W / 4 + 31) / 32, (op.b.ny + 7) / 8, op.b.nz);
#define HS4(A, B, C) k_half_sweep_v4<A, B, C><<<g, blk, 0, s>>>(op, alpha, col, f, u, uo)
    if (vb) {
      if (has_mask) { if (zero_other) HS4(true, true, true); else HS4(true, false, true); }
      else { if (zero_other) HS4(true, true, false); else HS4(true, false, false); }
    } else {
      if (zero_other) HS4(false, true, false); else HS4(false, false, false);
    }
#undef HS4
  } else {
    dim3 g((op.W + 31) / 32, (op.b.ny + 7) / 8, op.b.nz);
    if (vb) {
      if (zero_other) k_half_sweep<true, true><<<g, blk, 0, s>>>(op, alpha, col, f, u, uo);
      else k_half_sweep<true, false><<<g, blk, 0, s>>>(op, alpha, col, f, u, uo);
    } else {
      if (zero_other) k_half_sweep<false, true><<<g, blk, 0, s>>>(op, alpha, col, f, u, uo);
      else k_half_sweep<false, false><<<g, blk, 0, s>>>(op, alpha, col, f, u, uo);
    }
  }
  add_launches(1);
}

void launch_resid_restrict32s(const Split32& op, const Split32& cop, float alpha, Ptr2 f, Ptr2 u,
                              MPtr2 fc, MPtr2 uc, bool red_only, cudaStream_t s) {
  dim3 blk(32, 8), g((cop.b.nx + 31) / 32, (cop.b.ny + 7) / 8, cop.b.nz);
  if (op.beta[0]) {
    if (red_only) k_resid_restrict<true, true><<<g, blk, 0, s>>>(op, cop, alpha, f, u, fc, uc);
    else k_resid_restrict<true, false><<<g, blk, 0, s>>>(op, cop, alpha, f, u, fc, uc);
  } else {
    if (red_only) k_resid_restrict<false, true><<<g, blk, 0, s>>>(op, cop, alpha, f, u, fc, uc);
    else k_resid_restrict<false, false><<<g, blk, 0, s>>>(op, cop, alpha, f, u, fc, uc);
  }
  add_launches(1);
}

void launch_prolong32s(const Split32& op, const Split32& cop, Ptr2 ec, MPtr2 u, bool black_only,
                       cudaStream_t s) {
  dim3 blk(32, 8), g((op.W + 31) / 32, (op.b.ny + 7) / 8, op.b.nz);
  if (op.beta[0]) {
    if (black_only) k_prolong<true, true><<<g, blk, 0, s>>>(op, cop, ec, u);
    else k_prolong<true, false><<<g, blk, 0, s>>>(op, cop, ec, u);
  } else {
    if (black_only) k_prolong<false, true><<<g, blk, 0, s>>>(op, cop, ec, u);
    else k_prolong<false, false><<<g, blk, 0, s>>>(op, cop, ec, u);
  }
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
