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
// an electrode cell and 2 beta_c rho_f on a domain face (rho_f = 1 Dirichlet,
// 0 Neumann, (ah/2)/(1 + ah/2) Robin).  Each level stores hb = 1/(2 beta)
// per cell (hb < 0 marks an electrode cell), so the harmonic mean
// 2 b_c b_n / (b_c + b_n) is one add and one reciprocal: w = 1 / (hb_c +
// hb_n); towards an electrode w = 1 / (2 hb_c); on a domain face
// rho_f / hb_c.
#include <stdint.h>

#include "mg_internal.h"
#include "tma.cuh"

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
inline const float* bsel_h(const Split32& op, int c) { return c ? op.beta[1] : op.beta[0]; }

// Stacked levels (kernels instantiated with Stk, launched when op.nb > 1):
// the problem of global plane k, its planes, its alpha, and whether it takes
// part.  Without Stk the level is one problem and all of it folds away.
template <bool Stk>
__device__ __forceinline__ int sprob(const Stk32& st, int k, int nzp) {
  return Stk ? k / nzp : 0;
}
template <bool Stk>
__device__ __forceinline__ float salpha(const Stk32& st, int q, float alpha) {
  if (!Stk) return alpha;
  return q == 0 ? st.pa[0] : q == 1 ? st.pa[1] : q == 2 ? st.pa[2] : st.pa[3];
}
template <bool Stk>
__device__ __forceinline__ bool sactive(const Stk32& st, int q) {
  return !Stk || ((st.active >> q) & 1u) != 0;
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
  const float wd = VB ? wdir(bc) : 2.0f;           // Dirichlet face weight (rho = 1)
  float d = 0.0f, o = 0.0f, w;
  if (i > 0) {
    const long long q = rowo + (i >> 1) - 1 + s;
    w = VB ? wface(bc, bt[q]) : 1.0f;
    d += w;
    o += w * uo[q];
  } else {
    d = fmaf(wd, op.rho[0], d);
  }
  if (i + 1 < op.b.nx) {
    const long long q = rowo + (i >> 1) + s;
    w = VB ? wface(bc, bt[q]) : 1.0f;
    d += w;
    o += w * uo[q];
  } else {
    d = fmaf(wd, op.rho[1], d);
  }
  if (j > 0) {
    const long long q = t - W;
    w = VB ? wface(bc, bt[q]) : 1.0f;
    d += w;
    o += w * uo[q];
  } else {
    d = fmaf(wd, op.rho[2], d);
  }
  if (j + 1 < op.b.ny) {
    const long long q = t + W;
    w = VB ? wface(bc, bt[q]) : 1.0f;
    d += w;
    o += w * uo[q];
  } else {
    d = fmaf(wd, op.rho[3], d);
  }
  const long long sz = (long long)W * op.b.ny;
  if (k > 0) {
    const long long q = t - sz;
    w = VB ? wface(bc, bt[q]) : 1.0f;
    d += w;
    o += w * uo[q];
  } else {
    d = fmaf(wd, op.rho[4], d);
  }
  if (k + 1 < op.b.nz) {
    const long long q = t + sz;
    w = VB ? wface(bc, bt[q]) : 1.0f;
    d += w;
    o += w * uo[q];
  } else {
    d = fmaf(wd, op.rho[5], d);
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

// The same on a stack of constant-coefficient problems (Stk32): blockIdx.z
// runs over the stack's planes; the operator row sees the cell's own
// problem's planes.
template <bool ZeroOther>
__global__ void __launch_bounds__(kT) k_half_sweep_stk(Split32 op, Stk32 st, int col,
                                                       const float* __restrict__ f,
                                                       float* __restrict__ u,
                                                       const float* __restrict__ uo) {
  const int p = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
  const int q = k / st.nzp;
  if (p >= op.W || j >= op.b.ny || !sactive<true>(st, q)) return;
  const int i = 2 * p + ((j + k + col) & 1);
  if (i >= op.b.nx) return;
  const long long t = ((long long)k * op.b.ny + j) * op.W + p;
  Split32 opl = op;
  opl.b.nz = st.nzp;
  float diag, off;
  row32<false>(opl, col, t, i, j, k - q * st.nzp, uo, diag, off);
  u[t] = __fdividef(ZeroOther ? f[t] : f[t] + off, diag + salpha<true>(st, q, 0.0f));
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
    auto dface = [&](float r) { d = fmaf(VB ? wdir(hc) : 2.0f, r, d); };
    // x: other-colour neighbours at packed p - 1 + S and p + S
    if (!(S == 0 && p == 0)) face(q.bx[e + S], q.ux[e + S]);
    else dface(op.rho[0]);
    if (!(S == 1 && p == op.W - 1)) face(q.bx[e + S + 1], q.ux[e + S + 1]);
    else dface(op.rho[1]);
    if (ym) face(el(q.BYm, e), el(q.UYm, e)); else dface(op.rho[2]);
    if (yp) face(el(q.BYp, e), el(q.UYp, e)); else dface(op.rho[3]);
    if (zm) face(el(q.BZm, e), el(q.UZm, e)); else dface(op.rho[4]);
    if (zp) face(el(q.BZp, e), el(q.UZp, e)); else dface(op.rho[5]);
    float v = __fdividef(fmaf(o, op.ih2, el(q.F, e)), fmaf(d, op.ih2, alpha));
    if (HasMask && hc < 0.0f) v = el(q.U, e);
    out[e] = v;
  }
  return make_float4(out[0], out[1], out[2], out[3]);
}

// quad_update (other colour known) with each cell's face sums formed as
// trees: the six face weights are independent, so their reciprocals issue
// back to back, and the diagonal and off-diagonal sums are three adds deep
// instead of six.  The staged half-sweep, whose operands come from shared
// memory, is bound by the latency of these dependent chains rather than by
// HBM.  Same weights and faces as quad_update; only the order of the FP32
// additions differs.
// YZin: the row and plane have in-box neighbours in y and z (known for the
// whole warp), so only the x faces need the domain-face test.
template <bool VB, bool HasMask, int S, bool YZin = false>
__device__ __forceinline__ float4 quad_update_tree(const Split32& op, float alpha, const Quad& q,
                                                   int pp, bool ym, bool yp, bool zm, bool zp) {
  float out[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int p = pp + e;
    const float hc = VB ? el(q.BO, e) : 0.5f;
    const float wd = VB ? wdir(hc) : 2.0f;
    // faces -x, +x, -y, +y, -z, +z: in-box neighbour or domain face
    const bool inb[6] = {!(S == 0 && p == 0), !(S == 1 && p == op.W - 1), YZin || ym,
                         YZin || yp,          YZin || zm,                   YZin || zp};
    const float hn[6] = {q.bx[e + S], q.bx[e + S + 1], el(q.BYm, e),
                         el(q.BYp, e), el(q.BZm, e),   el(q.BZp, e)};
    const float un[6] = {q.ux[e + S], q.ux[e + S + 1], el(q.UYm, e),
                         el(q.UYp, e), el(q.UZm, e),   el(q.UZp, e)};
    float w[6], t[6];
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      float wf = 1.0f;
      if (VB) wf = HasMask ? wface(hc, hn[f]) : __fdividef(1.0f, hc + hn[f]);
      w[f] = inb[f] ? wf : wd * op.rho[f];  // a domain face adds wd rho_f to the diagonal
      t[f] = inb[f] ? wf * un[f] : 0.0f;
    }
    const float d = ((w[0] + w[1]) + (w[2] + w[3])) + (w[4] + w[5]);
    const float o = ((t[0] + t[1]) + (t[2] + t[3])) + (t[4] + t[5]);
    float v = __fdividef(fmaf(o, op.ih2, el(q.F, e)), fmaf(d, op.ih2, alpha));
    if (HasMask && hc < 0.0f) v = el(q.U, e);
    out[e] = v;
  }
  return make_float4(out[0], out[1], out[2], out[3]);
}

// Body of the vectorised half-sweep; Stk: on a stack of constant-coefficient
// problems (blockIdx.z runs over the stack's planes).
template <bool VB, bool ZeroOther, bool HasMask, bool Stk>
__device__ __forceinline__ void hs4_body(const Split32& op, const Stk32& st, float alpha, int col,
                                         const float* __restrict__ f, float* __restrict__ u,
                                         const float* __restrict__ uo) {
  const unsigned FULL = 0xffffffffu;
  const int W = op.W, ny = op.b.ny, nz = Stk ? st.nzp : op.b.nz;
  const int lane = threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
  const int sq = sprob<Stk>(st, k, nz);
  if (!sactive<Stk>(st, sq)) return;  // whole CTA
  const int kz = k - sq * nz;
  alpha = salpha<Stk>(st, sq, alpha);
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
  const bool ym = jj > 0, yp = jj < ny - 1, zm = kz > 0, zp = kz < nz - 1;
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

template <bool VB, bool ZeroOther, bool HasMask>
__global__ void __launch_bounds__(kT, 4) k_half_sweep_v4(Split32 op, float alpha, int col,
                                                         const float* __restrict__ f,
                                                         float* __restrict__ u,
                                                         const float* __restrict__ uo) {
  hs4_body<VB, ZeroOther, HasMask, false>(op, Stk32{}, alpha, col, f, u, uo);
}

template <bool ZeroOther>
__global__ void __launch_bounds__(kT, 4) k_half_sweep_v4_stk(Split32 op, Stk32 st, int col,
                                                             const float* __restrict__ f,
                                                             float* __restrict__ u,
                                                             const float* __restrict__ uo) {
  hs4_body<false, ZeroOther, false, true>(op, st, 0.0f, col, f, u, uo);
}

// ---- half-sweep with planes staged by the tensor memory accelerator ------
//
// The update of k_half_sweep_v4 (four packed cells per thread, a warp per
// row of 128 packed cells, block 32 x 8), but a CTA marches through zc (8,
// 16 or 32) planes of its 128 x 8 tile and every plane reaches shared memory by
// a tiled tensor copy issued ahead of its use: the other colour's u and hb
// with a halo of one row in y and four packed entries in x (the copy's x
// start, p0 - 4, stays on a 16-byte boundary), and the own colour's f and
// hb.  Plane k reads the other colour at k - 1, k and k + 1 (a ring of kRingO
// slots keeps the next plane in flight) and its own colour at k (ring of
// kRingW).  A thread's registers hold only the plane it updates, so the
// copies in flight no longer compete with the arithmetic for registers (the
// register-fed form keeps 14 float4 loads of one plane in flight and no
// more).  Copies outside the level (halo rows and columns past the edge) are
// filled with zeros and never enter a face weight; planes -1 and nz are not
// copied at all (their barrier phase completes by a plain arrive).
//
// Every wait on a plane is bounded (tma::kWaitNs); a CTA that gives up sets
// g_sweep_timeout, waits (bounded) for the copies it issued, and returns
// without writing the rest of its planes.  The host reads the flag after
// each solve.
constexpr int kRingO = 4;      // other-colour slots: planes k-1, k, k+1 and one in flight
constexpr int kRingW = 2;      // own-colour slots: plane k and one in flight
constexpr int kOX = 136;       // other-colour box: 128 + 2 x 4 packed entries
constexpr int kOY = 10;        // rows: 8 + 2
constexpr int kOArr = 5504;    // bytes of one other-colour array box (10 x 136 x 4), to 128
constexpr int kWArr = 4096;    // bytes of one own-colour array box (8 x 128 x 4)
__device__ unsigned g_sweep_timeout = 0;

template <bool VB>
struct TmaPlan {
  static constexpr int kO = (VB ? 2 : 1) * kOArr;  // one other-colour slot
  static constexpr int kW = (VB ? 2 : 1) * kWArr;  // one own-colour slot
  static constexpr int kBars = 8 * (kRingO + kRingW);
  static constexpr int smem() { return 128 + kRingO * kO + kRingW * kW + kBars; }
};

// One tensor map per array: the colour array as (W, ny, nz) FP32.
struct SweepMaps {
  CUtensorMap uo, bo_other, f, bo_own;
};

__device__ __forceinline__ float4 lds4(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}

template <bool VB, bool HasMask, bool Stk = false>
__global__ void __launch_bounds__(kT, VB ? 3 : 4)
    k_half_sweep_tma(Split32 op, Stk32 st, float alpha, int col, int zc, float* __restrict__ u,
                     const __grid_constant__ SweepMaps maps) {
  using P = TmaPlan<VB>;
  extern __shared__ unsigned char sweep_smem[];
  const unsigned FULL = 0xffffffffu;
  const int W = op.W, ny = op.b.ny, nz = op.b.nz;
  const int lane = threadIdx.x, warp = threadIdx.y, tid = warp * 32 + lane;
  const int p0 = blockIdx.x * 128, j0 = blockIdx.y * 8;
  // blockIdx.z: chunk of zc planes of problem sq of a stacked level (the
  // chunks of one problem never reach into the next)
  const int nzl = Stk ? st.nzp : nz, cpp = (nzl + zc - 1) / zc;
  const int sq = Stk ? (int)blockIdx.z / cpp : 0;
  if (!sactive<Stk>(st, sq)) return;  // whole CTA, before any barrier exists
  alpha = salpha<Stk>(st, sq, alpha);
  const int zbase = sq * nzl;
  const int ka = zbase + ((int)blockIdx.z - sq * cpp) * zc, kb = min(zbase + nzl, ka + zc);
  const uint32_t base = (tma::smem_addr(sweep_smem) + 127u) & ~127u;
  unsigned char* gbase = sweep_smem + (base - tma::smem_addr(sweep_smem));
  const uint32_t oslot0 = base, wslot0 = base + kRingO * P::kO;
  const uint32_t bar0 = wslot0 + kRingW * P::kW;
  auto obar = [&](int s) { return bar0 + 8u * (uint32_t)s; };
  auto wbar = [&](int s) { return bar0 + 8u * (uint32_t)(kRingO + s); };
  // generic pointers of the slots
  auto optr = [&](int s, int a) {
    return reinterpret_cast<const float*>(gbase + s * P::kO + a * kOArr);
  };
  auto wptr = [&](int s, int a) {
    return reinterpret_cast<const float*>(gbase + kRingO * P::kO + s * P::kW + a * kWArr);
  };
  const int no = kb - ka + 2;  // other-colour planes ka - 1 .. kb
  const int nw = kb - ka;      // own-colour planes ka .. kb - 1

  // producer (thread 0): other-colour sequence number q is plane ka - 1 + q
  auto issue_o = [&](int q) {
    const int s = q % kRingO, z = ka - 1 + q;
    const uint32_t b = obar(s);
    if (z < 0 || z >= nz) {
      tma::bar_arrive(b);
      return;
    }
    tma::bar_arrive_tx(b, (uint32_t)((VB ? 2 : 1) * kOX * kOY * 4));
    const uint32_t d = oslot0 + (uint32_t)(s * P::kO);
    tma::load3(d, &maps.uo, b, p0 - 4, j0 - 1, z);
    if (VB) tma::load3(d + kOArr, &maps.bo_other, b, p0 - 4, j0 - 1, z);
  };
  auto issue_w = [&](int q) {
    const int s = q % kRingW, z = ka + q;
    const uint32_t b = wbar(s);
    tma::bar_arrive_tx(b, (uint32_t)((VB ? 2 : 1) * 128 * 8 * 4));
    const uint32_t d = wslot0 + (uint32_t)(s * P::kW);
    tma::load3(d, &maps.f, b, p0, j0, z);
    if (VB) tma::load3(d + kWArr, &maps.bo_own, b, p0, j0, z);
  };

  if (tid == 0) {
    for (int i = 0; i < kRingO + kRingW; ++i) tma::bar_init(bar0 + 8u * i);
    tma::bar_init_fence();
    for (int q = 0; q < min(kRingO - 1, no); ++q) issue_o(q);
    for (int q = 0; q < min(kRingW - 1, nw); ++q) issue_w(q);
  }
  __syncthreads();

  const int j = j0 + warp, pp = p0 + 4 * lane;
  const bool active = j < ny && pp < W;
  const bool ym = j > 0, yp = j < ny - 1;
  const int r = warp + 1;  // the thread's row in the other-colour box
  const int c = 4 + 4 * lane;
  const float4 half = make_float4(0.5f, 0.5f, 0.5f, 0.5f);
  int issued_o = min(kRingO - 1, no), issued_w = min(kRingW - 1, nw);
  bool ok = true;
  for (int i = 0; i < nw; ++i) {
    const int k = ka + i;
    if (tid == 0) {
      if (issued_o < no) issue_o(issued_o++);
      if (issued_w < nw) issue_w(issued_w++);
    }
    // other planes k - 1, k, k + 1 are sequence numbers i, i + 1, i + 2
    if (i == 0) {
      ok = ok && tma::bar_wait(obar(0), 0u);
      ok = ok && tma::bar_wait(obar(1 % kRingO), (uint32_t)((1 / kRingO) & 1));
    }
    ok = ok && tma::bar_wait(obar((i + 2) % kRingO), (uint32_t)(((i + 2) / kRingO) & 1));
    ok = ok && tma::bar_wait(wbar(i % kRingW), (uint32_t)((i / kRingW) & 1));
    if (ok) {
      const int sm = i % kRingO, sc = (i + 1) % kRingO, sp = (i + 2) % kRingO;
      const float* uoc = optr(sc, 0) + r * kOX;
      const float* boc = optr(sc, 1) + r * kOX;
      Quad q;
      q.F = lds4(wptr(i % kRingW, 0) + warp * 128 + 4 * lane);
      q.BO = VB ? lds4(wptr(i % kRingW, 1) + warp * 128 + 4 * lane) : half;
      q.U = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      const float4 UO = lds4(uoc + c);
      const float4 BT = VB ? lds4(boc + c) : half;
      q.UYm = lds4(uoc - kOX + c);
      q.UYp = lds4(uoc + kOX + c);
      q.UZm = lds4(optr(sm, 0) + r * kOX + c);
      q.UZp = lds4(optr(sp, 0) + r * kOX + c);
      q.BYm = VB ? lds4(boc - kOX + c) : half;
      q.BYp = VB ? lds4(boc + kOX + c) : half;
      q.BZm = VB ? lds4(optr(sm, 1) + r * kOX + c) : half;
      q.BZp = VB ? lds4(optr(sp, 1) + r * kOX + c) : half;
      float uprev = __shfl_up_sync(FULL, UO.w, 1), unext = __shfl_down_sync(FULL, UO.x, 1);
      float bprev = __shfl_up_sync(FULL, BT.w, 1), bnext = __shfl_down_sync(FULL, BT.x, 1);
      if (lane == 0) {
        uprev = uoc[3];
        if (VB) bprev = boc[3];
      }
      if (lane == 31) {
        unext = uoc[4 + 128];
        if (VB) bnext = boc[4 + 128];
      }
      q.ux[0] = uprev; q.ux[1] = UO.x; q.ux[2] = UO.y; q.ux[3] = UO.z; q.ux[4] = UO.w;
      q.ux[5] = unext;
      q.bx[0] = bprev; q.bx[1] = BT.x; q.bx[2] = BT.y; q.bx[3] = BT.z; q.bx[4] = BT.w;
      q.bx[5] = bnext;
      const bool zm = k > zbase, zp = k < zbase + nzl - 1;
      const int sx = (j + k + col) & 1;  // warp-uniform
      // all but the boundary rows and planes: y and z faces without domain tests
      float4 v;
      if (ym && yp && zm && zp)
        v = sx ? quad_update_tree<VB, HasMask, 1, true>(op, alpha, q, pp, ym, yp, zm, zp)
               : quad_update_tree<VB, HasMask, 0, true>(op, alpha, q, pp, ym, yp, zm, zp);
      else
        v = sx ? quad_update_tree<VB, HasMask, 1>(op, alpha, q, pp, ym, yp, zm, zp)
               : quad_update_tree<VB, HasMask, 0>(op, alpha, q, pp, ym, yp, zm, zp);
      if (active) {
        float* dst = u + ((long long)k * ny + j) * W + pp;
        if (!HasMask || (q.BO.x >= 0.0f && q.BO.y >= 0.0f && q.BO.z >= 0.0f && q.BO.w >= 0.0f)) {
          *reinterpret_cast<float4*>(dst) = v;
        } else {
          // electrode cells keep their values
          if (q.BO.x >= 0.0f) dst[0] = v.x;
          if (q.BO.y >= 0.0f) dst[1] = v.y;
          if (q.BO.z >= 0.0f) dst[2] = v.z;
          if (q.BO.w >= 0.0f) dst[3] = v.w;
        }
      }
    }
    // the slots of other plane k - 1 and own plane k are free after this
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }
  }
  if (!ok && tid == 0) {
    atomicExch(&g_sweep_timeout, 1u);
    // the copies issued and not yet waited for by everyone: wait for each
    // slot's last issued phase (bounded) before the CTA's shared memory goes
    for (int q = max(0, issued_o - kRingO); q < issued_o; ++q)
      tma::bar_wait(obar(q % kRingO), (uint32_t)((q / kRingO) & 1));
    for (int q = max(0, issued_w - kRingW); q < issued_w; ++q)
      tma::bar_wait(wbar(q % kRingW), (uint32_t)((q / kRingW) & 1));
  }
}

__device__ __forceinline__ long long spos(const Split32& op, int i, int j, int k) {
  return ((long long)k * op.b.ny + j) * op.W + (i >> 1);
}

// Two adjacent packed entries of a colour array: one float2 when the packed
// width is even (8-byte aligned pair), else two scalars (the second only if
// it exists).
template <bool Vec2>
__device__ __forceinline__ float2 ld2(const float* __restrict__ a, long long t, bool has1) {
  if (Vec2) return *reinterpret_cast<const float2*>(a + t);
  return make_float2(a[t], has1 ? a[t + 1] : 0.0f);
}

// Residual of the fine children of each coarse cell, averaged (1/8) into the
// coarse right-hand side; the coarse unknown is zeroed.
// One thread per coarse packed pair P of a coarse row (J, K): the coarse
// cells X = 2P and 2P+1 (one of each colour, packed index P) have the fine
// children i = 4P..4P+3 in the fine rows (2J+b, 2K+c), which sit at packed
// positions 2P, 2P+1 of both fine colours.  For the cells of colour col the
// thread loads the other colour over the 4 x 4 window of fine rows (j, k) in
// 2J-1..2J+2 x 2K-1..2K+2 without its corners: the x-neighbours come from
// the four own rows, the y- and z-neighbours from the same packed positions
// of the adjacent rows.  x-neighbours outside the pair come from the
// neighbouring lanes (lanes 0 and 31 load them).  Block (32, 8) over (P, J),
// blockIdx.z = K.
// Only the red children carry a residual: the pre-smoothing (at least one
// sweep) ended with a black half-sweep, after which every black cell
// satisfies its own equation (Gauss-Seidel).
template <bool VB, bool Vec2, bool Stk>
__device__ __forceinline__ void rr_body(const Split32& op, const Split32& cop, const Stk32& st,
                                        float alpha, Ptr2 f, Ptr2 u, MPtr2 fc, MPtr2 uc) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x;
  const int J = blockIdx.y * 8 + threadIdx.y, K = blockIdx.z;
  const int cny = cop.b.ny, cnx = cop.b.nx, cW = cop.W;
  // stacked level: problem sq's fine planes are [kb0, kb0 + nz)
  const int sq = sprob<Stk>(st, K, Stk ? st.nzp / 2 : 1);
  if (J >= cny || !sactive<Stk>(st, sq)) return;  // whole warp
  alpha = salpha<Stk>(st, sq, alpha);
  const int Pl = blockIdx.x * 32 + lane;
  const bool live = Pl < cW;
  const int P = live ? Pl : cW - 1;  // idle lanes read a valid pair
  const bool has1 = 2 * P + 1 < cnx;
  const int nx = op.b.nx, ny = op.b.ny, nz = Stk ? st.nzp : op.b.nz, W = op.W;
  const int kb0 = sq * nz;
  const float half = 0.5f;
  float acc0 = 0.0f, acc1 = 0.0f;  // coarse X = 2P, 2P+1
  {
    constexpr int col = 0;  // red cells; black neighbours
    const float* uo = u.p[1];
    const float* bo = op.beta[1];
    // other colour over the row window: R[jj][kk] for j = 2J-1+jj,
    // k = 2K-1+kk (corners unused); rows outside the box are never read
    float2 UO[4][4], BO[4][4];
#pragma unroll
    for (int jj = 0; jj < 4; ++jj)
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const bool inner_j = jj == 1 || jj == 2, inner_k = kk == 1 || kk == 2;
        if (!inner_j && !inner_k) continue;
        const int j = 2 * J - 1 + jj, k = 2 * K - 1 + kk;
        const bool in = j >= 0 && j < ny && k >= kb0 && k < kb0 + nz;
        const long long t = ((long long)k * ny + j) * W + 2 * P;
        UO[jj][kk] = in ? ld2<Vec2>(uo, t, has1) : make_float2(0.0f, 0.0f);
        BO[jj][kk] = (VB && in) ? ld2<Vec2>(bo, t, has1) : make_float2(half, half);
      }
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int j = 2 * J + b, k = 2 * K + c;
        const int s = col ^ ((b + c) & 1);  // own cells at i = 4P+s, 4P+2+s
        const long long t = ((long long)k * ny + j) * W + 2 * P;
        const float2 F = ld2<Vec2>(sel(f, col), t, has1);
        const float2 U = ld2<Vec2>(sel(u, col), t, has1);
        const float2 HC = VB ? ld2<Vec2>(bsel(op, col), t, has1) : make_float2(half, half);
        const float2 ur = UO[b + 1][c + 1], br = BO[b + 1][c + 1];
        // other colour at packed 2P-1 (s = 0) or 2P+2 (s = 1)
        float uh = s ? __shfl_down_sync(FULL, ur.x, 1) : __shfl_up_sync(FULL, ur.y, 1);
        float bh = VB ? (s ? __shfl_down_sync(FULL, br.x, 1) : __shfl_up_sync(FULL, br.y, 1))
                      : half;
        if (s == 0 && lane == 0 && P > 0) {
          uh = uo[t - 1];
          if (VB) bh = bo[t - 1];
        }
        if (s == 1 && lane == 31 && 2 * P + 2 < W) {
          uh = uo[t + 2];
          if (VB) bh = bo[t + 2];
        }
        // x-neighbour packed positions of own cell e (0, 1): 2P+e-1+s, 2P+e+s
        const float ux[4] = {s ? ur.x : uh, s ? ur.y : ur.x, s ? uh : ur.y, 0.0f};
        const float bx[4] = {s ? br.x : bh, s ? br.y : br.x, s ? bh : br.y, 0.0f};
        const float2 yn[2] = {UO[b][c + 1], UO[b + 2][c + 1]};
        const float2 yb[2] = {BO[b][c + 1], BO[b + 2][c + 1]};
        const float2 zn[2] = {UO[b + 1][c], UO[b + 1][c + 2]};
        const float2 zb[2] = {BO[b + 1][c], BO[b + 1][c + 2]};
        const bool ym = j > 0, yp = j < ny - 1, zm = k > kb0, zp = k < kb0 + nz - 1;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int i = 4 * P + 2 * e + s;
          const float hc = e ? HC.y : HC.x;
          float d = 0.0f, o = 0.0f;
          auto face = [&](float hn, float un) {
            const float w = VB ? wface(hc, hn) : 1.0f;
            d += w;
            o = fmaf(w, un, o);
          };
          auto dface = [&](float r) { d = fmaf(VB ? wdir(hc) : 2.0f, r, d); };
          if (i > 0) face(bx[e], ux[e]); else dface(op.rho[0]);
          if (i < nx - 1) face(bx[e + 1], ux[e + 1]); else dface(op.rho[1]);
          if (ym) face(e ? yb[0].y : yb[0].x, e ? yn[0].y : yn[0].x); else dface(op.rho[2]);
          if (yp) face(e ? yb[1].y : yb[1].x, e ? yn[1].y : yn[1].x); else dface(op.rho[3]);
          if (zm) face(e ? zb[0].y : zb[0].x, e ? zn[0].y : zn[0].x); else dface(op.rho[4]);
          if (zp) face(e ? zb[1].y : zb[1].x, e ? zn[1].y : zn[1].x); else dface(op.rho[5]);
          const float uc0 = e ? U.y : U.x, fc0 = e ? F.y : F.x;
          float r = fc0 - fmaf(fmaf(d, op.ih2, alpha), uc0, -o * op.ih2);
          if ((VB && hc < 0.0f) || (e == 1 && !has1)) r = 0.0f;
          if (e == 0) acc0 += r; else acc1 += r;
        }
      }
  }
  if (!live) return;
  const int cpar = (J + K) & 1;  // colour of coarse X = 2P
  const long long ct = ((long long)K * cny + J) * cW + P;
  sel(fc, cpar)[ct] = 0.125f * acc0;
  sel(uc, cpar)[ct] = 0.0f;
  if (has1) {
    sel(fc, cpar ^ 1)[ct] = 0.125f * acc1;
    sel(uc, cpar ^ 1)[ct] = 0.0f;
  }
}

template <bool VB, bool Vec2>
__global__ void __launch_bounds__(kT, 3) k_resid_restrict(Split32 op, Split32 cop, float alpha,
                                                          Ptr2 f, Ptr2 u, MPtr2 fc, MPtr2 uc) {
  rr_body<VB, Vec2, false>(op, cop, Stk32{}, alpha, f, u, fc, uc);
}

// ---- variable-coefficient restriction with its planes staged by tensor copies
//
// rr_body's residual and restriction (variable coefficient, packed width a
// multiple of 4) for a CTA of 32 coarse pairs x 8 coarse rows that marches
// through kRrZ coarse planes.  The other (black) colour's u and hb arrive
// plane by plane over the CTA's fine window (box 72 x 18: packed 2 P0 - 4 ..
// 2 P0 + 67, a 16-byte start, fine rows 2 J0 - 1 .. 2 J0 + 16) into a ring of
// six slots: a coarse plane K reads fine planes 2K - 1 .. 2K + 2, and the next
// two are in flight.  The own (red) colour's f, u and hb of fine planes 2K and
// 2K + 1 (box 64 x 16) come through a ring of four.  The register-fed kernel
// loads its 36 float2 of a coarse plane into registers (80 registers with
// spills at three CTAs per SM); here they come from shared memory.  Fine
// planes outside the level are not copied (plain arrive: their slots hold
// stale data, which only faces that the boundary tests exclude would read).
// Waits are bounded as in the staged half-sweep (g_sweep_timeout).
constexpr int kRrZ = 16;               // coarse planes per CTA
constexpr int kRrB = 6, kRrW = 4;      // ring slots: black fine planes, own fine planes
constexpr int kRrBX = 72, kRrBY = 18;  // black box
constexpr int kRrBArr = 5248;          // one black array box (72 x 18 x 4 = 5184 bytes), to 128
constexpr int kRrWArr = 4096;          // one own array box (64 x 16 x 4)
constexpr int kRrBSlot = 2 * kRrBArr, kRrWSlot = 3 * kRrWArr;
constexpr int kRrSmem = 128 + kRrB * kRrBSlot + kRrW * kRrWSlot + 8 * (kRrB + kRrW);

struct RrMaps {
  CUtensorMap ub, hb, f, u, ho;  // black u, black hb; own f, own u, own hb
};

__device__ __forceinline__ float2 lds2(const float* p) {
  return *reinterpret_cast<const float2*>(p);
}

__global__ void __launch_bounds__(kT, 2)
    k_resid_restrict_tma(Split32 op, Split32 cop, float alpha, MPtr2 fc, MPtr2 uc,
                         const __grid_constant__ RrMaps maps) {
  extern __shared__ unsigned char rr_smem[];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x, warp = threadIdx.y, tid = warp * 32 + lane;
  const int cny = cop.b.ny, cnx = cop.b.nx, cW = cop.W, cnz = cop.b.nz;
  const int nx = op.b.nx, ny = op.b.ny, nz = op.b.nz;
  const int P0 = blockIdx.x * 32, J0 = blockIdx.y * 8;
  const int Ka = blockIdx.z * kRrZ, Kb = min(cnz, Ka + kRrZ);
  const int nk = Kb - Ka, nq = 2 * nk + 2, nw = 2 * nk;
  const uint32_t base = (tma::smem_addr(rr_smem) + 127u) & ~127u;
  unsigned char* gbase = rr_smem + (base - tma::smem_addr(rr_smem));
  const uint32_t wbase = base + kRrB * kRrBSlot;
  const uint32_t bar0 = wbase + kRrW * kRrWSlot;
  auto bbar = [&](int q) { return bar0 + 8u * (uint32_t)(q % kRrB); };
  auto wbar = [&](int w) { return bar0 + 8u * (uint32_t)(kRrB + w % kRrW); };
  auto bpar = [&](int q) { return (uint32_t)((q / kRrB) & 1); };
  auto wpar = [&](int w) { return (uint32_t)((w / kRrW) & 1); };
  // black sequence q is fine plane 2 Ka - 1 + q; own sequence w is 2 Ka + w
  auto issue_b = [&](int q) {
    const int z = 2 * Ka - 1 + q;
    const uint32_t b = bbar(q);
    if (z < 0 || z >= nz) {
      tma::bar_arrive(b);
      return;
    }
    tma::bar_arrive_tx(b, (uint32_t)(2 * kRrBX * kRrBY * 4));
    const uint32_t d = base + (uint32_t)((q % kRrB) * kRrBSlot);
    tma::load3(d, &maps.ub, b, 2 * P0 - 4, 2 * J0 - 1, z);
    tma::load3(d + kRrBArr, &maps.hb, b, 2 * P0 - 4, 2 * J0 - 1, z);
  };
  auto issue_w = [&](int w) {
    const int z = 2 * Ka + w;
    const uint32_t b = wbar(w);
    tma::bar_arrive_tx(b, (uint32_t)(3 * 64 * 16 * 4));
    const uint32_t d = wbase + (uint32_t)((w % kRrW) * kRrWSlot);
    tma::load3(d, &maps.f, b, 2 * P0, 2 * J0, z);
    tma::load3(d + kRrWArr, &maps.u, b, 2 * P0, 2 * J0, z);
    tma::load3(d + 2 * kRrWArr, &maps.ho, b, 2 * P0, 2 * J0, z);
  };
  auto bslot = [&](int q, int a) {
    return reinterpret_cast<const float*>(gbase + (q % kRrB) * kRrBSlot + a * kRrBArr);
  };
  auto wslot = [&](int w, int a) {
    return reinterpret_cast<const float*>(gbase + kRrB * kRrBSlot + (w % kRrW) * kRrWSlot +
                                          a * kRrWArr);
  };
  int issued_b = min(kRrB, nq), issued_w = min(kRrW, nw);
  if (tid == 0) {
    for (int i = 0; i < kRrB + kRrW; ++i) tma::bar_init(bar0 + 8u * i);
    tma::bar_init_fence();
    for (int q = 0; q < issued_b; ++q) issue_b(q);
    for (int w = 0; w < issued_w; ++w) issue_w(w);
  }
  __syncthreads();
  const int J = J0 + warp, Pl = P0 + lane;
  const bool live = Pl < cW && J < cny;
  const int P = Pl;  // lanes past the level read zero-filled columns and store nothing
  const bool has1 = 2 * P + 1 < cnx;
  bool ok = true;
  for (int i = 0; i < nk; ++i) {
    const int K = Ka + i;
    if (tid == 0 && i >= 1) {
      for (int q = 2 * i + 4; q < 2 * i + 6 && q < nq; ++q) issue_b(issued_b++);
      for (int w = 2 * i + 2; w < 2 * i + 4 && w < nw; ++w) issue_w(issued_w++);
    }
    // black fine planes 2K - 1 .. 2K + 2 are sequences 2i .. 2i + 3; own 2i, 2i + 1
    for (int q = (i == 0 ? 0 : 2 * i + 2); q < 2 * i + 4; ++q)
      ok = tma::bar_wait(bbar(q), bpar(q)) && ok;
    ok = tma::bar_wait(wbar(2 * i), wpar(2 * i)) && ok;
    ok = tma::bar_wait(wbar(2 * i + 1), wpar(2 * i + 1)) && ok;
    if (ok) {
      float acc0 = 0.0f, acc1 = 0.0f;  // coarse X = 2P, 2P+1
      const int col2 = 2 * lane + 4;   // packed 2P in the black box
      float2 UO[4][4], BO[4][4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const bool inner_j = jj == 1 || jj == 2, inner_k = kk == 1 || kk == 2;
          if (!inner_j && !inner_k) continue;
          const int row = 2 * warp + jj;
          UO[jj][kk] = lds2(bslot(2 * i + kk, 0) + row * kRrBX + col2);
          BO[jj][kk] = lds2(bslot(2 * i + kk, 1) + row * kRrBX + col2);
        }
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int j = 2 * J + b, k = 2 * K + c;
          const int s = (b + c) & 1;  // own (red) cells at i = 4P+s, 4P+2+s
          const int orow = (2 * warp + b) * 64 + 2 * lane;
          const float2 F = lds2(wslot(2 * i + c, 0) + orow);
          const float2 U = lds2(wslot(2 * i + c, 1) + orow);
          const float2 HC = lds2(wslot(2 * i + c, 2) + orow);
          const float2 ur = UO[b + 1][c + 1], br = BO[b + 1][c + 1];
          // other colour at packed 2P-1 (s = 0) or 2P+2 (s = 1), from the box
          const float* crow_u = bslot(2 * i + c + 1, 0) + (2 * warp + b + 1) * kRrBX;
          const float* crow_b = bslot(2 * i + c + 1, 1) + (2 * warp + b + 1) * kRrBX;
          const float uh = s ? crow_u[col2 + 2] : crow_u[col2 - 1];
          const float bh = s ? crow_b[col2 + 2] : crow_b[col2 - 1];
          const float ux[3] = {s ? ur.x : uh, s ? ur.y : ur.x, s ? uh : ur.y};
          const float bx[3] = {s ? br.x : bh, s ? br.y : br.x, s ? bh : br.y};
          const float2 yn[2] = {UO[b][c + 1], UO[b + 2][c + 1]};
          const float2 yb[2] = {BO[b][c + 1], BO[b + 2][c + 1]};
          const float2 zn[2] = {UO[b + 1][c], UO[b + 1][c + 2]};
          const float2 zb[2] = {BO[b + 1][c], BO[b + 1][c + 2]};
          const bool ym = j > 0, yp = j < ny - 1, zm = k > 0, zp = k < nz - 1;
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int ic = 4 * P + 2 * e + s;
            const float hc = e ? HC.y : HC.x;
            float d = 0.0f, o = 0.0f;
            auto face = [&](float hn, float un) {
              const float w = wface(hc, hn);
              d += w;
              o = fmaf(w, un, o);
            };
            auto dface = [&](float r) { d = fmaf(wdir(hc), r, d); };
            if (ic > 0) face(bx[e], ux[e]); else dface(op.rho[0]);
            if (ic < nx - 1) face(bx[e + 1], ux[e + 1]); else dface(op.rho[1]);
            if (ym) face(e ? yb[0].y : yb[0].x, e ? yn[0].y : yn[0].x); else dface(op.rho[2]);
            if (yp) face(e ? yb[1].y : yb[1].x, e ? yn[1].y : yn[1].x); else dface(op.rho[3]);
            if (zm) face(e ? zb[0].y : zb[0].x, e ? zn[0].y : zn[0].x); else dface(op.rho[4]);
            if (zp) face(e ? zb[1].y : zb[1].x, e ? zn[1].y : zn[1].x); else dface(op.rho[5]);
            const float uc0 = e ? U.y : U.x, fc0 = e ? F.y : F.x;
            float r = fc0 - fmaf(fmaf(d, op.ih2, alpha), uc0, -o * op.ih2);
            if (hc < 0.0f || (e == 1 && !has1)) r = 0.0f;
            if (e == 0) acc0 += r; else acc1 += r;
          }
        }
      if (live) {
        const int cpar = (J + K) & 1;  // colour of coarse X = 2P
        const long long ct = ((long long)K * cny + J) * cW + P;
        sel(fc, cpar)[ct] = 0.125f * acc0;
        sel(uc, cpar)[ct] = 0.0f;
        if (has1) {
          sel(fc, cpar ^ 1)[ct] = 0.125f * acc1;
          sel(uc, cpar ^ 1)[ct] = 0.0f;
        }
      }
    }
    // the slots of black planes 2K - 1, 2K and own planes 2K, 2K + 1 are free
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }
  }
  (void)FULL;
  if (!ok && tid == 0) {
    atomicExch(&g_sweep_timeout, 1u);
    for (int q = max(0, issued_b - kRrB); q < issued_b; ++q) tma::bar_wait(bbar(q), bpar(q));
    for (int w = max(0, issued_w - kRrW); w < issued_w; ++w) tma::bar_wait(wbar(w), wpar(w));
  }
}

template <bool Vec2>
__global__ void __launch_bounds__(kT, 3) k_resid_restrict_stk(Split32 op, Split32 cop, Stk32 st,
                                                              Ptr2 f, Ptr2 u, MPtr2 fc,
                                                              MPtr2 uc) {
  rr_body<false, Vec2, true>(op, cop, st, 0.0f, f, u, fc, uc);
}


// u_fine += trilinear (27, 9, 3, 1)/64 interpolation of the coarse
// correction; electrode cells untouched.  The interpolation is separable:
// each fine row (2J+b, 2K+c) first blends the coarse rows J, J +- 1 and
// planes K, K +- 1 into a line L(X) (weights 3/4 and 1/4 per axis), then
// fine cell 2X+s takes 3/4 L(X) + 1/4 L(X -+ 1).  Across a domain face the
// coarse neighbour is the ghost of the homogeneous face condition, the cell
// inside times 1 - 2 rho: -1 for Dirichlet (the correction vanishes on the
// face), +1 for Neumann, (1 - ah/2)/(1 + ah/2) for Robin.
//
// One thread per coarse packed pair P of a coarse row (J, K): the coarse
// cells X = 2P and 2P+1 sit at packed index P of the two colour arrays, so
// each of the 9 coarse rows costs one coalesced load per colour.  The thread
// writes fine cells i = 4P..4P+3 of the four fine rows of (J, K), at packed
// positions 2P and 2P+1 of both fine colours.  L(2P-1) and L(2P+2) come from
// the neighbouring lanes; lanes 0 and 31 load that coarse column themselves.
// Block (32, 8) over (P, J), blockIdx.z = K.
// Only black cells are corrected: the post-smoothing (at least one sweep)
// starts with a red half-sweep, which overwrites every red cell without
// reading it.
// Vec2: the fine packed width is even, so the pair (2P, 2P+1) is one float2.
// Tensor maps of the prefetching prolongation: the fine level's black u and
// hb as (W, ny, nz), copied in boxes of 64 packed x 16 rows x 2 planes (the
// fine black cells of one CTA of coarse pairs).
struct ProMaps {
  CUtensorMap ub, hb;
};

// Pre: the fine black rows (and hb) of the CTA are fetched by one tensor copy
// issued before the coarse loads, so their latency overlaps the coarse blend;
// the read-modify-write then reads them from shared memory (pm: the maps).
template <bool VB, bool Vec2, bool Stk, bool Pre = false>
__device__ __forceinline__ void pro_body(const Split32& op, const Split32& cop, const Stk32& st,
                                         Ptr2 ec, MPtr2 u, const ProMaps* pm = nullptr) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x;
  const int P = blockIdx.x * 32 + lane;
  const int J = blockIdx.y * 8 + threadIdx.y, K = blockIdx.z;
  const int cnx = cop.b.nx, cny = cop.b.ny, cW = cop.W;
  __shared__ __align__(128) float sfine[Pre ? (VB ? 2 : 1) : 1][Pre ? 2 : 1][Pre ? 16 : 1]
                                       [Pre ? 64 : 1];
  __shared__ __align__(8) unsigned long long pbar;
  if (Pre) {
    // thread 0 starts the copy of this CTA's fine black tile before anything else
    const uint32_t bar = tma::smem_addr(&pbar);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      tma::bar_init(bar);
      tma::bar_init_fence();
      tma::bar_arrive_tx(bar, (uint32_t)((VB ? 2 : 1) * 64 * 16 * 2 * 4));
      const int x0 = 2 * (int)blockIdx.x * 32, y0 = 2 * (int)blockIdx.y * 8, z0 = 2 * K;
      tma::load3(tma::smem_addr(&sfine[0][0][0][0]), &pm->ub, bar, x0, y0, z0);
      if (VB) tma::load3(tma::smem_addr(&sfine[VB ? 1 : 0][0][0][0]), &pm->hb, bar, x0, y0, z0);
    }
    __syncthreads();  // the barrier is initialised before anyone waits on it
  }
  // stacked level: problem sq owns coarse planes [kc0, kc1)
  const int cnz = Stk ? st.nzp / 2 : cop.b.nz;
  const int sq = sprob<Stk>(st, K, cnz);
  if (J >= cny || !sactive<Stk>(st, sq)) return;  // whole warp
  const int kc0 = sq * cnz, kc1 = kc0 + cnz;
  const bool live = P < cW;
  const bool has1 = 2 * P + 1 < cnx;
  // coarse rows J-1, J, J+1 and planes K-1, K, K+1 (reflected at the faces)
  const int Jr[3] = {J > 0 ? J - 1 : J, J, J < cny - 1 ? J + 1 : J};
  const int Kr[3] = {K > kc0 ? K - 1 : K, K, K < kc1 - 1 ? K + 1 : K};
  // ghost factors 1 - 2 rho of the coarse level's faces
  const float wJm = 0.25f * (J > 0 ? 1.0f : 1.0f - 2.0f * cop.rho[2]);
  const float wJp = 0.25f * (J < cny - 1 ? 1.0f : 1.0f - 2.0f * cop.rho[3]);
  const float wKm = 0.25f * (K > kc0 ? 1.0f : 1.0f - 2.0f * cop.rho[4]);
  const float wKp = 0.25f * (K < kc1 - 1 ? 1.0f : 1.0f - 2.0f * cop.rho[5]);
  const float sXm = 1.0f - 2.0f * cop.rho[0], sXp = 1.0f - 2.0f * cop.rho[1];

  // z blend of the three rows: Z[c][y] for c = 0 (towards K-1), 1 (K+1);
  // x = 0: coarse X = 2P, x = 1: X = 2P+1
  float Z[2][2][3];
#pragma unroll
  for (int y = 0; y < 3; ++y) {
    float e[3][2];
#pragma unroll
    for (int z = 0; z < 3; ++z) {
      const int par = (Jr[y] + Kr[z]) & 1;  // colour of coarse X = 2P
      const long long row = ((long long)Kr[z] * cny + Jr[y]) * cW + P;
      e[z][0] = live ? sel(ec, par)[row] : 0.0f;
      e[z][1] = (live && has1) ? sel(ec, par ^ 1)[row] : 0.0f;
    }
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      const float m = 0.75f * e[1][x];
      Z[0][x][y] = fmaf(wKm, e[0][x], m);
      Z[1][x][y] = fmaf(wKp, e[2][x], m);
    }
  }
  // lines L[b][c][x] of the four fine rows (2J+b, 2K+c)
  float L[2][2][2];
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      const float m = 0.75f * Z[c][x][1];
      L[0][c][x] = fmaf(wJm, Z[c][x][0], m);
      L[1][c][x] = fmaf(wJp, Z[c][x][2], m);
    }
  // L at X = 2P-1 (previous lane's X = 2P+1) and X = 2P+2 (next lane's 2P)
  float Lm[2][2], Lp[2][2];
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      Lm[b][c] = __shfl_up_sync(FULL, L[b][c][1], 1);
      Lp[b][c] = __shfl_down_sync(FULL, L[b][c][0], 1);
    }
  const bool halo_m = lane == 0 && live && P > 0;
  const bool halo_p = lane == 31 && live && 2 * P + 2 < cnx;
  if (halo_m || halo_p) {
    // the coarse column X = 2P-1 (colour of X = 2P flipped, packed P-1) or
    // X = 2P+2 (colour of X = 2P, packed P+1), blended like the others
    const int dp = halo_m ? -1 : 1;
    const int flip = halo_m ? 1 : 0;
    float Zh[2][3];
#pragma unroll
    for (int y = 0; y < 3; ++y) {
      float e[3];
#pragma unroll
      for (int z = 0; z < 3; ++z) {
        const int par = ((Jr[y] + Kr[z]) & 1) ^ flip;
        e[z] = sel(ec, par)[((long long)Kr[z] * cny + Jr[y]) * cW + P + dp];
      }
      const float m = 0.75f * e[1];
      Zh[0][y] = fmaf(wKm, e[0], m);
      Zh[1][y] = fmaf(wKp, e[2], m);
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float m = 0.75f * Zh[c][1];
      const float h0 = fmaf(wJm, Zh[c][0], m), h1 = fmaf(wJp, Zh[c][2], m);
      if (halo_m) { Lm[0][c] = h0; Lm[1][c] = h1; }
      else { Lp[0][c] = h0; Lp[1][c] = h1; }
    }
  }
  if (!live) return;
  const int ny = op.b.ny, W = op.W;
  float* ub = u.p[1];           // black cells only
  const float* hb = op.beta[1];
  // the four fine rows' black pairs (and their hb) are all read before any
  // is written, so the four read-modify-writes overlap
  long long t[2][2];
  float2 w[2][2], g[2][2];
  if (Pre && !tma::bar_wait(tma::smem_addr(&pbar), 0u)) {
    atomicExch(&g_sweep_timeout, 1u);  // the copy never arrived: leave the cells
    return;
  }
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      t[b][c] = ((long long)(2 * K + c) * ny + (2 * J + b)) * W + 2 * P;
      if (Pre) {
        const int row = 2 * (int)threadIdx.y + b;
        w[b][c] = *reinterpret_cast<const float2*>(&sfine[0][c][row][2 * lane]);
        if (VB) g[b][c] = *reinterpret_cast<const float2*>(&sfine[VB ? 1 : 0][c][row][2 * lane]);
      } else if (Vec2) {
        w[b][c] = *reinterpret_cast<const float2*>(ub + t[b][c]);
        if (VB) g[b][c] = *reinterpret_cast<const float2*>(hb + t[b][c]);
      } else {
        w[b][c] = make_float2(ub[t[b][c]], has1 ? ub[t[b][c] + 1] : 0.0f);
        if (VB) g[b][c] = make_float2(hb[t[b][c]], has1 ? hb[t[b][c] + 1] : 0.0f);
      }
    }
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float L0 = L[b][c][0], L1 = L[b][c][1];
      const float lm = P == 0 ? sXm * L0 : Lm[b][c];           // L(2P-1)
      const float lx = has1 ? L1 : sXp * L0;                    // L(2P+1)
      const float lp = 2 * P + 2 >= cnx ? sXp * L1 : Lp[b][c];  // L(2P+2)
      // colour pi = (b + c) & 1 holds fine cells 4P, 4P+2 of this row and
      // colour pi^1 holds 4P+1, 4P+3
      const bool even = ((b + c) & 1) == 1;  // black holds 4P and 4P+2
      const float a0 = even ? fmaf(0.25f, lm, 0.75f * L0) : fmaf(0.25f, lx, 0.75f * L0);
      const float a1 = even ? fmaf(0.25f, L0, 0.75f * L1) : fmaf(0.25f, lp, 0.75f * L1);
      float2 v = w[b][c];
      if (!(VB && g[b][c].x < 0.0f)) v.x += a0;
      if (!(VB && g[b][c].y < 0.0f)) v.y += a1;
      if (Vec2) {
        *reinterpret_cast<float2*>(ub + t[b][c]) = v;
      } else {
        ub[t[b][c]] = v.x;
        if (has1) ub[t[b][c] + 1] = v.y;
      }
    }
}

template <bool VB, bool Vec2>
__global__ void __launch_bounds__(kT) k_prolong(Split32 op, Split32 cop, Ptr2 ec, MPtr2 u) {
  pro_body<VB, Vec2, false>(op, cop, Stk32{}, ec, u);
}

template <bool Vec2>
__global__ void __launch_bounds__(kT) k_prolong_stk(Split32 op, Split32 cop, Stk32 st, Ptr2 ec,
                                                    MPtr2 u) {
  pro_body<false, Vec2, true>(op, cop, st, ec, u);
}

template <bool VB>
__global__ void __launch_bounds__(kT) k_prolong_tma(Split32 op, Split32 cop, Ptr2 ec, MPtr2 u,
                                                    const __grid_constant__ ProMaps maps) {
  pro_body<VB, true, false, true>(op, cop, Stk32{}, ec, u, &maps);
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

// A colour array of the level as a (W, ny, nz) FP32 tensor.
bool colour_map(CUtensorMap* m, const float* p, const Split32& op, int bx, int by) {
  return tma_map_f32(m, p, op.W, op.b.ny, op.b.nz, bx, by);
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

// The staged half-sweeps' shared-memory limits, set once (contexts call this
// on creation, outside any graph capture).
bool sweep_kernels_ready() {
  static const bool ok = [] {
    return cudaFuncSetAttribute(k_half_sweep_tma<true, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                TmaPlan<true>::smem()) == cudaSuccess &&
           cudaFuncSetAttribute(k_half_sweep_tma<true, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                TmaPlan<true>::smem()) == cudaSuccess &&
           cudaFuncSetAttribute(k_half_sweep_tma<false, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                TmaPlan<false>::smem()) == cudaSuccess &&
           cudaFuncSetAttribute(k_half_sweep_tma<false, false, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                TmaPlan<false>::smem()) == cudaSuccess &&
           cudaFuncSetAttribute(k_resid_restrict_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kRrSmem) == cudaSuccess;
  }();
  return ok;
}

namespace {

// The staged half-sweep where it applies (not the first half-sweep from
// zero, W a multiple of 4 and at least one 128-entry tile, 16-byte aligned
// arrays, tensor maps encodable); false otherwise (nothing launched).
bool try_half_sweep_tma(const Split32& op, float alpha, int col, const float* f, float* u,
                        const float* uo, bool has_mask, int zchunk, cudaStream_t s,
                        const Stk32* stk) {
  const bool vb = op.beta[0] != nullptr;
  if (zchunk < 0 || op.b.nx % 8 != 0 || op.W < 128) return false;
  const long long tiles = (long long)((op.W + 127) / 128) * ((op.b.ny + 7) / 8);
  const long long nbz = stk ? stk->nb : 1, nzl = stk ? stk->nzp : op.b.nz;
  auto ctas = [&](int z) { return tiles * nbz * ((nzl + z - 1) / z); };
  int zc = zchunk;
  if (zc == 0) {
    // about four CTAs per slot of the GPU (152 SMs x 3 CTAs), else two;
    // below that the register-fed kernel (one plane per CTA) fills it better
    constexpr long long kSlots = 152 * 3;
    zc = ctas(32) >= 4 * kSlots ? 32 : ctas(16) >= 4 * kSlots ? 16 : 8;
    if (ctas(zc) < 2 * kSlots) return false;
  }
  if (!aligned16(f) || !aligned16(u) || !aligned16(uo)) return false;
  if (vb && (!aligned16(op.beta[0]) || !aligned16(op.beta[1]))) return false;
  SweepMaps maps;
  if (!colour_map(&maps.uo, uo, op, kOX, kOY) || !colour_map(&maps.f, f, op, 128, 8)) return false;
  if (vb) {
    if (!colour_map(&maps.bo_other, bsel_h(op, col ^ 1), op, kOX, kOY) ||
        !colour_map(&maps.bo_own, bsel_h(op, col), op, 128, 8))
      return false;
  } else {
    maps.bo_other = maps.uo;
    maps.bo_own = maps.f;
  }
  if (!sweep_kernels_ready()) return false;
  dim3 blk(32, 8), g((op.W + 127) / 128, (op.b.ny + 7) / 8,
                    (unsigned)(nbz * ((nzl + zc - 1) / zc)));
  const Stk32 st = stk ? *stk : Stk32{};
  auto go = [&](auto kern, int smem) { kern<<<g, blk, smem, s>>>(op, st, alpha, col, zc, u, maps); };
  if (stk) {
    if (vb || has_mask) return false;  // stacks are constant-coefficient
    go(k_half_sweep_tma<false, false, true>, TmaPlan<false>::smem());
  } else if (vb) {
    if (has_mask) go(k_half_sweep_tma<true, true>, TmaPlan<true>::smem());
    else go(k_half_sweep_tma<true, false>, TmaPlan<true>::smem());
  } else {
    go(k_half_sweep_tma<false, false>, TmaPlan<false>::smem());
  }
  return true;
}

// The staged restriction where it applies (variable coefficient, packed width
// a multiple of 4 and at least 128, 16-byte aligned arrays, encodable maps);
// false otherwise (nothing launched).
bool try_resid_restrict_tma(const Split32& op, const Split32& cop, float alpha, Ptr2 f, Ptr2 u,
                            MPtr2 fc, MPtr2 uc, cudaStream_t s) {
  if (!op.beta[0] || op.W % 4 != 0 || op.W < 128 || op.b.nx % 8 != 0 || !sweep_kernels_ready())
    return false;
  RrMaps m;
  if (!colour_map(&m.ub, u.p[1], op, kRrBX, kRrBY) ||
      !colour_map(&m.hb, op.beta[1], op, kRrBX, kRrBY) || !colour_map(&m.f, f.p[0], op, 64, 16) ||
      !colour_map(&m.u, u.p[0], op, 64, 16) || !colour_map(&m.ho, op.beta[0], op, 64, 16))
    return false;
  dim3 blk(32, 8), g((cop.W + 31) / 32, (cop.b.ny + 7) / 8, (cop.b.nz + kRrZ - 1) / kRrZ);
  k_resid_restrict_tma<<<g, blk, kRrSmem, s>>>(op, cop, alpha, fc, uc, m);
  return true;
}

}  // namespace

// cuTensorMapEncodeTiled, fetched from the driver once (null if absent).
static PFN_cuTensorMapEncodeTiled_v12000 tma_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

bool tma_map_f32(CUtensorMap* m, const void* p, long long nx, long long ny, long long nz, int bx,
                 int by, int bz) {
  if (!tma_encoder() || ((uintptr_t)p & 15u) || (nx * 4) % 16) return false;
  const cuuint64_t dim[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t stride[2] = {(cuuint64_t)nx * 4, (cuuint64_t)(nx * ny * 4)};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
  const cuuint32_t es[3] = {1, 1, 1};
  return tma_encoder()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(p), dim, stride,
                       box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool sweep_timed_out() {
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, g_sweep_timeout, sizeof(v)) != cudaSuccess) return false;
  if (v) {
    const unsigned zero = 0;
    cudaMemcpyToSymbol(g_sweep_timeout, &zero, sizeof(zero));
  }
  return v != 0;
}

void launch_half_sweep32(const Split32& op, float alpha, int col, const float* f, float* u,
                         const float* uo, bool zero_other, bool has_mask, int zchunk,
                         cudaStream_t s, const Stk32* stk) {
  const bool vb = op.beta[0] != nullptr;
  if (!zero_other && try_half_sweep_tma(op, alpha, col, f, u, uo, has_mask, zchunk, s, stk)) {
    add_launches(1);
    return;
  }
  dim3 blk(32, 8);
  if (stk) {  // a stack of constant-coefficient problems
    const Stk32 st = *stk;
    if (op.b.nx % 8 == 0) {
      dim3 g((op.W / 4 + 31) / 32, (op.b.ny + 7) / 8, op.b.nz);
      if (zero_other) k_half_sweep_v4_stk<true><<<g, blk, 0, s>>>(op, st, col, f, u, uo);
      else k_half_sweep_v4_stk<false><<<g, blk, 0, s>>>(op, st, col, f, u, uo);
    } else {
      dim3 g((op.W + 31) / 32, (op.b.ny + 7) / 8, op.b.nz);
      if (zero_other) k_half_sweep_stk<true><<<g, blk, 0, s>>>(op, st, col, f, u, uo);
      else k_half_sweep_stk<false><<<g, blk, 0, s>>>(op, st, col, f, u, uo);
    }
    add_launches(1);
    return;
  }
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
                              MPtr2 fc, MPtr2 uc, cudaStream_t s, const Stk32* stk) {
  dim3 blk(32, 8), g((cop.W + 31) / 32, (cop.b.ny + 7) / 8, cop.b.nz);
  const bool vec2 = op.W % 2 == 0;
  if (!stk && try_resid_restrict_tma(op, cop, alpha, f, u, fc, uc, s)) {
    add_launches(1);
    return;
  }
  if (stk) {
    if (vec2) k_resid_restrict_stk<true><<<g, blk, 0, s>>>(op, cop, *stk, f, u, fc, uc);
    else k_resid_restrict_stk<false><<<g, blk, 0, s>>>(op, cop, *stk, f, u, fc, uc);
    add_launches(1);
    return;
  }
#define RR(A, B) k_resid_restrict<A, B><<<g, blk, 0, s>>>(op, cop, alpha, f, u, fc, uc)
  if (op.beta[0]) { if (vec2) RR(true, true); else RR(true, false); }
  else { if (vec2) RR(false, true); else RR(false, false); }
#undef RR
  add_launches(1);
}

void launch_prolong32s(const Split32& op, const Split32& cop, Ptr2 ec, MPtr2 u, cudaStream_t s,
                       const Stk32* stk) {
  // the fine black tile of a CTA by one tensor copy ahead of the coarse blend
  if (!stk && op.W % 4 == 0 && op.W >= 128 && op.b.nx % 8 == 0) {
    ProMaps m;
    const bool vbp = op.beta[0] != nullptr;
    if (tma_map_f32(&m.ub, u.p[1], op.W, op.b.ny, op.b.nz, 64, 16, 2) &&
        (!vbp || tma_map_f32(&m.hb, op.beta[1], op.W, op.b.ny, op.b.nz, 64, 16, 2))) {
      if (!vbp) m.hb = m.ub;
      dim3 blk(32, 8), g((cop.W + 31) / 32, (cop.b.ny + 7) / 8, cop.b.nz);
      if (vbp) k_prolong_tma<true><<<g, blk, 0, s>>>(op, cop, ec, u, m);
      else k_prolong_tma<false><<<g, blk, 0, s>>>(op, cop, ec, u, m);
      add_launches(1);
      return;
    }
  }
  dim3 blk(32, 8), g((cop.W + 31) / 32, (cop.b.ny + 7) / 8, cop.b.nz);
  const bool vec2 = op.W % 2 == 0;
  if (stk) {
    if (vec2) k_prolong_stk<true><<<g, blk, 0, s>>>(op, cop, *stk, ec, u);
    else k_prolong_stk<false><<<g, blk, 0, s>>>(op, cop, *stk, ec, u);
    add_launches(1);
    return;
  }
#define PRO(A, B) k_prolong<A, B><<<g, blk, 0, s>>>(op, cop, ec, u)
  if (op.beta[0]) { if (vec2) PRO(true, true); else PRO(true, false); }
  else { if (vec2) PRO(false, true); else PRO(false, false); }
#undef PRO
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
