// Iterative-refinement step of the mixed-precision solve:
//
//     u_new = u + e            (FP32 correction from the inner V-cycle)
//     r     = b - A u_new      (b = rhs * scale + Dirichlet lifts)
//     r32   = (float) r        (right-hand side of the next inner V-cycle)
//     ||r||^2 partial sums per CTA
//
// in one pass.  The operator and lifts follow Sec. 2 items (ii)-(iii) of
// arXiv:1809.08857 (second-order cell-centred finite volumes for Eqs. 2-3).
//
// u, b and the operator are FP64 data, but the arithmetic of r is done in
// double-float (pairs of FP32 numbers, 48 significant bits): on GB300 the
// FP64 pipe issues about 1/57 of the FP32 rate, and an FP64 stencil of about
// ten operations per cell left this pass at 20 % of the HBM bandwidth.  The
// iterate itself is kept as double-floats during a solve, so no FP64
// instruction is left per cell.  Each thread marches one (i, j) column of a
// z-chunk with its planes in registers; y-neighbours go through shared
// memory, x-neighbours through warp shuffles.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/mg.h"
#include "df.cuh"
#include <algorithm>

#include "mg_internal.h"
#include "tma.cuh"

// Largest number of CTAs (partial sums) one call may use: 16384 doubles,
// 128 KiB.  Every GPU that loads libmg holds this array until process exit.
#define MG_NOALLOC_MAX_PARTIALS 16384

static __device__ __align__(256) double g_noalloc_scratch[MG_NOALLOC_MAX_PARTIALS];

namespace mg {

namespace {

using namespace df;

constexpr int TX = 32, TY = 16, NT = TX * TY;  // a CTA's patch of columns (own: inner 30 x 14)

// Template arguments:
//   Faces   variable-coefficient operator (double-float face arrays);
//           otherwise beta = 1
//   HasE    the iterate is udf_in + e (a refinement step)
//   U64     the iterate is the FP64 array u_in (split on load); otherwise
//           the double-float array udf_in
//   BIn     0: b = bdf (double-float); 1: b = rhs (FP64); 2: b = rhs *
//           rhs_scale + Dirichlet lifts, formed here in FP64
//   ZNorm   also the norm of the residual of the guess that is 0 on free
//           cells and u on electrode cells (||b|| of the stopping test),
//           into partial_z
// A CTA of 32 x 16 threads covers a 32 x 16 patch of (i, j) columns, of
// which the inner 30 x 14 are its own cells and the rim is the halo.  Every
// thread marches its column along z with u + e of planes k-1, k, k+1 in
// registers (the z-neighbours), its raw loads of plane k+2 in flight; each
// plane's u + e goes through a double-buffered shared-memory plane for the
// y-neighbours, and the x-neighbours come from the adjacent lanes (a warp
// is one row) by shuffle.  One barrier per plane.
template <bool Faces, bool HasE, bool U64, int BIn, bool ZNorm>
__global__ void __launch_bounds__(NT, Faces ? 2 : 3) k_ir_df(IrArgs a) {
  __shared__ float2 pl[2][TY][TX];
  __shared__ unsigned char mk[ZNorm ? 2 : 1][ZNorm ? TY : 1][TX];  // electrode flags
  __shared__ float red[2][NT / 32];
  const unsigned FULL = 0xffffffffu;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int nx = a.op.b.nx, ny = a.op.b.ny, nz = a.op.b.nz;
  const int i = blockIdx.x * (TX - 2) - 1 + tx, j = blockIdx.y * (TY - 2) - 1 + ty;
  const int z0 = blockIdx.z * a.zchunk, z1 = min(nz, z0 + a.zchunk);
  const int W = a.W;
  const long long sz = (long long)nx * ny, szW = (long long)W * ny;
  const bool in = i >= 0 && i < nx && j >= 0 && j < ny;
  const bool own = in && tx >= 1 && tx <= TX - 2 && ty >= 1 && ty <= TY - 2;
  const int off = in ? j * nx + i : 0;        // in-plane offsets of the column
  const int eoff = in ? j * W + (i >> 1) : 0;
  const int par0 = (i + j) & 1;               // colour of the column at k = 0
  const bool zmask = ZNorm && a.op.mask != nullptr;
  const bool xm = i > 0, xp = i < nx - 1, ym = j > 0, yp = j < ny - 1;
  // beta = 1: diagonal (in-box faces + 2 rho per domain face) / h^2 +
  // alpha; interior cells use the launcher's double-float 6/h^2 + alpha,
  // boundary cells form theirs in FP64
  double dxy = 0.0;
  if (!Faces) {
    dxy += xm ? 1.0 : 2.0 * a.op.rho[0];
    dxy += xp ? 1.0 : 2.0 * a.op.rho[1];
    dxy += ym ? 1.0 : 2.0 * a.op.rho[2];
    dxy += yp ? 1.0 : 2.0 * a.op.rho[3];
  }
  const bool xy_in = xm && xp && ym && yp;

  // ---- the column: raw loads of a plane (fetch) and u + e (combine)
  double rd = 0.0;
  float2 ru = make_float2(0.0f, 0.0f);
  float re = 0.0f;
  bool rm = false;
  auto fetch = [&](int k) {
    if (!(in && k >= 0 && k < nz)) return;
    const long long c = (long long)k * sz + off;
    if (zmask) rm = a.op.mask[c] != 0;
    if (U64) {
      rd = a.u_in[c];
      if (a.in_scale != 1.0) rd *= a.in_scale;
    } else {
      ru = a.udf_in[c];
      if (HasE) {
        const long long t = (long long)k * szW + eoff;
        re = ((par0 + k) & 1) ? a.e[1][t] : a.e[0][t];
      }
    }
  };
  auto combine = [&](int k, float2& v, bool& m) {
    v = make_float2(0.0f, 0.0f);
    m = false;
    if (!(in && k >= 0 && k < nz)) return;
    v = U64 ? split_df(rd) : (HasE ? df_add(ru, re) : ru);
    m = rm;
  };

  // ---- own cell of a plane: b, electrode flag, coefficients
  struct Cell {
    double bd;
    float2 bb, dg, cxm, cxp, cym, cyp, czm, czp;
    bool m;
  };
  auto cell_fetch = [&](int k, Cell& C) {
    if (!own || k >= z1) return;
    const long long c = (long long)k * sz + off;
    if (Faces) {
      C.dg = a.op.Dd[c];
      const float2* cx = a.op.cxd + c;
      const float2* cy = a.op.cyd + c;
      const float2* cz = a.op.czd + c;
      C.cxm = cx[0];
      if (xp) C.cxp = cx[1];
      C.cym = cy[0];
      if (yp) C.cyp = cy[nx];
      C.czm = cz[0];
      if (k < nz - 1) C.czp = cz[sz];
    } else {
      C.m = a.op.mask && a.op.mask[c];
    }
    if (BIn == 0) C.bb = a.bdf[c];
    else C.bd = a.in_scale != 1.0 ? a.rhs[c] * a.in_scale : a.rhs[c];
  };

  float2 um, uc, up;
  bool mm, mc, mp;
  fetch(z0 - 1);
  combine(z0 - 1, um, mm);
  fetch(z0);
  combine(z0, uc, mc);
  fetch(z0 + 1);
  combine(z0 + 1, up, mp);
  fetch(z0 + 2);
  Cell C{}, Cn{};
  cell_fetch(z0, C);
  float ss = 0.0f, sz2 = 0.0f;
  for (int k = z0; k < z1; ++k) {
    const int buf = (k - z0) & 1;
    pl[buf][ty][tx] = uc;
    if (ZNorm) mk[buf][ty][tx] = mc;
    const long long c = (long long)k * sz + off;
    if (own && a.udf_out) a.udf_out[c] = uc;
    cell_fetch(k + 1, Cn);
    __syncthreads();
    // x-neighbours from the adjacent lanes of the row
    float2 ul, ur;
    ul.x = __shfl_up_sync(FULL, uc.x, 1);
    ul.y = __shfl_up_sync(FULL, uc.y, 1);
    ur.x = __shfl_down_sync(FULL, uc.x, 1);
    ur.y = __shfl_down_sync(FULL, uc.y, 1);
    const bool ml = __shfl_up_sync(FULL, mc, 1), mr = __shfl_down_sync(FULL, mc, 1);
    if (own) {
      float r = 0.0f, rz = 0.0f;
      const bool m = Faces ? C.dg.x < 0.0f : C.m;
      float2 bb;
      if (BIn == 0) {
        bb = C.bb;
      } else {
        double bd = C.bd;
        if (BIn == 2) {
          bd *= a.rhs_scale;
          const bool edge = !xy_in || k == 0 || k == nz - 1;
          if (a.lift && edge && !m) {
            const double l = 2.0 * (a.beta0 ? a.beta0[c] : 1.0) * a.op.ih2;
            if (!xm && a.op.rho[0] == 1.0) bd += l * a.bval.v[0];
            if (!xp && a.op.rho[1] == 1.0) bd += l * a.bval.v[1];
            if (!ym && a.op.rho[2] == 1.0) bd += l * a.bval.v[2];
            if (!yp && a.op.rho[3] == 1.0) bd += l * a.bval.v[3];
            if (k == 0 && a.op.rho[4] == 1.0) bd += l * a.bval.v[4];
            if (k == nz - 1 && a.op.rho[5] == 1.0) bd += l * a.bval.v[5];
          }
        }
        bb = split_df(bd);
        if (a.bdf_out) a.bdf_out[c] = bb;
      }
      if (!m) {
        DfAcc acc{bb.x, bb.y};
        DfAcc az{bb.x, bb.y};  // zero guess: only electrode neighbours contribute
        const bool zm = k > 0, zp = k < nz - 1;
        float2 dg;
        if (Faces) {
          dg = C.dg;
          if (a.has_alpha) acc.add(a.nalpha, uc);
        } else if (xy_in && zm && zp) {
          dg = a.dint;
        } else {
          const double d = dxy + (zm ? 1.0 : 2.0 * a.op.rho[4]) + (zp ? 1.0 : 2.0 * a.op.rho[5]);
          dg = split_df(fma(d, a.op.ih2, a.alpha));
        }
        acc.add(make_float2(-dg.x, -dg.y), uc);
        auto nb = [&](bool inb, float2 w, float2 v, bool mk_) {
          if (!inb) return;
          acc.add(w, v);
          if (zmask && mk_) az.add(w, v);
        };
        const float2 us = pl[buf][ty - 1][tx], un = pl[buf][ty + 1][tx];
        const bool ms = ZNorm && mk[buf][ty - 1][tx], mn = ZNorm && mk[buf][ty + 1][tx];
        if (Faces) {
          nb(xm, C.cxm, ul, ml);
          nb(xp, C.cxp, ur, mr);
          nb(ym, C.cym, us, ms);
          nb(yp, C.cyp, un, mn);
          nb(zm, C.czm, um, mm);
          nb(zp, C.czp, up, mp);
        } else {
          const float2 w = a.ih2d;
          nb(xm, w, ul, ml);
          nb(xp, w, ur, mr);
          nb(ym, w, us, ms);
          nb(yp, w, un, mn);
          nb(zm, w, um, mm);
          nb(zp, w, up, mp);
        }
        r = acc.value();
        rz = az.value();
      }
      if (a.r[0]) (((par0 + k) & 1) ? a.r[1] : a.r[0])[(long long)k * szW + eoff] = r;
      ss = fmaf(r, r, ss);
      if (ZNorm) sz2 = fmaf(rz, rz, sz2);
    }
    // advance the column: plane k+2 (loaded last step) becomes k+1
    um = uc;
    mm = mc;
    uc = up;
    mc = mp;
    combine(k + 2, up, mp);
    if (k + 3 <= z1) fetch(k + 3);
    C = Cn;
  }
  // CTA sums of r^2 (FP32 is ample for a stopping test; the partials and the
  // final sum are accumulated in FP64)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ss += __shfl_xor_sync(FULL, ss, o);
    if (ZNorm) sz2 += __shfl_xor_sync(FULL, sz2, o);
  }
  if (tx == 0) {
    red[0][ty] = ss;
    if (ZNorm) red[1][ty] = sz2;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const long long cta = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
#pragma unroll
    for (int h = 0; h < (ZNorm ? 2 : 1); ++h) {
      double v = threadIdx.x < NT / 32 ? (double)red[h][threadIdx.x] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
      if (threadIdx.x == 0) (h ? a.partial_z : a.partial)[cta] = v;
    }
  }
}

// The same pass for the constant-coefficient operator (beta = 1) with two
// x-adjacent cells per thread, the pair (i0, i0 + 1) with i0 even (cell A,
// cell B): every double-float operation of the pair is one FP32x2
// instruction (DfAcc2, df_add2), the x-neighbours of the pair are two
// shuffles (B of the previous lane, A of the next), a thread's plane entry in
// shared memory is one 16-byte word.  Needs nx even and 16-byte aligned
// arrays (the launcher checks and otherwise runs k_ir_df).  A CTA of 32 x 16
// threads covers 64 x 16 columns, of which the inner 60 x 14 are its own.
// Template arguments as for k_ir_df (no Faces, no ZNorm: the first pass of
// a solve runs k_ir_df).
template <bool HasE, bool U64, int BIn>
__global__ void __launch_bounds__(NT, 2) k_ir_df2(IrArgs a) {
  __shared__ float4 pl[2][TY][TX];
  __shared__ float red[NT / 32];
  const unsigned FULL = 0xffffffffu;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int nx = a.op.b.nx, ny = a.op.b.ny, nz = a.op.b.nz;
  const int i0 = 2 * (blockIdx.x * (TX - 2) - 1 + tx), j = blockIdx.y * (TY - 2) - 1 + ty;
  const int z0 = blockIdx.z * a.zchunk, z1 = min(nz, z0 + a.zchunk);
  const int W = a.W;
  const long long sz = (long long)nx * ny, szW = (long long)W * ny;
  const bool in = i0 >= 0 && i0 < nx && j >= 0 && j < ny;  // nx even: i0 + 1 < nx as well
  const bool own = in && tx >= 1 && tx <= TX - 2 && ty >= 1 && ty <= TY - 2;
  const int off = in ? j * nx + i0 : 0;  // in-plane offset of cell A
  const int eoff = in ? j * W + (i0 >> 1) : 0;  // packed index of A and of B
  const int par0 = (i0 + j) & 1;                // colour of A at k = 0; B has the other
  const bool xmA = i0 > 0, xpB = i0 + 2 < nx, ym = j > 0, yp = j < ny - 1;
  const float2 zero2 = make_float2(0.0f, 0.0f);
  // beta = 1: the diagonal of each cell of the pair on an interior plane,
  // 4/h^2 for its in-plane in-box faces plus 2 rho/h^2 for its domain faces
  // (A's +x neighbour and B's -x neighbour are each other) plus 2/h^2 + alpha,
  // formed once in FP64 here; the planes k = 0 and nz - 1 add the double-float
  // correction (2 rho - 1)/h^2 of their z face in the loop (FP32 only)
  Df2 dxy;
  if (xmA && xpB && ym && yp) {
    dxy = Df2{make_float2(a.dint.x, a.dint.x), make_float2(a.dint.y, a.dint.y)};
  } else {
    const double dy = (ym ? 1.0 : 2.0 * a.op.rho[2]) + (yp ? 1.0 : 2.0 * a.op.rho[3]);
    const double dA = (xmA ? 1.0 : 2.0 * a.op.rho[0]) + 1.0 + dy + 2.0;
    const double dB = 1.0 + (xpB ? 1.0 : 2.0 * a.op.rho[1]) + dy + 2.0;
    const float2 sA = split_df(fma(dA, a.op.ih2, a.alpha));
    const float2 sB = split_df(fma(dB, a.op.ih2, a.alpha));
    dxy = Df2{make_float2(sA.x, sB.x), make_float2(sA.y, sB.y)};
  }

  // ---- the column pair: raw loads of a plane (fetch) and u + e (combine)
  double2 rd = make_double2(0.0, 0.0);
  Df2 ru{zero2, zero2};
  float2 re = zero2;
  auto fetch = [&](int k) {
    if (!(in && k >= 0 && k < nz)) return;
    const long long c = (long long)k * sz + off;
    if (U64) {
      rd = *reinterpret_cast<const double2*>(a.u_in + c);
      if (a.in_scale != 1.0) rd = make_double2(rd.x * a.in_scale, rd.y * a.in_scale);
    } else {
      const float4 v = *reinterpret_cast<const float4*>(a.udf_in + c);
      ru = Df2{make_float2(v.x, v.z), make_float2(v.y, v.w)};
      if (HasE) {
        const long long t = (long long)k * szW + eoff;
        const bool ca = (par0 + k) & 1;
        re = make_float2(ca ? a.e[1][t] : a.e[0][t], ca ? a.e[0][t] : a.e[1][t]);
      }
    }
  };
  auto combine = [&](int k, Df2& v) {
    v = Df2{zero2, zero2};
    if (!(in && k >= 0 && k < nz)) return;
    if (U64) {
      const float2 A = split_df(rd.x), B = split_df(rd.y);
      v = Df2{make_float2(A.x, B.x), make_float2(A.y, B.y)};
    } else {
      v = HasE ? df_add2(ru, re) : ru;
    }
  };
  auto pair4 = [](const float4& v) { return Df2{make_float2(v.x, v.z), make_float2(v.y, v.w)}; };

  // ---- own cells of a plane: b and electrode flags
  struct Cell {
    double2 bd;
    Df2 bb;
    uchar2 m;
  };
  auto cell_fetch = [&](int k, Cell& C) {
    if (!own || k >= z1) return;
    const long long c = (long long)k * sz + off;
    C.m = a.op.mask ? *reinterpret_cast<const uchar2*>(a.op.mask + c) : make_uchar2(0, 0);
    if (BIn == 0) C.bb = pair4(*reinterpret_cast<const float4*>(a.bdf + c));
    else C.bd = *reinterpret_cast<const double2*>(a.rhs + c);
    if (BIn != 0 && a.in_scale != 1.0) C.bd = make_double2(C.bd.x * a.in_scale, C.bd.y * a.in_scale);
  };
  // b of one cell formed in FP64 (BIn 1: as given; 2: scaled plus the
  // Dirichlet-face lifts of the cell's domain faces)
  auto form_b = [&](double bd, long long c, bool m, bool xm, bool xp, int k) {
    if (BIn == 2) {
      bd *= a.rhs_scale;
      const bool edge = !(xm && xp && ym && yp) || k == 0 || k == nz - 1;
      if (a.lift && edge && !m) {
        const double l = 2.0 * (a.beta0 ? a.beta0[c] : 1.0) * a.op.ih2;
        if (!xm && a.op.rho[0] == 1.0) bd += l * a.bval.v[0];
        if (!xp && a.op.rho[1] == 1.0) bd += l * a.bval.v[1];
        if (!ym && a.op.rho[2] == 1.0) bd += l * a.bval.v[2];
        if (!yp && a.op.rho[3] == 1.0) bd += l * a.bval.v[3];
        if (k == 0 && a.op.rho[4] == 1.0) bd += l * a.bval.v[4];
        if (k == nz - 1 && a.op.rho[5] == 1.0) bd += l * a.bval.v[5];
      }
    }
    return bd;
  };

  Df2 um, uc, up;
  fetch(z0 - 1);
  combine(z0 - 1, um);
  fetch(z0);
  combine(z0, uc);
  fetch(z0 + 1);
  combine(z0 + 1, up);
  fetch(z0 + 2);
  // the own cells' data of the next plane is fetched one plane ahead
  Cell C{}, Cn{};
  cell_fetch(z0, C);
  float2 ss = zero2;
  for (int k = z0; k < z1; ++k) {
    const int buf = (k - z0) & 1;
    const float4 uc4 = make_float4(uc.hi.x, uc.lo.x, uc.hi.y, uc.lo.y);
    pl[buf][ty][tx] = uc4;
    const long long c = (long long)k * sz + off;
    if (own && a.udf_out) *reinterpret_cast<float4*>(a.udf_out + c) = uc4;
    cell_fetch(k + 1, Cn);
    __syncthreads();
    // x-neighbours: L = (B of the previous lane, own A), R = (own B, A of the
    // next lane)
    const float pbh = __shfl_up_sync(FULL, uc.hi.y, 1), pbl = __shfl_up_sync(FULL, uc.lo.y, 1);
    const float nah = __shfl_down_sync(FULL, uc.hi.x, 1), nal = __shfl_down_sync(FULL, uc.lo.x, 1);
    if (own) {
      const Df2 L{make_float2(pbh, uc.hi.x), make_float2(pbl, uc.lo.x)};
      const Df2 R{make_float2(uc.hi.y, nah), make_float2(uc.lo.y, nal)};
      const bool mA = C.m.x != 0, mB = C.m.y != 0;
      Df2 bb;
      if (BIn == 0) {
        bb = C.bb;
      } else {
        const float2 bA = split_df(form_b(C.bd.x, c, mA, xmA, true, k));
        const float2 bB = split_df(form_b(C.bd.y, c + 1, mB, true, xpB, k));
        bb = Df2{make_float2(bA.x, bB.x), make_float2(bA.y, bB.y)};
        if (a.bdf_out)
          *reinterpret_cast<float4*>(a.bdf_out + c) = make_float4(bA.x, bA.y, bB.x, bB.y);
      }
      DfAcc2 acc{bb.hi, bb.lo};
      const bool zm = k > 0, zp = k < nz - 1;
      Df2 dg = dxy;
      if (!zm) dg = df_add_df2(dg, a.dzm);
      if (!zp) dg = df_add_df2(dg, a.dzp);
      acc.add(Df2{make_float2(-dg.hi.x, -dg.hi.y), make_float2(-dg.lo.x, -dg.lo.y)}, uc);
      const float4 s4 = pl[buf][ty - 1][tx], n4 = pl[buf][ty + 1][tx];
      const Df2 w{make_float2(a.ih2d.x, a.ih2d.x), make_float2(a.ih2d.y, a.ih2d.y)};
      // the six neighbours summed first (none across A's -x or B's +x domain
      // face), then one product by 1/h^2
      DfSum2 nb{make_float2(xmA ? L.hi.x : 0.0f, L.hi.y), make_float2(xmA ? L.lo.x : 0.0f, L.lo.y)};
      nb.add(Df2{make_float2(R.hi.x, xpB ? R.hi.y : 0.0f), make_float2(R.lo.x, xpB ? R.lo.y : 0.0f)});
      if (ym) nb.add(pair4(s4));
      if (yp) nb.add(pair4(n4));
      if (zm) nb.add(um);
      if (zp) nb.add(up);
      acc.add(w, Df2{nb.s, nb.e});
      float2 r = acc.value();
      if (mA) r.x = 0.0f;
      if (mB) r.y = 0.0f;
      if (a.r[0]) {
        const long long t = (long long)k * szW + eoff;
        const bool ca = (par0 + k) & 1;
        (ca ? a.r[1] : a.r[0])[t] = r.x;
        (ca ? a.r[0] : a.r[1])[t] = r.y;
      }
      ss = fma2(r, r, ss);
    }
    // advance the column pair: plane k+2 (loaded last step) becomes k+1
    um = uc;
    uc = up;
    combine(k + 2, up);
    if (k + 3 <= z1) fetch(k + 3);
    C = Cn;
  }
  // CTA sums of r^2 (FP32 per thread, FP64 across the CTA)
  float s1 = ss.x + ss.y;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s1 += __shfl_xor_sync(FULL, s1, o);
  if (tx == 0) red[ty] = s1;
  __syncthreads();
  if (threadIdx.x < 32) {
    const long long cta = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    double v = threadIdx.x < NT / 32 ? (double)red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (threadIdx.x == 0) a.partial[cta] = v;
  }
}

// ---- the two-cell refinement step with its planes staged by tensor copies --
//
// k_ir_df2<HasE=1, U64=0, BIn=0> (a constant-coefficient refinement step
// after the first pass, on a grid without electrode cells) with its inputs
// brought to shared memory by tiled tensor copies instead of register
// prefetches.  Per plane: the CTA's 64 x 16 patch of the double-float iterate
// (box 128 x 16 floats from x = 2 i0, a 16-byte boundary), the 32 packed
// corrections of each colour (box 36 x 16 from the packed start rounded down
// to a multiple of 4 entries; a thread indexes from the remainder) and b of
// the 60 x 14 own cells (box 120 x 14).  The iterate and correction of plane
// k + 2 are combined into registers at the end of plane k from a ring of
// three slots, whose copies are issued two to three planes ahead; b of plane
// k comes from a ring of three.  Everything else (the y-neighbours through
// the shared plane, the x-neighbours by shuffle, the FP32x2 double-float
// arithmetic) is k_ir_df2's.  Waits are bounded (tma::kWaitNs); a CTA that
// gives up sets g_ir_timeout, waits for its own copies and stops.
constexpr int kIrU = 3, kIrB = 3;                  // ring slots
constexpr int kIrUBytes = TY * 4 * TX * 4;         // 16 rows x 128 floats = 8192
constexpr int kIrEBytes = TY * 36 * 4;             // 2304 per colour
constexpr int kIrUSlot = kIrUBytes + 2 * kIrEBytes;  // 12800 = 100 x 128
constexpr int kIrBBytes = (TY - 2) * 120 * 4;      // 6720
constexpr int kIrBSlot = 6784;                     // 53 x 128
constexpr int kIrSmem = 128 + kIrU * kIrUSlot + kIrB * kIrBSlot + 8 * (kIrU + kIrB);

struct IrMaps {
  CUtensorMap u, e0, e1, b;
};

__device__ unsigned g_ir_timeout = 0;

__global__ void __launch_bounds__(NT, 2) k_ir_df2_tma(IrArgs a,
                                                      const __grid_constant__ IrMaps maps) {
  extern __shared__ unsigned char ir_smem[];
  __shared__ float4 pl[2][TY][TX];
  __shared__ float red[NT / 32];
  const unsigned FULL = 0xffffffffu;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int nx = a.op.b.nx, ny = a.op.b.ny, nz = a.op.b.nz;
  const int bx = blockIdx.x, by = blockIdx.y;
  const int i0 = 2 * (bx * (TX - 2) - 1 + tx), j = by * (TY - 2) - 1 + ty;
  const int z0 = blockIdx.z * a.zchunk, z1 = min(nz, z0 + a.zchunk);
  const int n = z1 - z0, nq = n + 2;
  const int W = a.W;
  const long long sz = (long long)nx * ny, szW = (long long)W * ny;
  const bool in = i0 >= 0 && i0 < nx && j >= 0 && j < ny;
  const bool own = in && tx >= 1 && tx <= TX - 2 && ty >= 1 && ty <= TY - 2;
  const int off = in ? j * nx + i0 : 0;
  const int eoff = in ? j * W + (i0 >> 1) : 0;
  const int par0 = (i0 + j) & 1;
  const bool xmA = i0 > 0, xpB = i0 + 2 < nx, ym = j > 0, yp = j < ny - 1;
  const float2 zero2 = make_float2(0.0f, 0.0f);
  // box origins: the iterate and b in floats (two per cell), the corrections
  // in packed entries rounded down to a multiple of 4
  const int ux = 4 * (bx * (TX - 2) - 1), uy = by * (TY - 2) - 1;
  const int pe = bx * (TX - 2) - 1, ex = pe & ~3, eo = pe - ex;
  const int bxo = 4 * bx * (TX - 2), byo = by * (TY - 2);

  const uint32_t base = (tma::smem_addr(ir_smem) + 127u) & ~127u;
  unsigned char* gbase = ir_smem + (base - tma::smem_addr(ir_smem));
  const uint32_t bar0 = base + kIrU * kIrUSlot + kIrB * kIrBSlot;
  auto ubar = [&](int q) { return bar0 + 8u * (uint32_t)(q % kIrU); };
  auto bbar = [&](int w) { return bar0 + 8u * (uint32_t)(kIrU + w % kIrB); };
  auto upar = [&](int q) { return (uint32_t)((q / kIrU) & 1); };
  auto bpar = [&](int w) { return (uint32_t)((w / kIrB) & 1); };
  // the consumers walk both rings in order: slot and phase parity of the
  // next sequence number, advanced without divisions
  struct Ring {
    int slot = 0;
    uint32_t par = 0;
    __device__ void next(int n) {
      if (++slot == n) {
        slot = 0;
        par ^= 1u;
      }
    }
  };

  // producer (thread 0): iterate/correction sequence q is plane z0 - 1 + q,
  // b sequence w is plane z0 + w
  auto issue_u = [&](int q) {
    const int z = z0 - 1 + q;
    const uint32_t b = ubar(q);
    if (z < 0 || z >= nz) {
      tma::bar_arrive(b);
      return;
    }
    tma::bar_arrive_tx(b, (uint32_t)kIrUSlot);  // the three boxes fill the slot exactly
    const uint32_t d = base + (uint32_t)((q % kIrU) * kIrUSlot);
    tma::load3(d, &maps.u, b, ux, uy, z);
    tma::load3(d + kIrUBytes, &maps.e0, b, ex, uy, z);
    tma::load3(d + kIrUBytes + kIrEBytes, &maps.e1, b, ex, uy, z);
  };
  auto issue_b = [&](int w) {
    const uint32_t b = bbar(w);
    tma::bar_arrive_tx(b, (uint32_t)kIrBBytes);
    tma::load3(base + (uint32_t)(kIrU * kIrUSlot + (w % kIrB) * kIrBSlot), &maps.b, b, bxo, byo,
               z0 + w);
  };
  // u + e of plane z0 - 1 + q for the thread's pair, from ring slot `slot`
  auto combine = [&](int q, int slot, Df2& v) {
    const int k = z0 - 1 + q;
    v = Df2{zero2, zero2};
    if (!(in && k >= 0 && k < nz)) return;
    const unsigned char* sl = gbase + slot * kIrUSlot;
    const float4 u4 = reinterpret_cast<const float4*>(sl)[ty * TX + tx];
    const float* e0 = reinterpret_cast<const float*>(sl + kIrUBytes) + ty * 36 + tx + eo;
    const float* e1 = reinterpret_cast<const float*>(sl + kIrUBytes + kIrEBytes) + ty * 36 + tx + eo;
    const bool ca = (par0 + k) & 1;
    const float2 re = make_float2(ca ? *e1 : *e0, ca ? *e0 : *e1);
    v = df_add2(Df2{make_float2(u4.x, u4.z), make_float2(u4.y, u4.w)}, re);
  };

  Df2 dxy;
  if (xmA && xpB && ym && yp) {
    dxy = Df2{make_float2(a.dint.x, a.dint.x), make_float2(a.dint.y, a.dint.y)};
  } else {
    const double dy = (ym ? 1.0 : 2.0 * a.op.rho[2]) + (yp ? 1.0 : 2.0 * a.op.rho[3]);
    const double dA = (xmA ? 1.0 : 2.0 * a.op.rho[0]) + 1.0 + dy + 2.0;
    const double dB = 1.0 + (xpB ? 1.0 : 2.0 * a.op.rho[1]) + dy + 2.0;
    const float2 sA = split_df(fma(dA, a.op.ih2, a.alpha));
    const float2 sB = split_df(fma(dB, a.op.ih2, a.alpha));
    dxy = Df2{make_float2(sA.x, sB.x), make_float2(sA.y, sB.y)};
  }

  int issued_u = min(kIrU, nq), issued_b = min(kIrB, n);
  if (tid == 0) {
    for (int i = 0; i < kIrU + kIrB; ++i) tma::bar_init(bar0 + 8u * i);
    tma::bar_init_fence();
    for (int q = 0; q < issued_u; ++q) issue_u(q);
    for (int w = 0; w < issued_b; ++w) issue_b(w);
  }
  __syncthreads();
  bool ok = tma::bar_wait(ubar(0), 0u) && tma::bar_wait(ubar(1), 0u) && tma::bar_wait(ubar(2), 0u);
  Df2 um, uc, up;
  combine(0, 0, um);
  combine(1, 1, uc);
  combine(2, 2, up);
  Ring ur, br;  // next iterate sequence to combine: 3 (slot 0, parity 1); next b: 0
  ur.par = 1u;
  float2 ss = zero2;
  if (!__syncthreads_or(!ok)) {
    if (tid == 0)
      for (; issued_u < min(nq, 6); ++issued_u) issue_u(issued_u);
    for (int i = 0; i < n; ++i) {
      const int k = z0 + i;
      ok = tma::bar_wait(bar0 + 8u * (uint32_t)(kIrU + br.slot), br.par) && ok;
      const unsigned char* bsl = gbase + kIrU * kIrUSlot + br.slot * kIrBSlot;
      br.next(kIrB);
      const int buf = i & 1;
      const float4 uc4 = make_float4(uc.hi.x, uc.lo.x, uc.hi.y, uc.lo.y);
      pl[buf][ty][tx] = uc4;
      const long long c = (long long)k * sz + off;
      if (own && a.udf_out) *reinterpret_cast<float4*>(a.udf_out + c) = uc4;
      if (__syncthreads_or(!ok)) {
        ok = false;
        break;
      }
      // every thread is past plane k - 1: its b slot and the slot of the
      // iterate it combined last are free
      if (tid == 0 && i >= 1) {
        if (issued_u < nq) issue_u(issued_u++);
        if (issued_b < n) issue_b(issued_b++);
      }
      const float pbh = __shfl_up_sync(FULL, uc.hi.y, 1), pbl = __shfl_up_sync(FULL, uc.lo.y, 1);
      const float nah = __shfl_down_sync(FULL, uc.hi.x, 1), nal = __shfl_down_sync(FULL, uc.lo.x, 1);
      if (own) {
        const Df2 L{make_float2(pbh, uc.hi.x), make_float2(pbl, uc.lo.x)};
        const Df2 R{make_float2(uc.hi.y, nah), make_float2(uc.lo.y, nal)};
        const float4 b4 = reinterpret_cast<const float4*>(bsl)[(ty - 1) * (TX - 2) + (tx - 1)];
        DfAcc2 acc{make_float2(b4.x, b4.z), make_float2(b4.y, b4.w)};
        const bool zm = k > 0, zp = k < nz - 1;
        Df2 dg = dxy;
        if (!zm) dg = df_add_df2(dg, a.dzm);
        if (!zp) dg = df_add_df2(dg, a.dzp);
        acc.add(Df2{make_float2(-dg.hi.x, -dg.hi.y), make_float2(-dg.lo.x, -dg.lo.y)}, uc);
        const float4 s4 = pl[buf][ty - 1][tx], n4 = pl[buf][ty + 1][tx];
        const Df2 w{make_float2(a.ih2d.x, a.ih2d.x), make_float2(a.ih2d.y, a.ih2d.y)};
        // the six neighbours summed first (none across A's -x or B's +x
        // domain face), then one product by 1/h^2
        DfSum2 nb{make_float2(xmA ? L.hi.x : 0.0f, L.hi.y),
                  make_float2(xmA ? L.lo.x : 0.0f, L.lo.y)};
        nb.add(Df2{make_float2(R.hi.x, xpB ? R.hi.y : 0.0f),
                   make_float2(R.lo.x, xpB ? R.lo.y : 0.0f)});
        if (ym) nb.add(Df2{make_float2(s4.x, s4.z), make_float2(s4.y, s4.w)});
        if (yp) nb.add(Df2{make_float2(n4.x, n4.z), make_float2(n4.y, n4.w)});
        if (zm) nb.add(um);
        if (zp) nb.add(up);
        acc.add(w, Df2{nb.s, nb.e});
        const float2 r = acc.value();
        if (a.r[0]) {
          const long long t = (long long)k * szW + eoff;
          const bool ca = (par0 + k) & 1;
          (ca ? a.r[1] : a.r[0])[t] = r.x;
          (ca ? a.r[0] : a.r[1])[t] = r.y;
        }
        ss = fma2(r, r, ss);
      }
      um = uc;
      uc = up;
      if (i + 1 < n) {
        ok = tma::bar_wait(bar0 + 8u * (uint32_t)ur.slot, ur.par) && ok;
        combine(i + 3, ur.slot, up);
        ur.next(kIrU);
      }
    }
  } else {
    ok = false;
  }
  if (!ok && tid == 0) {
    atomicExch(&g_ir_timeout, 1u);
    for (int q = max(0, issued_u - kIrU); q < issued_u; ++q) tma::bar_wait(ubar(q), upar(q));
    for (int w = max(0, issued_b - kIrB); w < issued_b; ++w) tma::bar_wait(bbar(w), bpar(w));
  }
  // CTA sums of r^2 (FP32 per thread, FP64 across the CTA)
  float s1 = ss.x + ss.y;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s1 += __shfl_xor_sync(FULL, s1, o);
  if (tx == 0) red[ty] = s1;
  __syncthreads();
  if (threadIdx.x < 32) {
    const long long cta = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    double v = threadIdx.x < NT / 32 ? (double)red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (threadIdx.x == 0) a.partial[cta] = v;
  }
}

// ---- the face-array refinement step with its planes staged by tensor copies --
//
// k_ir_df<Faces=1, HasE=1, U64=0, BIn=0> (the variable-coefficient refinement
// step after the first pass) with its inputs brought to shared memory by
// tiled tensor copies: per plane the CTA's 32 x 16 patch of the double-float
// iterate (box 68 x 16 floats from 2 i0 - 2, a 16-byte boundary; a thread
// indexes from the remainder) and of both colours' packed corrections (box
// 24 x 16 from the packed start rounded down to 4 entries) into a ring of
// three slots; b, the diagonal, the -x faces (one column more, for the +x
// face) and the -y faces (one row more) of the 30 x 14 own cells into a ring
// of three; the -z faces into a ring of four (plane k + 1 gives the +z face
// of plane k).  The march, the shared plane for the y-neighbours, the
// shuffles for the x-neighbours and the double-float arithmetic are k_ir_df's.
constexpr int kFsU = 3, kFsO = 3, kFsZ = 4;         // ring slots
constexpr int kFsUBytes = 16 * 68 * 4;              // 4352
constexpr int kFsEBytes = 16 * 24 * 4;              // 1536 per colour
constexpr int kFsUSlot = kFsUBytes + 2 * kFsEBytes;  // 7424 = 58 x 128
constexpr int kFsB = 14 * 60 * 4;                   // 3360: b, D, cz (60 floats x 14 rows)
constexpr int kFsBPad = 3456;                       // to 128
constexpr int kFsX = 14 * 64 * 4;                   // 3584: -x faces, 31 cells
constexpr int kFsY = 15 * 60 * 4;                   // 3600: -y faces, 15 rows
constexpr int kFsYPad = 3712;
constexpr int kFsOSlot = 2 * kFsBPad + kFsX + kFsYPad;  // b, D, cx, cy: 14208 = 111 x 128
constexpr int kFsSmem = 128 + kFsU * kFsUSlot + kFsO * kFsOSlot + kFsZ * kFsBPad +
                        8 * (kFsU + kFsO + kFsZ);

struct FsMaps {
  CUtensorMap u, e0, e1, b, d, cx, cy, cz;
};

__global__ void __launch_bounds__(NT, 2) k_ir_dff_tma(IrArgs a,
                                                      const __grid_constant__ FsMaps maps) {
  extern __shared__ unsigned char fs_smem[];
  __shared__ float2 pl[2][TY][TX];
  __shared__ float red[NT / 32];
  const unsigned FULL = 0xffffffffu;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int nx = a.op.b.nx, ny = a.op.b.ny, nz = a.op.b.nz;
  const int bx = blockIdx.x, by = blockIdx.y;
  const int i = bx * (TX - 2) - 1 + tx, j = by * (TY - 2) - 1 + ty;
  const int z0 = blockIdx.z * a.zchunk, z1 = min(nz, z0 + a.zchunk);
  const int n = z1 - z0, nq = n + 2, nv = min(z1 + 1, nz) - z0;
  const int W = a.W;
  const long long sz = (long long)nx * ny, szW = (long long)W * ny;
  const bool in = i >= 0 && i < nx && j >= 0 && j < ny;
  const bool own = in && tx >= 1 && tx <= TX - 2 && ty >= 1 && ty <= TY - 2;
  const int off = in ? j * nx + i : 0;
  const int eoff = in ? j * W + (i >> 1) : 0;
  const int par0 = (i + j) & 1;
  const bool xm = i > 0, xp = i < nx - 1, ym = j > 0, yp = j < ny - 1;
  // box origins: the iterate from 2 i0 - 2 floats rounded down to a multiple
  // of 4 (2 i0 = 60 bx - 2, so 60 bx - 4; a thread's pair sits at 2 tx + 2),
  // the corrections from the packed start rounded down to 4, the own cells'
  // arrays from cell 30 bx (60 bx floats) and row 14 by
  const int ux = 2 * bx * (TX - 2) - 4, uy = by * (TY - 2) - 1;
  const int ex = ((bx * (TX - 2) - 1) >> 1) & ~3;
  const int ecol = in ? (i >> 1) - ex : 0;
  const int ox = 2 * bx * (TX - 2), oy = by * (TY - 2);
  const float2 zero2 = make_float2(0.0f, 0.0f);

  const uint32_t base = (tma::smem_addr(fs_smem) + 127u) & ~127u;
  unsigned char* gbase = fs_smem + (base - tma::smem_addr(fs_smem));
  const uint32_t oS = base + kFsU * kFsUSlot, zS = oS + kFsO * kFsOSlot;
  const uint32_t bar0 = zS + kFsZ * kFsBPad;
  auto ubar = [&](int q) { return bar0 + 8u * (uint32_t)(q % kFsU); };
  auto obar = [&](int w) { return bar0 + 8u * (uint32_t)(kFsU + w % kFsO); };
  auto zbar = [&](int v) { return bar0 + 8u * (uint32_t)(kFsU + kFsO + v % kFsZ); };
  auto par3 = [](int q) { return (uint32_t)((q / 3) & 1); };
  auto par4 = [](int q) { return (uint32_t)((q / 4) & 1); };
  // producer (thread 0): iterate/correction sequence q is plane z0 - 1 + q;
  // own-cell sequence w and -z face sequence v are plane z0 + w (v)
  auto issue_u = [&](int q) {
    const int z = z0 - 1 + q;
    const uint32_t b = ubar(q);
    if (z < 0 || z >= nz) {
      tma::bar_arrive(b);
      return;
    }
    tma::bar_arrive_tx(b, (uint32_t)kFsUSlot);  // the three boxes fill the slot exactly
    const uint32_t d = base + (uint32_t)((q % kFsU) * kFsUSlot);
    tma::load3(d, &maps.u, b, ux, uy, z);
    tma::load3(d + kFsUBytes, &maps.e0, b, ex, uy, z);
    tma::load3(d + kFsUBytes + kFsEBytes, &maps.e1, b, ex, uy, z);
  };
  auto issue_o = [&](int w) {
    const uint32_t b = obar(w);
    tma::bar_arrive_tx(b, (uint32_t)(2 * kFsB + kFsX + kFsY));
    const uint32_t d = oS + (uint32_t)((w % kFsO) * kFsOSlot);
    tma::load3(d, &maps.b, b, ox, oy, z0 + w);
    tma::load3(d + kFsBPad, &maps.d, b, ox, oy, z0 + w);
    tma::load3(d + 2 * kFsBPad, &maps.cx, b, ox, oy, z0 + w);
    tma::load3(d + 2 * kFsBPad + kFsX, &maps.cy, b, ox, oy, z0 + w);
  };
  auto issue_z = [&](int v) {
    const uint32_t b = zbar(v);
    tma::bar_arrive_tx(b, (uint32_t)kFsB);
    tma::load3(zS + (uint32_t)((v % kFsZ) * kFsBPad), &maps.cz, b, ox, oy, z0 + v);
  };
  // u + e of plane z0 - 1 + q from ring slot `slot`
  auto combine = [&](int q, int slot, float2& v) {
    const int k = z0 - 1 + q;
    v = zero2;
    if (!(in && k >= 0 && k < nz)) return;
    const unsigned char* sl = gbase + slot * kFsUSlot;
    const float2 u2 = reinterpret_cast<const float2*>(sl)[ty * 34 + tx + 1];
    const float* e0 = reinterpret_cast<const float*>(sl + kFsUBytes) + ty * 24 + ecol;
    const float* e1 = reinterpret_cast<const float*>(sl + kFsUBytes + kFsEBytes) + ty * 24 + ecol;
    v = df_add(u2, ((par0 + k) & 1) ? *e1 : *e0);
  };

  int issued_u = min(kFsU, nq), issued_o = min(kFsO, n), issued_z = min(kFsZ, nv);
  if (tid == 0) {
    for (int q = 0; q < kFsU + kFsO + kFsZ; ++q) tma::bar_init(bar0 + 8u * q);
    tma::bar_init_fence();
    for (int q = 0; q < issued_u; ++q) issue_u(q);
    for (int w = 0; w < issued_o; ++w) issue_o(w);
    for (int v = 0; v < issued_z; ++v) issue_z(v);
  }
  __syncthreads();
  bool ok = tma::bar_wait(ubar(0), 0u) && tma::bar_wait(ubar(1), 0u) && tma::bar_wait(ubar(2), 0u);
  float2 um, uc, up;
  combine(0, 0, um);
  combine(1, 1, uc);
  combine(2, 2, up);
  float ss = 0.0f;
  if (!__syncthreads_or(!ok)) {
    if (tid == 0)
      for (; issued_u < min(nq, 6); ++issued_u) issue_u(issued_u);
    for (int it = 0; it < n; ++it) {
      const int k = z0 + it;
      ok = tma::bar_wait(obar(it), par3(it)) && ok;
      if (it == 0) ok = tma::bar_wait(zbar(0), 0u) && ok;
      if (k + 1 < nz) ok = tma::bar_wait(zbar(it + 1), par4(it + 1)) && ok;
      const int buf = it & 1;
      pl[buf][ty][tx] = uc;
      const long long c = (long long)k * sz + off;
      if (own && a.udf_out) a.udf_out[c] = uc;
      if (__syncthreads_or(!ok)) {
        ok = false;
        break;
      }
      // every thread is past plane k - 1: its slots are free
      if (tid == 0 && it >= 1) {
        if (issued_u < nq) issue_u(issued_u++);
        if (issued_o < n) issue_o(issued_o++);
        if (issued_z < nv) issue_z(issued_z++);
      }
      float2 ul, ur;
      ul.x = __shfl_up_sync(FULL, uc.x, 1);
      ul.y = __shfl_up_sync(FULL, uc.y, 1);
      ur.x = __shfl_down_sync(FULL, uc.x, 1);
      ur.y = __shfl_down_sync(FULL, uc.y, 1);
      if (own) {
        const float2* os = reinterpret_cast<const float2*>(gbase + kFsU * kFsUSlot +
                                                           (it % kFsO) * kFsOSlot);
        const int o30 = (ty - 1) * 30 + (tx - 1);
        const float2 bb = os[o30];
        const float2 dg = reinterpret_cast<const float2*>(
            reinterpret_cast<const unsigned char*>(os) + kFsBPad)[o30];
        const float2* cxs =
            reinterpret_cast<const float2*>(reinterpret_cast<const unsigned char*>(os) + 2 * kFsBPad);
        const float2* cys = reinterpret_cast<const float2*>(
            reinterpret_cast<const unsigned char*>(os) + 2 * kFsBPad + kFsX);
        const float2* czs = reinterpret_cast<const float2*>(gbase + kFsU * kFsUSlot +
                                                            kFsO * kFsOSlot);
        float r = 0.0f;
        if (!(dg.x < 0.0f)) {  // electrode cells (negative diagonal) keep r = 0
          const bool zm = k > 0, zp = k < nz - 1;
          DfAcc acc{bb.x, bb.y};
          if (a.has_alpha) acc.add(a.nalpha, uc);
          acc.add(make_float2(-dg.x, -dg.y), uc);
          const float2 us = pl[buf][ty - 1][tx], un = pl[buf][ty + 1][tx];
          const int o32 = (ty - 1) * 32 + (tx - 1);
          if (xm) acc.add(cxs[o32], ul);
          if (xp) acc.add(cxs[o32 + 1], ur);
          if (ym) acc.add(cys[o30], us);
          if (yp) acc.add(cys[o30 + 30], un);
          if (zm) acc.add(czs[(it % kFsZ) * (kFsBPad / 8) + o30], um);
          if (zp) acc.add(czs[((it + 1) % kFsZ) * (kFsBPad / 8) + o30], up);
          r = acc.value();
        }
        if (a.r[0]) (((par0 + k) & 1) ? a.r[1] : a.r[0])[(long long)k * szW + eoff] = r;
        ss = fmaf(r, r, ss);
      }
      um = uc;
      uc = up;
      if (it + 1 < n) {
        const int q = it + 3;
        ok = tma::bar_wait(ubar(q), par3(q)) && ok;
        combine(q, q % kFsU, up);
      }
    }
  } else {
    ok = false;
  }
  if (!ok && tid == 0) {
    atomicExch(&g_ir_timeout, 1u);
    for (int q = max(0, issued_u - kFsU); q < issued_u; ++q) tma::bar_wait(ubar(q), par3(q));
    for (int w = max(0, issued_o - kFsO); w < issued_o; ++w) tma::bar_wait(obar(w), par3(w));
    for (int v = max(0, issued_z - kFsZ); v < issued_z; ++v) tma::bar_wait(zbar(v), par4(v));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(FULL, ss, o);
  if (tx == 0) red[ty] = ss;
  __syncthreads();
  if (threadIdx.x < 32) {
    const long long cta = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    double v = threadIdx.x < NT / 32 ? (double)red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (threadIdx.x == 0) a.partial[cta] = v;
  }
}

// 1.0 into *flag (mapped host memory) if any of u[0..n) is neither +0 nor -0
// (a NaN counts as nonzero); at most one store per block.
// The test is on the bits (all but the sign zero), on the integer pipe, 16
// bytes per load where u is 16-byte aligned.
__global__ void k_nonzero(const double* __restrict__ u, long long n, double* flag) {
  const unsigned long long mag = 0x7fffffffffffffffull;
  unsigned long long any = 0;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long head = 0;
  if (((uintptr_t)u & 15u) == 0) {
    const ulonglong2* u2 = reinterpret_cast<const ulonglong2*>(u);
    const long long n2 = n / 2;
    for (long long c = t0; c < n2; c += 2 * stride) {
      const ulonglong2 a = u2[c];
      const ulonglong2 b = c + stride < n2 ? u2[c + stride] : make_ulonglong2(0, 0);
      any |= (a.x | a.y | b.x | b.y) & mag;
    }
    head = 2 * n2;
  }
  const unsigned long long* ub = reinterpret_cast<const unsigned long long*>(u);
  for (long long c = head + t0; c < n; c += stride) any |= ub[c] & mag;
  if (__syncthreads_or(any != 0) && threadIdx.x == 0) *flag = 1.0;
}

// First pass of a solve from a zero guess on a grid without electrode cells:
// the residual is b itself, so the pass is pointwise.  b (times in_scale) as
// double-floats into bdf_out, the zero iterate into udf_out, r = b rounded to
// FP32 (the value the stencil pass forms for this guess: hi + lo) into the
// split arrays r, and per-block sums of r^2 into partial and partial_z (the
// zero guess's residual is the same r).  Blocks take rows (j, k) in turn.
__global__ void __launch_bounds__(256) k_first_zero(IrArgs a) {
  __shared__ float red[8];
  const int nx = a.op.b.nx, ny = a.op.b.ny;
  const long long rows = (long long)ny * a.op.b.nz;
  float ss = 0.0f;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const int j = (int)(row % ny), k = (int)(row / ny);
    const long long base = row * nx, rbase = row * a.W;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const long long c = base + i;
      double bd = a.rhs[c];
      if (a.in_scale != 1.0) bd *= a.in_scale;
      const float2 bb = split_df(bd);
      a.bdf_out[c] = bb;
      a.udf_out[c] = make_float2(0.0f, 0.0f);
      const float r = __fadd_rn(bb.x, bb.y);
      (((i + j + k) & 1) ? a.r[1] : a.r[0])[rbase + (i >> 1)] = r;
      ss = fmaf(r, r, ss);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < 8 ? (double)red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) {
      a.partial[blockIdx.x] = v;
      a.partial_z[blockIdx.x] = v;
    }
  }
}

// FP64 result of a double-float iterate: exact widening of both parts on
// the integer pipe, one FP64 add, times the power-of-two scale that undoes a
// scaled solve (exact).  Electrode cells keep the caller's value.
__global__ void k_df_to_f64(const float2* __restrict__ in, const uint8_t* __restrict__ mask,
                            double* __restrict__ out, long long n, double scale) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n || (mask && mask[c])) return;
  const float2 v = in[c];
  const double u = widen(v.x) + widen(v.y);
  out[c] = scale != 1.0 ? u * scale : u;
}

// The same for two cells per thread (n even, arrays on 16-byte boundaries):
// one 16-byte load and one 16-byte store per pair, kX2 pairs per thread a
// grid stride apart (their loads issue back to back).  Scaled: the answer
// of a rescaled problem (times 1 / scale); Masked: electrode cells keep the
// caller's values.
constexpr int kX2 = 4;
template <bool Scaled, bool Masked>
__global__ void __launch_bounds__(256) k_df_to_f64x2(const float4* __restrict__ in,
                                                     const uchar2* __restrict__ mask,
                                                     double2* __restrict__ out, long long npair,
                                                     double scale) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long c0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float4 v[kX2];
#pragma unroll
  for (int q = 0; q < kX2; ++q) {
    const long long c = c0 + q * stride;
    v[q] = c < npair ? in[c] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
#pragma unroll
  for (int q = 0; q < kX2; ++q) {
    const long long c = c0 + q * stride;
    if (c >= npair) break;
    double2 u = make_double2(widen(v[q].x) + widen(v[q].y), widen(v[q].z) + widen(v[q].w));
    if (Scaled) u = make_double2(u.x * scale, u.y * scale);
    if (Masked) {
      const uchar2 m = mask[c];
      if (m.x || m.y) {
        double* o = reinterpret_cast<double*>(out + c);
        if (!m.x) o[0] = u.x;
        if (!m.y) o[1] = u.y;
        continue;
      }
    }
    out[c] = u;
  }
}

}  // namespace

// CTA columns of the refinement pass along x and y (30 x 14 own columns
// per CTA, 60 x 14 for the two-cell kernel), in 64-bit so that no grid size
// can wrap them.
static long long ir_gx(const Box& b, bool paired) {
  const long long own = paired ? 2 * (TX - 2) : TX - 2;
  return ((long long)b.nx + own - 1) / own;
}
static long long ir_gy(const Box& b) { return ((long long)b.ny + TY - 3) / (TY - 2); }

// Grid of the refinement pass for z planes per CTA column `hint` (0:
// automatic; halved for the two-cell kernel); *zchunk receives the planes
// used.  The automatic choice halves
// the z run while the grid has fewer than 8 * 152 * 3 CTAs (8 waves of three
// 512-thread CTAs on each of GB300's 152 SMs) and the run is longer than 16
// planes, so its CTA count is gx * gy when gx * gy >= 3648 and below
// 3 * 3648 otherwise: at most max(gx * gy, 10944).
static int ir_planes(int hint, bool paired) {
  // a two-cell CTA covers twice the columns of a one-cell CTA: half the
  // planes give it the same cells, so one tile setting suits both kernels
  return paired ? std::max(1, hint / 2) : hint;
}

static dim3 ir_grid(const Box& b, int hint, int* zchunk, bool paired) {
  const long long gx = ir_gx(b, paired), gy = ir_gy(b);
  int zc = b.nz;
  if (hint > 0) {
    zc = std::min(ir_planes(hint, paired), b.nz);
  } else {
    while (zc > 16 && gx * gy * (((long long)b.nz + zc - 1) / zc) < 8 * 152 * 3)
      zc = (zc + 1) / 2;
  }
  *zchunk = zc;
  return dim3((unsigned)gx, (unsigned)gy, (unsigned)((b.nz + zc - 1) / zc));
}

// CTAs of the refinement pass (64-bit, computed before any dim3 narrowing)
// for either kernel, whichever is larger.
static long long ir_ctas(const Box& b, int zchunk) {
  long long most = 0;
  for (int paired = 0; paired < 2; ++paired) {
    int zc = b.nz;
    if (zchunk > 0) zc = std::min(ir_planes(zchunk, paired != 0), b.nz);
    else ir_grid(b, 0, &zc, paired != 0);
    most = std::max(most, ir_gx(b, paired != 0) * ir_gy(b) * (((long long)b.nz + zc - 1) / zc));
  }
  return most;
}

int ir_partials(const Box& b, int zchunk) { return (int)ir_ctas(b, zchunk); }

bool ir_tma_ready() {
  static const bool ok =
      cudaFuncSetAttribute(k_ir_df2_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, kIrSmem) ==
          cudaSuccess &&
      cudaFuncSetAttribute(k_ir_dff_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, kFsSmem) ==
          cudaSuccess;
  return ok;
}

bool ir_timed_out() {
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, g_ir_timeout, sizeof(v)) != cudaSuccess) return false;
  if (v) {
    const unsigned zero = 0;
    cudaMemcpyToSymbol(g_ir_timeout, &zero, sizeof(zero));
  }
  return v != 0;
}

// The two-cell kernel runs the constant-coefficient operator (beta = 1)
// except the first pass of a solve (the norm of the zero guess as well); it
// needs an even nx (whole pairs) and arrays on 16-byte boundaries (one
// 16-byte load per pair; 2 bytes for the electrode flags).  With face arrays
// the pair's 28 coefficient values leave no room to fetch them a plane ahead
// in 64 registers, and the one-cell kernel, which does, is faster (280
// against 327 us per 256^3 step on GB300); the first pass spills in 64
// registers and is faster one cell per thread too (2.9 against 2.4 ms at
// 512^3).
static bool ir_pairable(const IrArgs& a) {
  auto al = [](const void* p, unsigned m) { return ((uintptr_t)p & (m - 1)) == 0; };
  return !a.op.cxd && !a.partial_z && a.op.b.nx % 2 == 0 && al(a.udf_in, 16) &&
         al(a.udf_out, 16) && al(a.bdf, 16) && al(a.bdf_out, 16) && al(a.u_in, 16) &&
         al(a.rhs, 16) && al(a.op.mask, 2);
}

// The staged two-cell step (k_ir_df2_tma) where it applies: a refinement
// step (double-float iterate plus correction, double-float b) on a grid
// without electrode cells, nx a multiple of 8 (the packed corrections' rows
// on 16-byte boundaries) and at least 128 x 16 cells per plane, 16-byte
// aligned arrays and encodable tensor maps.  False: nothing launched.
static bool ir_tma(const IrArgs& a, dim3 g, cudaStream_t s) {
  const Box& b = a.op.b;
  if (a.op.mask || b.nx % 8 != 0 || b.nx < 128 || b.ny < 16 || !a.udf_in || !a.bdf ||
      !a.e[0] || !a.e[1] || !ir_tma_ready())
    return false;
  IrMaps m;
  if (!tma_map_f32(&m.u, a.udf_in, 2LL * b.nx, b.ny, b.nz, 4 * TX, TY) ||
      !tma_map_f32(&m.e0, a.e[0], a.W, b.ny, b.nz, 36, TY) ||
      !tma_map_f32(&m.e1, a.e[1], a.W, b.ny, b.nz, 36, TY) ||
      !tma_map_f32(&m.b, a.bdf, 2LL * b.nx, b.ny, b.nz, 4 * (TX - 2), TY - 2))
    return false;
  k_ir_df2_tma<<<g, NT, kIrSmem, s>>>(a, m);
  return true;
}

// The staged face-array step (k_ir_dff_tma) where it applies: a
// variable-coefficient refinement step (double-float iterate plus correction,
// double-float b), nx a multiple of 8 and at least 64 x 16 cells per plane,
// 16-byte aligned arrays and encodable tensor maps.  False: nothing launched.
static bool ir_tma_faces(const IrArgs& a, dim3 g, cudaStream_t s) {
  const Box& b = a.op.b;
  if (b.nx % 8 != 0 || b.nx < 64 || b.ny < 16 || !a.udf_in || !a.bdf || !a.e[0] || !a.e[1] ||
      !a.op.cxd || !a.op.cyd || !a.op.czd || !a.op.Dd || !ir_tma_ready())
    return false;
  FsMaps m;
  const long long fx = 2LL * b.nx;
  if (!tma_map_f32(&m.u, a.udf_in, fx, b.ny, b.nz, 68, TY) ||
      !tma_map_f32(&m.e0, a.e[0], a.W, b.ny, b.nz, 24, TY) ||
      !tma_map_f32(&m.e1, a.e[1], a.W, b.ny, b.nz, 24, TY) ||
      !tma_map_f32(&m.b, a.bdf, fx, b.ny, b.nz, 2 * (TX - 2), TY - 2) ||
      !tma_map_f32(&m.d, a.op.Dd, fx, b.ny, b.nz, 2 * (TX - 2), TY - 2) ||
      !tma_map_f32(&m.cx, a.op.cxd, fx, b.ny, b.nz, 2 * TX, TY - 2) ||
      !tma_map_f32(&m.cy, a.op.cyd, fx, b.ny, b.nz, 2 * (TX - 2), TY - 1) ||
      !tma_map_f32(&m.cz, a.op.czd, fx, b.ny, b.nz, 2 * (TX - 2), TY - 2))
    return false;
  k_ir_dff_tma<<<g, NT, kFsSmem, s>>>(a, m);
  return true;
}

template <bool P, bool F, bool E, bool U, int B, bool Z>
static void go(const IrArgs& a, dim3 g, cudaStream_t s) {
  if (P && !Z) {
    if (E && !U && B == 0 && ir_tma(a, g, s)) return;
    k_ir_df2<E, U, B><<<g, NT, 0, s>>>(a);
  } else {
    if (F && E && !U && B == 0 && !Z && ir_tma_faces(a, g, s)) return;
    k_ir_df<F, E, U, B, Z><<<g, NT, 0, s>>>(a);
  }
}

template <bool P, bool F>
static void dispatch_f(const IrArgs& a, dim3 g, cudaStream_t s) {
  const int bin = a.bdf ? 0 : (a.lift || a.rhs_scale != 1.0 ? 2 : 1);
  if (a.udf_in) {  // double-float iterate (+ correction)
    if (a.e[0]) go<P, F, true, false, 0, false>(a, g, s);
    else go<P, F, false, false, 0, false>(a, g, s);
  } else if (a.partial_z) {  // FP64 guess, both norms
    if (bin == 0) go<P, F, false, true, 0, true>(a, g, s);
    else go<P, F, false, true, 1, true>(a, g, s);
  } else if (bin == 0) {
    go<P, F, false, true, 0, false>(a, g, s);
  } else if (bin == 1) {
    go<P, F, false, true, 1, false>(a, g, s);
  } else {
    go<P, F, false, true, 2, false>(a, g, s);
  }
}

static void dispatch(const IrArgs& a, dim3 g, bool paired, cudaStream_t s) {
  if (paired) {
    dispatch_f<true, false>(a, g, s);  // beta = 1 only (ir_pairable)
  } else {
    if (a.op.cxd) dispatch_f<false, true>(a, g, s);
    else dispatch_f<false, false>(a, g, s);
  }
}

// double-float of a host double
static float2 df_host(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

// Launch constants: 1/h^2, -alpha and the interior beta = 1 diagonal
// 6/h^2 + alpha as double-floats.
static void ir_constants(IrArgs& a) {
  a.ih2d = df_host(a.op.ih2);
  a.nalpha = df_host(-a.alpha);
  a.dint = df_host(6.0 * a.op.ih2 + a.alpha);
  a.has_alpha = a.alpha != 0.0;
  a.dzm = df_host((2.0 * a.op.rho[4] - 1.0) * a.op.ih2);
  a.dzp = df_host((2.0 * a.op.rho[5] - 1.0) * a.op.ih2);
}

int launch_ir_fused(const IrArgs& args, cudaStream_t s) {
  IrArgs a = args;
  if (a.in_scale == 0.0) a.in_scale = 1.0;  // zero-initialised arguments: no scaling
  const bool paired = ir_pairable(a);
  dim3 g = ir_grid(a.op.b, args.zchunk, &a.zchunk, paired);
  ir_constants(a);
  dispatch(a, g, paired, s);
  add_launches(1);
  return (int)(g.x * g.y * g.z);
}

void launch_nonzero(const double* u, long long n, double* flag, cudaStream_t s) {
  k_nonzero<<<152 * 8, 256, 0, s>>>(u, n, flag);
  add_launches(1);
}

int launch_first_zero(const IrArgs& args, int max_blocks, cudaStream_t s) {
  IrArgs a = args;
  if (a.in_scale == 0.0) a.in_scale = 1.0;
  const long long rows = (long long)a.op.b.ny * a.op.b.nz;
  const int g = (int)std::max(1LL, std::min<long long>(rows, max_blocks));
  k_first_zero<<<g, 256, 0, s>>>(a);
  add_launches(1);
  return g;
}

void launch_df_to_f64(const float2* in, const uint8_t* mask, double* out, long long n,
                      double scale, cudaStream_t s) {
  auto al = [](const void* p, unsigned m) { return ((uintptr_t)p & (m - 1)) == 0; };
  if (n % 2 == 0 && al(in, 16) && al(out, 16) && al(mask, 2)) {
    const long long np = n / 2;
    const unsigned g = (unsigned)((np + 256LL * kX2 - 1) / (256LL * kX2));
    const auto* i4 = reinterpret_cast<const float4*>(in);
    const auto* m2 = reinterpret_cast<const uchar2*>(mask);
    auto* o2 = reinterpret_cast<double2*>(out);
    if (scale != 1.0) {
      if (mask) k_df_to_f64x2<true, true><<<g, 256, 0, s>>>(i4, m2, o2, np, scale);
      else k_df_to_f64x2<true, false><<<g, 256, 0, s>>>(i4, m2, o2, np, scale);
    } else {
      if (mask) k_df_to_f64x2<false, true><<<g, 256, 0, s>>>(i4, m2, o2, np, scale);
      else k_df_to_f64x2<false, false><<<g, 256, 0, s>>>(i4, m2, o2, np, scale);
    }
  } else {
    k_df_to_f64<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, mask, out, n, scale);
  }
  add_launches(1);
}

}  // namespace mg

// ---- allocation-free residual norm ------------------------------------------
//
// mg_residual_norm_noalloc (include/mg.h) runs the refinement-residual kernel
// above for a constant-coefficient operator described entirely by the
// caller's arguments, and keeps its per-CTA partial sums in the file-scope
// device array g_noalloc_scratch (top of this file) instead of in memory
// obtained from cudaMalloc.  It is for callers that must not allocate device
// memory during the call: codes whose device memory is already owned by their
// own pool allocator, and time-stepping loops that cannot afford the implicit
// device-wide synchronisation that cudaMalloc and cudaFree may perform.  Every
// call overwrites the partial sums it later reads, so nothing needs clearing;
// calls that overlap on the GPU (two streams, or two host threads) share the
// array and race.

namespace mg {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {};  // device address of the array, per device

// Sum of the partials (same order as the solver's reduction), then sqrt.
__global__ void k_noalloc_finish(const double* __restrict__ partial, int n, double* out) {
  __shared__ double ws[NT / 32];
  double s = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) s += partial[t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) ws[w] = s;
  __syncthreads();
  if (w == 0) {
    double v = lane < NT / 32 ? ws[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) *out = sqrt(v);
  }
}

// Device address of g_noalloc_scratch on the current device.  The first call
// on a device resolves it with cudaGetSymbolAddress (host code only holds a
// stand-in for the symbol, never its device address).
mg_status noalloc_scratch(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    mg::set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return MG_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    mg::set_last_error("device ordinal out of range for the allocation-free scratch");
    return MG_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      mg::set_last_error(std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") +
                         cudaGetErrorString(e));
      return MG_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return MG_OK;
}

}  // namespace

// The refinement-residual kernel (no correction, not the norm of b) with its
// partial sums in the static scratch, then the final sum and square root.
void launch_noalloc(IrArgs a, double* scratch, double* norm_out, cudaStream_t s) {
  a.partial = scratch;
  const bool paired = ir_pairable(a);
  dim3 g = ir_grid(a.op.b, 0, &a.zchunk, paired);
  ir_constants(a);
  dispatch(a, g, paired, s);
  k_noalloc_finish<<<1, NT, 0, s>>>(scratch, (int)(g.x * g.y * g.z), norm_out);
  add_launches(2);
}

}  // namespace mg

extern "C" mg_status mg_residual_norm_noalloc(const mg_grid* grid, const mg_bc* bc, double alpha,
                                              const double* rhs, double rhs_scale,
                                              const uint8_t* mask, const double* u,
                                              double* norm_out, void* cuda_stream) {
  mg::set_last_error("");
  if (!grid || !bc || !rhs || !u || !norm_out) {
    mg::set_last_error("NULL argument");
    return MG_ERR_INVALID_ARG;
  }
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->h > 0.0) ||
      !(alpha >= 0.0) || !std::isfinite(rhs_scale)) {
    mg::set_last_error("grid sizes must be >= 1, h > 0, alpha >= 0, rhs_scale finite");
    return MG_ERR_INVALID_ARG;
  }
  for (int f = 0; f < 6; ++f)
    if ((bc->kind[f] != MG_BC_DIRICHLET && bc->kind[f] != MG_BC_NEUMANN) ||
        !std::isfinite(bc->value[f])) {
      mg::set_last_error("bad boundary condition");
      return MG_ERR_INVALID_ARG;
    }
  mg::Box box{grid->nx, grid->ny, grid->nz};
  // launch limits of the kernel's grid: y and z extents below 65536
  if (mg::ir_gy(box) > 65535 || box.nz > 65535) {  // (same for either kernel)
    mg::set_last_error("grid too large for the refinement kernel's launch: ceil(ny/14) and nz "
                       "must not exceed 65535");
    return MG_ERR_UNSUPPORTED;
  }
  const long long nparts = mg::ir_ctas(box, 0);
  if (nparts > MG_NOALLOC_MAX_PARTIALS) {
    char msg[256];
    std::snprintf(msg, sizeof msg,
                  "grid too large for the allocation-free scratch: the residual kernel needs "
                  "up to %lld partial sums (ceil(nx/30) * ceil(ny/14) * z-chunks), more than "
                  "the "
                  "16384 of the static array",
                  nparts);
    mg::set_last_error(msg);
    return MG_ERR_UNSUPPORTED;
  }
  double* scratch = nullptr;
  mg_status st = mg::noalloc_scratch(&scratch);
  if (st != MG_OK) return st;

  mg::IrArgs a{};
  a.op.b = box;
  a.op.ih2 = 1.0 / (grid->h * grid->h);
  a.op.mask = mask;
  for (int f = 0; f < 6; ++f) {
    a.op.rho[f] = bc->kind[f] == MG_BC_DIRICHLET ? 1.0 : 0.0;
    a.bval.v[f] = bc->value[f];
  }
  a.alpha = alpha;
  a.rhs = rhs;
  a.rhs_scale = rhs_scale;
  a.lift = 1;
  a.u_in = u;
  a.in_scale = 1.0;
  mg::launch_noalloc(a, scratch, norm_out, (cudaStream_t)cuda_stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    mg::set_last_error(std::string("kernel launch: ") + cudaGetErrorString(e));
    return MG_ERR_CUDA;
  }
  return MG_OK;
}
