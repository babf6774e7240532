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
    else C.bd = a.rhs[c];
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

// FP64 result of a double-float iterate: exact widening of both parts on
// the integer pipe, one FP64 add.  Electrode cells keep the caller's value.
__global__ void k_df_to_f64(const float2* __restrict__ in, const uint8_t* __restrict__ mask,
                            double* __restrict__ out, long long n) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n || (mask && mask[c])) return;
  const float2 v = in[c];
  out[c] = widen(v.x) + widen(v.y);
}

}  // namespace

// CTA columns of the refinement pass along x and y (30 x 14 own columns
// per CTA), in 64-bit so that no grid size can wrap them.
static long long ir_gx(const Box& b) { return ((long long)b.nx + TX - 3) / (TX - 2); }
static long long ir_gy(const Box& b) { return ((long long)b.ny + TY - 3) / (TY - 2); }

// Grid of the refinement pass for z planes per CTA column `hint` (0:
// automatic); *zchunk receives the planes used.  The automatic choice halves
// the z run while the grid has fewer than 8 * 152 * 3 CTAs (8 waves of three
// 512-thread CTAs on each of GB300's 152 SMs) and the run is longer than 16
// planes, so its CTA count is gx * gy when gx * gy >= 3648 and below
// 3 * 3648 otherwise: at most max(gx * gy, 10944).
static dim3 ir_grid(const Box& b, int hint, int* zchunk) {
  const long long gx = ir_gx(b), gy = ir_gy(b);
  int zc = b.nz;
  if (hint > 0) {
    zc = std::min(hint, b.nz);
  } else {
    while (zc > 16 && gx * gy * (((long long)b.nz + zc - 1) / zc) < 8 * 152 * 3)
      zc = (zc + 1) / 2;
  }
  *zchunk = zc;
  return dim3((unsigned)gx, (unsigned)gy, (unsigned)((b.nz + zc - 1) / zc));
}

// CTAs of the refinement pass (64-bit, computed before any dim3 narrowing).
static long long ir_ctas(const Box& b, int zchunk) {
  int zc = b.nz;
  if (zchunk > 0) {
    zc = std::min(zchunk, b.nz);
  } else {
    ir_grid(b, 0, &zc);
  }
  return ir_gx(b) * ir_gy(b) * (((long long)b.nz + zc - 1) / zc);
}

int ir_partials(const Box& b, int zchunk) { return (int)ir_ctas(b, zchunk); }

template <bool F, bool E, bool U, int B, bool Z>
static void go(const IrArgs& a, dim3 g, cudaStream_t s) {
  k_ir_df<F, E, U, B, Z><<<g, NT, 0, s>>>(a);
}

template <bool F>
static void dispatch_f(const IrArgs& a, dim3 g, cudaStream_t s) {
  const int bin = a.bdf ? 0 : (a.lift || a.rhs_scale != 1.0 ? 2 : 1);
  if (a.udf_in) {  // double-float iterate (+ correction)
    if (a.e[0]) go<F, true, false, 0, false>(a, g, s);
    else go<F, false, false, 0, false>(a, g, s);
  } else if (a.partial_z) {  // FP64 guess, both norms
    if (bin == 0) go<F, false, true, 0, true>(a, g, s);
    else go<F, false, true, 1, true>(a, g, s);
  } else if (bin == 0) {
    go<F, false, true, 0, false>(a, g, s);
  } else if (bin == 1) {
    go<F, false, true, 1, false>(a, g, s);
  } else {
    go<F, false, true, 2, false>(a, g, s);
  }
}

static void dispatch(const IrArgs& a, dim3 g, cudaStream_t s) {
  if (a.op.cxd) dispatch_f<true>(a, g, s);
  else dispatch_f<false>(a, g, s);
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
}

void launch_ir_fused(const IrArgs& args, cudaStream_t s) {
  IrArgs a = args;
  dim3 g = ir_grid(a.op.b, args.zchunk, &a.zchunk);
  ir_constants(a);
  dispatch(a, g, s);
  add_launches(1);
}

void launch_df_to_f64(const float2* in, const uint8_t* mask, double* out, long long n,
                      cudaStream_t s) {
  k_df_to_f64<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, mask, out, n);
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
void launch_noalloc(IrArgs a, double* scratch, int nparts, double* norm_out, cudaStream_t s) {
  a.partial = scratch;
  dim3 g = ir_grid(a.op.b, 0, &a.zchunk);
  ir_constants(a);
  dispatch(a, g, s);
  k_noalloc_finish<<<1, NT, 0, s>>>(scratch, nparts, norm_out);
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
  if (mg::ir_gy(box) > 65535 || box.nz > 65535) {
    mg::set_last_error("grid too large for the refinement kernel's launch: ceil(ny/14) and nz "
                       "must not exceed 65535");
    return MG_ERR_UNSUPPORTED;
  }
  const long long nparts = mg::ir_ctas(box, 0);
  if (nparts > MG_NOALLOC_MAX_PARTIALS) {
    char msg[256];
    std::snprintf(msg, sizeof msg,
                  "grid too large for the allocation-free scratch: the residual kernel needs "
                  "%lld partial sums (ceil(nx/30) * ceil(ny/14) * z-chunks), more than the "
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
  mg::launch_noalloc(a, scratch, (int)nparts, norm_out, (cudaStream_t)cuda_stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    mg::set_last_error(std::string("kernel launch: ") + cudaGetErrorString(e));
    return MG_ERR_CUDA;
  }
  return MG_OK;
}
