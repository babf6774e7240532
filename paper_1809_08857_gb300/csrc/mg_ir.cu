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
// instruction is left per cell.  Each CTA marches along z through a 32 x 16
// (x, y) tile, keeping three planes of u + e (with a one-cell halo) in
// shared memory as double-floats.
#include <cmath>
#include <mutex>
#include <string>

#include "../../include/mg.h"
#include "df.cuh"
#include "mg_internal.h"

// Largest number of CTAs (partial sums) one call may use: 16384 doubles,
// 128 KiB.  Every GPU that loads libmg holds this array until process exit.
#define MG_NOALLOC_MAX_PARTIALS 16384

static __device__ __align__(256) double g_noalloc_scratch[MG_NOALLOC_MAX_PARTIALS];

namespace mg {

namespace {

using namespace df;

constexpr int TX = 32, TY = 16, NT = TX * TY;
constexpr int PX = TX + 2, PY = TY + 2, PN = PX * PY;

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
// Software pipeline along z with four plane buffers: while plane k is
// computed, plane k+2 is stored to shared memory from registers and the
// loads of plane k+3 and of the own cells' b and coefficients of plane k+1
// are in flight; one barrier per plane.
template <bool Faces, bool HasE, bool U64, int BIn, bool ZNorm>
__global__ void __launch_bounds__(NT, 2) k_ir_df(IrArgs a) {
  __shared__ float2 pl[4][PN];
  __shared__ unsigned char mk[ZNorm ? 4 : 1][ZNorm ? PN : 1];  // electrode flags
  __shared__ float red[2][NT / 32];
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * a.zchunk;
  const int nx = a.op.b.nx, ny = a.op.b.ny, nz = a.op.b.nz;
  const int z1 = min(nz, z0 + a.zchunk);
  const int W = a.W;
  const int sy = nx;
  const long long sz = (long long)nx * ny, szW = (long long)W * ny;
  const int i = x0 + tx, j = y0 + ty;
  const bool own = i < nx && j < ny;
  const int ooff = j * nx + i;        // in-plane offset of the own cell
  const int oeoff = j * W + (i >> 1);  // and of its packed (split) position
  const bool zmask = ZNorm && a.op.mask != nullptr;
  // beta = 1: diagonal (in-box faces + 2 rho per domain face) / h^2 +
  // alpha; interior cells use the launcher's double-float 6/h^2 + alpha,
  // boundary cells form theirs in FP64 (a few cells per plane)
  double dxy = 0.0;
  bool xy_in = true;
  if (!Faces) {
    dxy += i > 0 ? 1.0 : 2.0 * a.op.rho[0];
    dxy += i < nx - 1 ? 1.0 : 2.0 * a.op.rho[1];
    dxy += j > 0 ? 1.0 : 2.0 * a.op.rho[2];
    dxy += j < ny - 1 ? 1.0 : 2.0 * a.op.rho[3];
    xy_in = i > 0 && i < nx - 1 && j > 0 && j < ny - 1;
  }
  // the (at most two) tile cells this thread loads per plane
  constexpr int NS = (PN + NT - 1) / NT;
  int qoff[NS], qeoff[NS], qpar[NS];
  bool qin[NS], qown[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const int q = threadIdx.x + s * NT;
    const int lx = q % PX, ly = q / PX;
    const int gi = x0 + lx - 1, gj = y0 + ly - 1;
    qin[s] = q < PN && gi >= 0 && gi < nx && gj >= 0 && gj < ny;
    qown[s] = qin[s] && lx >= 1 && lx <= TX && ly >= 1 && ly <= TY;
    qoff[s] = gj * nx + gi;
    qeoff[s] = gj * W + (gi >> 1);
    qpar[s] = (gi + gj) & 1;
  }

  // ---- tile planes: raw loads (fetch) and their use one iteration later (commit)
  double rd[NS];         // FP64 iterate
  float2 ru[NS];         // double-float iterate
  float re[NS];          // correction
  unsigned char rm[NS];  // electrode flag
  auto fetch = [&](int k) {
    const bool kin = k >= 0 && k < nz;
    const long long pb = (long long)k * sz, pe = (long long)k * szW;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      if (!(kin && qin[s])) continue;
      const long long c = pb + qoff[s];
      if (zmask) rm[s] = a.op.mask[c];
      if (U64) {
        rd[s] = a.u_in[c];
      } else {
        ru[s] = a.udf_in[c];
        if (HasE) {
          const long long t = pe + qeoff[s];
          re[s] = ((qpar[s] + k) & 1) ? a.e[1][t] : a.e[0][t];
        }
      }
    }
  };
  auto commit = [&](int buf, int k) {
    const bool kin = k >= 0 && k < nz, kown = k >= z0 && k < z1;
    const long long pb = (long long)k * sz;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const int q = threadIdx.x + s * NT;
      if (NS * NT > PN && q >= PN) break;
      float2 v = make_float2(0.0f, 0.0f);
      unsigned char m = 0;
      if (kin && qin[s]) {
        if (U64) v = split_df(rd[s]);
        else v = HasE ? df_add(ru[s], re[s]) : ru[s];
        if (kown && qown[s] && a.udf_out) a.udf_out[pb + qoff[s]] = v;
        if (zmask) m = rm[s];
      }
      pl[buf][q] = v;
      if (ZNorm) mk[buf][q] = m;
    }
  };

  // ---- own cell of a plane: b, electrode flag, coefficients
  struct Cell {
    double bd;
    float2 bb, dg, cxm, cxp, cym, cyp, czm, czp;
    bool m;
  };
  auto cell_fetch = [&](int k, Cell& C) {
    if (!own || k >= z1) return;
    const long long c = (long long)k * sz + ooff;
    if (Faces) {
      C.dg = a.op.Dd[c];
      const float2* cx = a.op.cxd + c;
      const float2* cy = a.op.cyd + c;
      const float2* cz = a.op.czd + c;
      C.cxm = cx[0];
      if (i < nx - 1) C.cxp = cx[1];
      C.cym = cy[0];
      if (j < ny - 1) C.cyp = cy[sy];
      C.czm = cz[0];
      if (k < nz - 1) C.czp = cz[sz];
    } else {
      C.m = a.op.mask && a.op.mask[c];
    }
    if (BIn == 0) C.bb = a.bdf[c];
    else C.bd = a.rhs[c];
  };

  fetch(z0 - 1);
  commit(0, z0 - 1);
  fetch(z0);
  commit(1, z0);
  fetch(z0 + 1);
  commit(2, z0 + 1);
  if (z0 + 2 <= z1) fetch(z0 + 2);
  Cell C{}, Cn{};
  cell_fetch(z0, C);
  __syncthreads();
  float ss = 0.0f, sz2 = 0.0f;
  for (int k = z0; k < z1; ++k) {
    // plane p sits in buffer (p - z0 + 1) & 3
    const int b0 = (k - z0) & 3, bm = (k - z0 + 1) & 3, bp = (k - z0 + 2) & 3;
    if (k + 2 <= z1) commit((k - z0 + 3) & 3, k + 2);
    if (k + 3 <= z1) fetch(k + 3);
    cell_fetch(k + 1, Cn);
    if (own) {
      const long long c = (long long)k * sz + ooff;
      const int q = (ty + 1) * PX + (tx + 1);
      float r = 0.0f, rz = 0.0f;
      const bool m = Faces ? C.dg.x < 0.0f : C.m;
      float2 bb;
      if (BIn == 0) {
        bb = C.bb;
      } else {
        double bd = C.bd;
        if (BIn == 2) {
          bd *= a.rhs_scale;
          const bool edge = i == 0 || i == nx - 1 || j == 0 || j == ny - 1 || k == 0 || k == nz - 1;
          if (a.lift && edge && !m) {
            const double l = 2.0 * (a.beta0 ? a.beta0[c] : 1.0) * a.op.ih2;
            if (i == 0 && a.op.rho[0] == 1.0) bd += l * a.bval.v[0];
            if (i == nx - 1 && a.op.rho[1] == 1.0) bd += l * a.bval.v[1];
            if (j == 0 && a.op.rho[2] == 1.0) bd += l * a.bval.v[2];
            if (j == ny - 1 && a.op.rho[3] == 1.0) bd += l * a.bval.v[3];
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
        // r = b - diag u_c + sum_f w_f u_nb
        const float2 uc = pl[bm][q];
        float2 dg;
        if (Faces) {
          dg = C.dg;
          if (a.has_alpha) acc.add(a.nalpha, uc);
        } else {
          if (xy_in && k > 0 && k < nz - 1) {
            dg = a.dint;
          } else {
            const double d = dxy + (k > 0 ? 1.0 : 2.0 * a.op.rho[4]) +
                             (k < nz - 1 ? 1.0 : 2.0 * a.op.rho[5]);
            dg = split_df(fma(d, a.op.ih2, a.alpha));
          }
        }
        acc.add(make_float2(-dg.x, -dg.y), uc);
        auto nb = [&](bool in, float2 w, int buf, int qq) {
          if (!in) return;
          const float2 un = pl[buf][qq];
          acc.add(w, un);
          if (zmask && mk[buf][qq]) az.add(w, un);
        };
        if (Faces) {
          nb(i > 0, C.cxm, bm, q - 1);
          nb(i < nx - 1, C.cxp, bm, q + 1);
          nb(j > 0, C.cym, bm, q - PX);
          nb(j < ny - 1, C.cyp, bm, q + PX);
          nb(k > 0, C.czm, b0, q);
          nb(k < nz - 1, C.czp, bp, q);
        } else {
          const float2 w = a.ih2d;
          nb(i > 0, w, bm, q - 1);
          nb(i < nx - 1, w, bm, q + 1);
          nb(j > 0, w, bm, q - PX);
          nb(j < ny - 1, w, bm, q + PX);
          nb(k > 0, w, b0, q);
          nb(k < nz - 1, w, bp, q);
        }
        r = acc.value();
        rz = az.value();
      }
      if (a.r[0]) (((i + j + k) & 1) ? a.r[1] : a.r[0])[(long long)k * szW + oeoff] = r;
      ss = fmaf(r, r, ss);
      if (ZNorm) sz2 = fmaf(rz, rz, sz2);
    }
    C = Cn;
    __syncthreads();
  }
  // CTA sums of r^2 (FP32 is ample for a stopping test; the partials and the
  // final sum are accumulated in FP64)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (ZNorm) sz2 += __shfl_xor_sync(0xffffffffu, sz2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = ss;
    if (ZNorm) red[1][threadIdx.x >> 5] = sz2;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const long long cta = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
#pragma unroll
    for (int h = 0; h < (ZNorm ? 2 : 1); ++h) {
      double v = threadIdx.x < NT / 32 ? (double)red[h][threadIdx.x] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
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

static dim3 ir_grid(const Box& b, int* zchunk) {
  const int gx = (b.nx + TX - 1) / TX, gy = (b.ny + TY - 1) / TY;
  // enough CTAs to fill every SM (152 on GB300) a few times, long z runs
  int zc = b.nz;
  while (zc > 16 && (long long)gx * gy * ((b.nz + zc - 1) / zc) < 4 * 152 * 2) zc = (zc + 1) / 2;
  *zchunk = zc;
  return dim3(gx, gy, (b.nz + zc - 1) / zc);
}

int ir_partials(const Box& b) {
  int zc;
  dim3 g = ir_grid(b, &zc);
  return (int)(g.x * g.y * g.z);
}

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
  dim3 g = ir_grid(a.op.b, &a.zchunk);
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
  dim3 g = ir_grid(a.op.b, &a.zchunk);
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
  const int nparts = mg::ir_partials(box);
  if (nparts > MG_NOALLOC_MAX_PARTIALS) {
    mg::set_last_error("grid too large for the allocation-free scratch: ceil(nx/32)*ceil(ny/8) "
                       "must not exceed 16384");
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
  mg::launch_noalloc(a, scratch, nparts, norm_out, (cudaStream_t)cuda_stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    mg::set_last_error(std::string("kernel launch: ") + cudaGetErrorString(e));
    return MG_ERR_CUDA;
  }
  return MG_OK;
}
