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
// only FP64 instruction left per cell is u + e.  Each CTA marches along z
// through a 32 x 16 (x, y) tile, keeping three planes of u + e (with a
// one-cell halo) in shared memory as double-floats.
#include <cmath>
#include <mutex>
#include <string>

#include "../../include/mg.h"
#include "mg_internal.h"

// Largest number of CTAs (partial sums) one call may use: 16384 doubles,
// 128 KiB.  Every GPU that loads libmg holds this array until process exit.
#define MG_NOALLOC_MAX_PARTIALS 16384

static __device__ __align__(256) double g_noalloc_scratch[MG_NOALLOC_MAX_PARTIALS];

namespace mg {

namespace {

constexpr int TX = 32, TY = 16, NT = TX * TY;
constexpr int PX = TX + 2, PY = TY + 2, PN = PX * PY;

// IEEE-754 binary32 -> binary64 by re-biasing the exponent (1023 - 127 = 896)
// and widening the fraction, on the integer pipe (the FP64 pipe is the
// bottleneck of this kernel).  Zeros and binary32 subnormals (< 1.2e-38,
// never reached by a correction of a physical field) map to a signed zero;
// infinities and NaNs keep their class.
__device__ __forceinline__ double widen(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned long long sgn = (unsigned long long)(b >> 31) << 63;
  const unsigned ex = (b >> 23) & 0xffu;
  const unsigned long long man = (unsigned long long)(b & 0x7fffffu) << 29;
  const unsigned long long e64 = ex == 0xffu ? 0x7ffull : (unsigned long long)ex + 896ull;
  const unsigned long long bits = ex == 0u ? sgn : (sgn | (e64 << 52) | man);
  return __longlong_as_double((long long)bits);
}

// binary64 -> binary32 by truncation (round toward zero: at most one FP32
// ulp, harmless for the right-hand side of the FP32 inner cycle), integer
// pipe.  Values below the binary32 normal range flush to zero, values above
// it become infinity, NaN stays NaN.
__device__ __forceinline__ float narrow(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sgn = (unsigned)(b >> 63) << 31;
  const int ex = (int)((b >> 52) & 0x7ffull);
  const unsigned man = (unsigned)((b >> 29) & 0x7fffffull);
  const int e32 = ex - 896;
  unsigned bits;
  if (ex == 0x7ff) bits = sgn | 0x7f800000u | (man ? 0x400000u : 0u);
  else if (e32 >= 255) bits = sgn | 0x7f800000u;
  else if (e32 <= 0) bits = sgn;
  else bits = sgn | ((unsigned)e32 << 23) | man;
  return __uint_as_float(bits);
}

// electrode test on the integer pipe: D < 0 marks an electrode cell
__device__ __forceinline__ bool masked64(const Op64& op, long long c) {
  if (op.Dd) return op.Dd[c].x < 0.0f;
  return op.mask != nullptr && op.mask[c] != 0;
}

// ---- double-float arithmetic ------------------------------------------------
//
// A double-float is an unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi): 48 significant bits, enough for a residual whose stopping
// test sits at 1e-10 of ||b||.  Products and sums are made exact with the
// classical error-free transformations (Dekker's product via FMA, Knuth's
// two-sum); the _rn intrinsics keep the compiler from contracting or
// reassociating them.

// binary64 -> double-float without an FP64 instruction: hi = x truncated to
// 24 significant bits (integer pipe), lo = the remaining 29 bits rounded to
// FP32 (one integer -> float conversion and a power-of-two scale).  For
// |x| < 2^-74 lo is dropped; below the FP32 normal range x flushes to 0.
__device__ __forceinline__ float2 split_df(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const float hi = narrow(x);
  const int se = (int)((b >> 52) & 0x7ffull) - 948;  // FP32 exponent field of 2^(ex - 1075)
  const float scale = (se >= 1 && se <= 254) ? __uint_as_float((unsigned)se << 23) : 0.0f;
  const float lo = __fmul_rn(__uint2float_rn((unsigned)(b & 0x1fffffffull)), scale);
  return make_float2(hi, (b >> 63) ? -lo : lo);
}

// Running sum s + e of double-float products.  add(c, u): s + e += c * u.
// The product's rounding error (FMA) and its cross terms, and the two-sum
// error of s, go into e; e itself is a plain FP32 sum of terms 2^-24 below
// the leading ones, so the total error stays near 2^-48 of the largest term.
struct DfAcc {
  float s, e;
  __device__ __forceinline__ void add(float2 c, float2 u) {
    const float p = __fmul_rn(c.x, u.x);
    float q = fmaf(c.x, u.x, -p);
    q = fmaf(c.x, u.y, q);
    q = fmaf(c.y, u.x, q);
    const float t = __fadd_rn(s, p);
    const float v = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, v)), __fsub_rn(p, v));
    s = t;
    e = __fadd_rn(e, __fadd_rn(err, q));
  }
  __device__ __forceinline__ float value() const { return __fadd_rn(s, e); }
};

// u + e at cell (i, j, k) as a double-float (0 outside the box).  The one FP64
// instruction per cell is the add of the FP32 correction; own cells (not
// the halo of the tile) also store it to u_out.
template <bool HasE, bool ZeroFree>
__device__ __forceinline__ float2 load_cell(const IrArgs& a, int i, int j, int k, bool own) {
  if (i < 0 || j < 0 || k < 0 || i >= a.op.b.nx || j >= a.op.b.ny || k >= a.op.b.nz)
    return make_float2(0.0f, 0.0f);
  const long long c = ((long long)k * a.op.b.ny + j) * a.op.b.nx + i;
  if (ZeroFree) return masked64(a.op, c) ? split_df(a.u_in[c]) : make_float2(0.0f, 0.0f);
  double v = a.u_in[c];
  if (HasE) {
    const long long t = ((long long)k * a.op.b.ny + j) * a.W + (i >> 1);
    v += widen(((i + j + k) & 1) ? a.e[1][t] : a.e[0][t]);
  }
  if (own && a.u_out) a.u_out[c] = v;
  return split_df(v);
}

// Faces: variable-coefficient operator (face arrays); otherwise beta = 1.
// OnTheFlyB: b = rhs * rhs_scale + Dirichlet lifts formed here (FP64);
// otherwise b is read as given (the solver precomputes it once per solve).
template <bool Faces, bool HasE, bool ZeroFree, bool OnTheFlyB>
__global__ void __launch_bounds__(NT) k_ir_df(IrArgs a) {
  __shared__ float2 pl[3][PN];
  __shared__ float red[NT / 32];
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * a.zchunk;
  const int z1 = min(a.op.b.nz, z0 + a.zchunk);
  const int nx = a.op.b.nx, ny = a.op.b.ny, nz = a.op.b.nz;
  const long long sy = nx, sz = (long long)nx * ny;
  const int i = x0 + tx, j = y0 + ty;
  const bool own = i < nx && j < ny;
  // beta = 1: diagonal (in-box faces + 2 per Dirichlet face) / h^2 + alpha
  int dxy = 0;
  if (!Faces) {
    dxy += i > 0 ? 1 : (a.op.dir[0] ? 2 : 0);
    dxy += i < nx - 1 ? 1 : (a.op.dir[1] ? 2 : 0);
    dxy += j > 0 ? 1 : (a.op.dir[2] ? 2 : 0);
    dxy += j < ny - 1 ? 1 : (a.op.dir[3] ? 2 : 0);
  }

  auto load_plane = [&](int buf, int k) {
    const bool kown = k >= z0 && k < z1;
    for (int q = threadIdx.x; q < PN; q += NT) {
      const int lx = q % PX, ly = q / PX;
      const bool own_cell = kown && lx >= 1 && lx <= TX && ly >= 1 && ly <= TY;
      pl[buf][q] = load_cell<HasE, ZeroFree>(a, x0 + lx - 1, y0 + ly - 1, k, own_cell);
    }
  };
  load_plane(0, z0 - 1);
  load_plane(1, z0);
  int b0 = 0, b1 = 1, b2 = 2;
  float ss = 0.0f;
  for (int k = z0; k < z1; ++k) {
    load_plane(b2, k + 1);
    __syncthreads();
    if (own) {
      const long long c = ((long long)k * ny + j) * nx + i;
      const int q = (ty + 1) * PX + (tx + 1);
      float r = 0.0f;
      if (!masked64(a.op, c)) {
        double bd;
        if (OnTheFlyB) {
          bd = a.rhs[c] * a.rhs_scale;
          const bool edge = i == 0 || i == nx - 1 || j == 0 || j == ny - 1 || k == 0 || k == nz - 1;
          if (a.lift && edge) {
            const double l = 2.0 * (a.beta0 ? a.beta0[c] : 1.0) * a.op.ih2;
            if (i == 0 && a.op.dir[0]) bd += l * a.bval.v[0];
            if (i == nx - 1 && a.op.dir[1]) bd += l * a.bval.v[1];
            if (j == 0 && a.op.dir[2]) bd += l * a.bval.v[2];
            if (j == ny - 1 && a.op.dir[3]) bd += l * a.bval.v[3];
            if (k == 0 && a.op.dir[4]) bd += l * a.bval.v[4];
            if (k == nz - 1 && a.op.dir[5]) bd += l * a.bval.v[5];
          }
        } else {
          bd = a.rhs[c];
        }
        const float2 bb = split_df(bd);
        DfAcc acc{bb.x, bb.y};
        // r = b - diag u_c + sum_f w_f u_nb
        if (!ZeroFree) {
          const float2 uc = pl[b1][q];
          float2 dg;
          if (Faces) {
            dg = a.op.Dd[c];
            if (a.has_alpha) acc.add(a.nalpha, uc);
          } else {
            const int d = dxy + (k > 0 ? 1 : (a.op.dir[4] ? 2 : 0)) +
                          (k < nz - 1 ? 1 : (a.op.dir[5] ? 2 : 0));
            dg = a.diag[d];
          }
          acc.add(make_float2(-dg.x, -dg.y), uc);
        }
        if (Faces) {
          if (i > 0) acc.add(a.op.cxd[c], pl[b1][q - 1]);
          if (i < nx - 1) acc.add(a.op.cxd[c + 1], pl[b1][q + 1]);
          if (j > 0) acc.add(a.op.cyd[c], pl[b1][q - PX]);
          if (j < ny - 1) acc.add(a.op.cyd[c + sy], pl[b1][q + PX]);
          if (k > 0) acc.add(a.op.czd[c], pl[b0][q]);
          if (k < nz - 1) acc.add(a.op.czd[c + sz], pl[b2][q]);
        } else {
          const float2 w = a.ih2d;
          if (i > 0) acc.add(w, pl[b1][q - 1]);
          if (i < nx - 1) acc.add(w, pl[b1][q + 1]);
          if (j > 0) acc.add(w, pl[b1][q - PX]);
          if (j < ny - 1) acc.add(w, pl[b1][q + PX]);
          if (k > 0) acc.add(w, pl[b0][q]);
          if (k < nz - 1) acc.add(w, pl[b2][q]);
        }
        r = acc.value();
      }
      if (a.r[0]) (((i + j + k) & 1) ? a.r[1] : a.r[0])[((long long)k * ny + j) * a.W + (i >> 1)] = r;
      ss = fmaf(r, r, ss);
    }
    __syncthreads();
    const int t = b0;
    b0 = b1;
    b1 = b2;
    b2 = t;
  }
  // CTA sum of r^2 (FP32 is ample for a stopping test; the partials and the
  // final sum are accumulated in FP64)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < NT / 32 ? (double)red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0)
      a.partial[((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = v;
  }
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

template <bool F, bool E, bool Z, bool O>
static void go(const IrArgs& a, dim3 g, cudaStream_t s) {
  k_ir_df<F, E, Z, O><<<g, NT, 0, s>>>(a);
}

// double-float of a host double
static float2 df_host(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

// Launch constants: 1/h^2, -alpha and the beta = 1 diagonals d/h^2 + alpha
// (d = in-box faces + 2 per Dirichlet face, 0..12) as double-floats.
static void ir_constants(IrArgs& a) {
  a.ih2d = df_host(a.op.ih2);
  a.nalpha = df_host(-a.alpha);
  for (int d = 0; d <= 12; ++d) a.diag[d] = df_host(d * a.op.ih2 + a.alpha);
  a.has_alpha = a.alpha != 0.0;
}

static void dispatch(const IrArgs& a, dim3 g, bool zero_free, bool on_the_fly, cudaStream_t s) {
  const bool faces = a.op.cxd != nullptr;
  const bool has_e = a.e[0] != nullptr && !zero_free;
  if (on_the_fly) {
    if (faces) go<true, false, false, true>(a, g, s);
    else go<false, false, false, true>(a, g, s);
  } else if (zero_free) {
    if (faces) go<true, false, true, false>(a, g, s);
    else go<false, false, true, false>(a, g, s);
  } else if (has_e) {
    if (faces) go<true, true, false, false>(a, g, s);
    else go<false, true, false, false>(a, g, s);
  } else {
    if (faces) go<true, false, false, false>(a, g, s);
    else go<false, false, false, false>(a, g, s);
  }
}

void launch_ir_fused(const IrArgs& args, bool zero_free, cudaStream_t s) {
  IrArgs a = args;
  dim3 g = ir_grid(a.op.b, &a.zchunk);
  ir_constants(a);
  dispatch(a, g, zero_free, false, s);
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
  dispatch(a, g, false, true, s);
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
    a.op.dir[f] = bc->kind[f] == MG_BC_DIRICHLET;
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
