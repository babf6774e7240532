// Host side of libmg: context and level hierarchy, V-cycle schedules, FP64
// iterative refinement around FP32 V-cycles, instrumentation, and the
// extern "C" entry points declared in include/mg.h.
//
// Method: geometric multigrid with red-black Gauss-Seidel smoothing for the
// second-order cell-centred discretisations of Eqs. 2 and 3 (Sec. 2 of
// arXiv:1809.08857, items (ii)-(iii)).  The paper's bottom solver (BiCGStab)
// is replaced by an exact dense inverse of the small coarsest grid.
//
// Two precision modes:
//  - FP64: V(nu1,nu2)-cycles in FP64 on natural-layout arrays.
//  - mixed: FP64 iterative refinement.  Each step forms r = b - A u in FP64
//    (fused kernel, mg_ir.cu), runs FP32 V-cycles on A e = r in red/black
//    split storage (mg_split32.cu) and adds e to u in the next fused step.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mg.h"
#include "mg_internal.h"

namespace {

constexpr double kEps0 = 8.8541878128e-12;  // F/m (CODATA 2018)
constexpr int kDenseMax = 4096;             // largest coarsest grid inverted densely

thread_local std::string g_last_error;

mg_status fail(mg_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

}  // namespace

void mg::set_last_error(const std::string& msg) { g_last_error = msg; }

namespace {

#define MG_CUDA(call)                                                         \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      return fail(e_ == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA, \
                  std::string(#call) + ": " + cudaGetErrorString(e_));        \
    }                                                                         \
  } while (0)

#define MG_TRY(expr)            \
  do {                          \
    mg_status s_ = (expr);      \
    if (s_ != MG_OK) return s_; \
  } while (0)

enum Kind { kPoisson = 0, kHelmholtz = 1 };

struct Level {
  mg::Box b{};
  double h = 0, ih2 = 0;
  int W = 0;             // packed row width of the split arrays
  long long ns = 0;      // entries per colour array
  uint8_t* mask = nullptr;  // null when there are no electrode cells
  // Poisson FP64 coefficients (null when eps_r == 1 everywhere)
  double* beta64 = nullptr;
  double *cx = nullptr, *cy = nullptr, *cz = nullptr, *D = nullptr;
  // FP32 split coefficients: Poisson (eps or mask), Helmholtz (mask only)
  float* bp[2] = {nullptr, nullptr};
  float* bh[2] = {nullptr, nullptr};
  // FP64 correction arrays (levels >= 1) and coarsest residual
  double *u64 = nullptr, *f64 = nullptr, *r64 = nullptr;
  // FP32 split work arrays
  float* u32[2] = {nullptr, nullptr};
  float* f32[2] = {nullptr, nullptr};
  float* r32[2] = {nullptr, nullptr};
};

struct Coarse {
  int kind;
  double alpha;
  double* Minv;
};

struct ProfRec {
  int cls;
  double bytes;
  cudaEvent_t a, b;
};

}  // namespace

struct mg_ctx {
  mg_grid grid{};
  mg_bc bc{};
  mg_options opt{};
  cudaStream_t stream = nullptr;
  std::vector<Level> lv;
  double* mask_value = nullptr;
  double* b64 = nullptr;      // FP64-mode Poisson right-hand side with lifts
  double* phi_tmp = nullptr;  // ping-pong partner of the caller's iterate
  double* partial = nullptr;
  int npartial = 0;
  double* norm_dev = nullptr;
  double* norm_host = nullptr;  // pinned
  double *gj_row = nullptr, *gj_col = nullptr;
  std::vector<Coarse> coarse;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<void*> allocs;
  // instrumentation
  bool prof = false;
  std::vector<ProfRec> pending;
  std::vector<cudaEvent_t> pool;
  mg_kprof acc[MG_KCLASS_COUNT] = {};

  template <class T>
  mg_status alloc(T** p, size_t count, bool zero = false) {
    *p = nullptr;
    if (count == 0) return MG_OK;
    MG_CUDA(cudaMalloc((void**)p, sizeof(T) * count));
    allocs.push_back(*p);
    if (zero) MG_CUDA(cudaMemsetAsync(*p, 0, sizeof(T) * count, stream));
    return MG_OK;
  }
};

namespace {

// ---- instrumentation --------------------------------------------------------

struct Scope {
  mg_ctx* c;
  int cls;
  double bytes;
  cudaEvent_t a = nullptr;
  Scope(mg_ctx* ctx, int k, double by) : c(ctx), cls(k), bytes(by) {
    c->acc[cls].launches += 1;
    if (!c->prof) return;
    if (c->pool.size() < 2) {
      for (int q = 0; q < 16; ++q) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) == cudaSuccess) c->pool.push_back(e);
      }
    }
    if (c->pool.size() < 2) return;
    a = c->pool.back();
    c->pool.pop_back();
    cudaEventRecord(a, c->stream);
  }
  ~Scope() {
    if (!a) return;
    cudaEvent_t b = c->pool.back();
    c->pool.pop_back();
    cudaEventRecord(b, c->stream);
    c->pending.push_back({cls, bytes, a, b});
  }
};

// After a stream synchronisation: fold the finished event pairs in.
void harvest(mg_ctx* c) {
  for (const ProfRec& r : c->pending) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      c->acc[r.cls].ms += ms;
      c->acc[r.cls].bytes += r.bytes;
    }
    c->pool.push_back(r.a);
    c->pool.push_back(r.b);
  }
  c->pending.clear();
}

uint8_t poisson_dir(const mg_ctx* c, int f) { return c->bc.kind[f] == MG_BC_DIRICHLET; }

mg::Op64 op64(const mg_ctx* c, int l, Kind kind) {
  const Level& L = c->lv[l];
  mg::Op64 op{};
  op.b = L.b;
  op.ih2 = L.ih2;
  op.mask = L.mask;
  if (kind == kPoisson) {
    op.cx = L.cx;
    op.cy = L.cy;
    op.cz = L.cz;
    op.D = L.D;
  }
  for (int f = 0; f < 6; ++f) op.dir[f] = kind == kPoisson ? poisson_dir(c, f) : 1;
  return op;
}

mg::Split32 sop(const mg_ctx* c, int l, Kind kind) {
  const Level& L = c->lv[l];
  mg::Split32 op{};
  op.b = L.b;
  op.W = L.W;
  op.ih2 = (float)L.ih2;
  float* const* beta = kind == kPoisson ? L.bp : L.bh;
  op.beta[0] = beta[0];
  op.beta[1] = beta[1];
  for (int f = 0; f < 6; ++f) op.dir[f] = kind == kPoisson ? poisson_dir(c, f) : 1;
  return op;
}

mg::Ptr2 cp(float* const* a) { return mg::Ptr2{{a[0], a[1]}}; }
mg::MPtr2 mp(float* const* a) { return mg::MPtr2{{a[0], a[1]}}; }

bool can_coarsen(const mg::Box& b) {
  return b.nx % 2 == 0 && b.ny % 2 == 0 && b.nz % 2 == 0 && b.nx >= 8 && b.ny >= 8 && b.nz >= 8;
}

mg_status check_launch() {
  MG_CUDA(cudaGetLastError());
  return MG_OK;
}

// Dense inverse of the coarsest operator for (kind, alpha), built on first use.
mg_status coarse_inverse(mg_ctx* c, Kind kind, double alpha, const double** out) {
  for (const Coarse& q : c->coarse)
    if (q.kind == kind && q.alpha == alpha) {
      *out = q.Minv;
      return MG_OK;
    }
  const int l = (int)c->lv.size() - 1;
  const long long n = c->lv[l].b.n();
  if (n > kDenseMax) return fail(MG_ERR_UNSUPPORTED, "coarsest grid too large for a dense inverse");
  double* M = nullptr;
  MG_TRY(c->alloc(&M, (size_t)n * n));
  mg::launch_assemble_dense(op64(c, l, kind), alpha, M, c->stream);
  mg::launch_gj_invert(M, (int)n, c->gj_row, c->gj_col, c->stream);
  MG_TRY(check_launch());
  c->coarse.push_back({kind, alpha, M});
  *out = M;
  return MG_OK;
}

// ---- FP64 V-cycle (natural layout) ----------------------------------------

mg_status vcycle64(mg_ctx* c, Kind kind, double alpha, int l, const double* f, double* u) {
  cudaStream_t s = c->stream;
  const int Lc = (int)c->lv.size() - 1;
  mg::Op64 op = op64(c, l, kind);
  const double n = (double)op.b.n();
  const double fb = op.cx ? 32.0 : (op.mask ? 1.0 : 0.0);  // coefficient bytes per cell
  const int cls_s = l == 0 ? MG_KCLASS_SMOOTH : MG_KCLASS_COARSE;
  if (l == Lc) {
    const double* Minv;
    MG_TRY(coarse_inverse(c, kind, alpha, &Minv));
    {
      Scope sc(c, MG_KCLASS_COARSE, 0);
      mg::launch_resid64(op, alpha, f, u, c->lv[l].r64, s);
    }
    {
      Scope sc(c, MG_KCLASS_COARSE, 0);
      mg::launch_dense_apply64(Minv, (int)c->lv[l].b.n(), c->lv[l].r64, u, s);
    }
    return check_launch();
  }
  auto smooth = [&](int sweeps) {
    for (int q = 0; q < sweeps; ++q)
      for (int col = 0; col < 2; ++col) {
        Scope sc(c, cls_s, n * (8.0 + 4.0 + 4.0 + fb));
        mg::launch_rbgs64(op, alpha, f, u, col, s);
      }
  };
  smooth(c->opt.nu1);
  Level& C = c->lv[l + 1];
  {
    Scope sc(c, l == 0 ? MG_KCLASS_RESTRICT : MG_KCLASS_COARSE, n * (16.0 + fb + 2.0));
    mg::launch_resid_restrict64(op, alpha, f, u, C.f64, C.u64, s);
  }
  MG_TRY(vcycle64(c, kind, alpha, l + 1, C.f64, C.u64));
  {
    Scope sc(c, l == 0 ? MG_KCLASS_PROLONG : MG_KCLASS_COARSE, n * (16.0 + 1.0 + fb));
    mg::launch_prolong64(op, C.u64, u, s);
  }
  smooth(c->opt.nu2);
  return check_launch();
}

// ---- FP32 V-cycle (red/black split storage) --------------------------------

// first_zero: the level's unknown is zero on entry (the first half-sweep
// need not read the other colour).
mg_status vcycle32(mg_ctx* c, Kind kind, double alpha, int l, bool first_zero) {
  cudaStream_t s = c->stream;
  const int Lc = (int)c->lv.size() - 1;
  Level& L = c->lv[l];
  mg::Split32 op = sop(c, l, kind);
  const float a32 = (float)alpha;
  const double n = (double)L.b.n();
  const double fb = op.beta[0] ? 4.0 : 0.0;
  if (l == Lc) {
    const double* Minv;
    MG_TRY(coarse_inverse(c, kind, alpha, &Minv));
    {
      Scope sc(c, MG_KCLASS_COARSE, 0);
      mg::launch_resid32s(op, a32, cp(L.f32), cp(L.u32), mp(L.r32), s);
    }
    {
      Scope sc(c, MG_KCLASS_COARSE, 0);
      mg::launch_dense_apply32s(op, Minv, cp(L.r32), mp(L.u32), s);
    }
    return check_launch();
  }
  const int cls_s = l == 0 ? MG_KCLASS_SMOOTH : MG_KCLASS_COARSE;
  auto smooth = [&](int sweeps, bool zero) {
    for (int q = 0; q < sweeps; ++q)
      for (int col = 0; col < 2; ++col) {
        const bool zo = zero && q == 0 && col == 0;
        // other colour (unless known zero) + own rhs + own write + coefficients
        Scope sc(c, cls_s, n * ((zo ? 0.0 : 2.0) + 2.0 + 2.0 + fb));
        mg::launch_half_sweep32(op, a32, col, L.f32[col], L.u32[col], L.u32[col ^ 1], zo,
                                L.mask != nullptr, s);
      }
  };
  smooth(c->opt.nu1, first_zero);
  Level& C = c->lv[l + 1];
  mg::Split32 cop = sop(c, l + 1, kind);
  {
    const bool red_only = c->opt.nu1 > 0;
    // u both colours, f (red only if red_only), beta both colours, coarse f and u
    Scope sc(c, l == 0 ? MG_KCLASS_RESTRICT : MG_KCLASS_COARSE,
             n * (4.0 + (red_only ? 2.0 : 4.0) + fb + 1.0));
    mg::launch_resid_restrict32s(op, cop, a32, cp(L.f32), cp(L.u32), mp(C.f32), mp(C.u32),
                                 red_only, s);
  }
  MG_TRY(vcycle32(c, kind, alpha, l + 1, true));
  {
    const bool black_only = c->opt.nu2 > 0;
    // fine u read + write (black only if black_only), coarse e, beta for the electrode test
    Scope sc(c, l == 0 ? MG_KCLASS_PROLONG : MG_KCLASS_COARSE,
             n * ((black_only ? 4.0 : 8.0) + 0.5 + (black_only ? fb / 2 : fb)));
    mg::launch_prolong32s(op, cop, cp(C.u32), mp(L.u32), black_only, s);
  }
  smooth(c->opt.nu2, false);
  return check_launch();
}

// ---- FP64 refinement step / residual norm ----------------------------------

struct Rhs {
  const double* p;
  double scale;
  bool lift;
};

// One fused FP64 pass on level 0 (see mg_ir.cu); returns ||r||_2 (syncs).
mg_status ir_step(mg_ctx* c, Kind kind, double alpha, const Rhs& rhs, const double* u_in,
                  double* u_out, bool with_e, bool store_r, bool zero_free, double* norm) {
  Level& L0 = c->lv[0];
  mg::IrArgs a{};
  a.op = op64(c, 0, kind);
  a.alpha = alpha;
  a.rhs = rhs.p;
  a.rhs_scale = rhs.scale;
  a.lift = rhs.lift ? 1 : 0;
  a.beta0 = L0.beta64;
  for (int f = 0; f < 6; ++f) a.bval.v[f] = kind == kPoisson ? c->bc.value[f] : 0.0;
  a.u_in = u_in;
  a.u_out = u_out;
  a.e[0] = with_e ? L0.u32[0] : nullptr;
  a.e[1] = with_e ? L0.u32[1] : nullptr;
  a.r[0] = store_r ? L0.f32[0] : nullptr;
  a.r[1] = store_r ? L0.f32[1] : nullptr;
  a.W = L0.W;
  a.partial = c->partial;
  const double n = (double)L0.b.n();
  const double bytes = n * (8.0 + 8.0 + (a.op.cx ? 32.0 : (a.op.mask ? 1.0 : 0.0)) +
                            (with_e ? 4.0 : 0.0) + (u_out ? 8.0 : 0.0) + (store_r ? 4.0 : 0.0));
  {
    Scope sc(c, MG_KCLASS_RESID64, bytes);
    mg::launch_ir_fused(a, zero_free, c->stream);
  }
  {
    Scope sc(c, MG_KCLASS_COARSE, 0);
    mg::launch_sum_partials(c->partial, c->npartial, c->norm_dev, c->stream);
  }
  MG_TRY(check_launch());
  MG_CUDA(cudaMemcpyAsync(c->norm_host, c->norm_dev, sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
  MG_CUDA(cudaStreamSynchronize(c->stream));
  harvest(c);
  *norm = std::sqrt(*c->norm_host);
  return MG_OK;
}

// Solve A u = b on level 0 for one problem.  Electrode cells of u already
// hold their values.  b64 (FP64 mode only) is b with the lifts.
mg_status solve_one(mg_ctx* c, Kind kind, double alpha, const Rhs& rhs, const double* b64,
                    double* u, double tol, mg_stats* st) {
  if (st) {
    std::memset(st, 0, sizeof(*st));
    MG_CUDA(cudaEventRecord(c->ev0, c->stream));
  }
  const bool mixed = c->opt.precision == MG_PREC_MIXED;
  double bnorm, rnorm;
  MG_TRY(ir_step(c, kind, alpha, rhs, u, nullptr, false, false, true, &bnorm));
  if (!std::isfinite(bnorm)) return fail(MG_ERR_NONFINITE, "non-finite right-hand side");
  if (bnorm == 0.0) bnorm = 1.0;
  MG_TRY(ir_step(c, kind, alpha, rhs, u, nullptr, false, mixed, false, &rnorm));
  double rel = rnorm / bnorm;
  int cyc = 0;
  if (st) st->hist[0] = rel;
  double* cur = u;
  double* other = c->phi_tmp;
  while (std::isfinite(rel) && rel > tol && cyc < c->opt.max_cycles) {
    if (mixed) {
      for (int q = 0; q < c->opt.inner_cycles; ++q) MG_TRY(vcycle32(c, kind, alpha, 0, q == 0));
      MG_TRY(ir_step(c, kind, alpha, rhs, cur, other, true, true, false, &rnorm));
      std::swap(cur, other);
    } else {
      MG_TRY(vcycle64(c, kind, alpha, 0, b64, u));
      MG_TRY(ir_step(c, kind, alpha, rhs, u, nullptr, false, false, false, &rnorm));
    }
    rel = rnorm / bnorm;
    ++cyc;
    if (st && cyc < 64) st->hist[cyc] = rel;
  }
  if (cur != u) {
    MG_CUDA(cudaMemcpyAsync(u, cur, sizeof(double) * c->lv[0].b.n(), cudaMemcpyDeviceToDevice,
                            c->stream));
  }
  if (st) {
    MG_CUDA(cudaEventRecord(c->ev1, c->stream));
    MG_CUDA(cudaEventSynchronize(c->ev1));
    float ms = 0;
    MG_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    st->cycles = cyc;
    st->rel_resid = rel;
    st->converged = rel <= tol;
    st->time_ms = ms;
  } else {
    MG_CUDA(cudaStreamSynchronize(c->stream));
  }
  harvest(c);
  if (!std::isfinite(rel)) return fail(MG_ERR_NONFINITE, "non-finite residual");
  if (rel > tol) {
    char msg[128];
    std::snprintf(msg, sizeof msg, "not converged: rel. residual %.3e after %d cycles", rel, cyc);
    return fail(MG_ERR_NOT_CONVERGED, msg);
  }
  return MG_OK;
}

void destroy(mg_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (const ProfRec& r : c->pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  for (void* p : c->allocs) cudaFree(p);
  if (c->norm_host) cudaFreeHost(c->norm_host);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  delete c;
}

mg_status build(mg_ctx* c, const double* eps_r, const uint8_t* mask, const double* mask_value) {
  cudaStream_t s = c->stream;
  const mg_grid& g = c->grid;
  mg::Box b{g.nx, g.ny, g.nz};
  double h = g.h;
  for (;;) {
    Level L;
    L.b = b;
    L.h = h;
    L.ih2 = 1.0 / (h * h);
    L.W = (b.nx + 1) / 2;
    L.ns = (long long)L.W * b.ny * b.nz;
    c->lv.push_back(L);
    if (!can_coarsen(b)) break;
    b = mg::Box{b.nx / 2, b.ny / 2, b.nz / 2};
    h *= 2.0;
  }
  const int nlev = (int)c->lv.size();
  for (int l = 0; l < nlev; ++l) {
    Level& L = c->lv[l];
    const size_t n = (size_t)L.b.n();
    if (mask) MG_TRY(c->alloc(&L.mask, n));
    if (eps_r) {
      MG_TRY(c->alloc(&L.beta64, n));
      MG_TRY(c->alloc(&L.cx, n));
      MG_TRY(c->alloc(&L.cy, n));
      MG_TRY(c->alloc(&L.cz, n));
      MG_TRY(c->alloc(&L.D, n));
    }
    for (int col = 0; col < 2; ++col) {
      if (eps_r || mask) MG_TRY(c->alloc(&L.bp[col], (size_t)L.ns, true));
      if (mask) MG_TRY(c->alloc(&L.bh[col], (size_t)L.ns, true));
      MG_TRY(c->alloc(&L.u32[col], (size_t)L.ns, true));
      MG_TRY(c->alloc(&L.f32[col], (size_t)L.ns, true));
      if (l == nlev - 1) MG_TRY(c->alloc(&L.r32[col], (size_t)L.ns, true));
    }
    if (l > 0) {
      MG_TRY(c->alloc(&L.u64, n));
      MG_TRY(c->alloc(&L.f64, n));
    }
    if (l == nlev - 1) MG_TRY(c->alloc(&L.r64, n));
  }
  Level& L0 = c->lv[0];
  const size_t n0 = (size_t)L0.b.n();
  if (mask) MG_CUDA(cudaMemcpyAsync(L0.mask, mask, n0, cudaMemcpyDeviceToDevice, s));
  if (eps_r)
    MG_CUDA(cudaMemcpyAsync(L0.beta64, eps_r, sizeof(double) * n0, cudaMemcpyDeviceToDevice, s));
  if (mask && mask_value) {
    MG_TRY(c->alloc(&c->mask_value, n0));
    MG_CUDA(cudaMemcpyAsync(c->mask_value, mask_value, sizeof(double) * n0,
                            cudaMemcpyDeviceToDevice, s));
  }
  if (eps_r || mask)
    for (int l = 1; l < nlev; ++l)
      mg::launch_coarsen(c->lv[l - 1].beta64, c->lv[l - 1].mask, c->lv[l - 1].b, c->lv[l].beta64,
                         c->lv[l].mask, s);
  uint8_t dir[6];
  for (int f = 0; f < 6; ++f) dir[f] = poisson_dir(c, f);
  for (int l = 0; l < nlev; ++l) {
    Level& L = c->lv[l];
    if (eps_r) mg::launch_faces64(L.beta64, L.mask, L.b, L.ih2, dir, L.cx, L.cy, L.cz, L.D, s);
    if (eps_r || mask) mg::launch_split_beta(L.beta64, L.mask, sop(c, l, kPoisson), mp(L.bp), s);
    if (mask) mg::launch_split_beta(nullptr, L.mask, sop(c, l, kHelmholtz), mp(L.bh), s);
  }
  MG_TRY(c->alloc(&c->b64, n0));
  MG_TRY(c->alloc(&c->phi_tmp, n0));
  c->npartial = mg::ir_partials(L0.b);
  MG_TRY(c->alloc(&c->partial, (size_t)c->npartial));
  MG_TRY(c->alloc(&c->norm_dev, 1));
  const long long nc = c->lv.back().b.n();
  if (nc <= kDenseMax) {
    MG_TRY(c->alloc(&c->gj_row, (size_t)nc));
    MG_TRY(c->alloc(&c->gj_col, (size_t)nc));
  }
  MG_CUDA(cudaMallocHost((void**)&c->norm_host, sizeof(double)));
  MG_CUDA(cudaEventCreate(&c->ev0));
  MG_CUDA(cudaEventCreate(&c->ev1));
  MG_TRY(check_launch());
  MG_CUDA(cudaStreamSynchronize(s));
  if (nc > kDenseMax)
    return fail(MG_ERR_UNSUPPORTED, "grid does not coarsen to <= 4096 cells (need even sizes)");
  return MG_OK;
}

mg_status normalise_options(const mg_options* in, mg_options* out) {
  mg_default_options(out);
  if (!in) return MG_OK;
  if (in->nu1 < 0 || in->nu2 < 0 || in->max_cycles < 0 || in->inner_cycles < 0)
    return fail(MG_ERR_INVALID_ARG, "negative option");
  if (in->precision != MG_PREC_FP64 && in->precision != MG_PREC_MIXED)
    return fail(MG_ERR_INVALID_ARG, "unknown precision");
  for (int q = 0; q < 3; ++q)
    if (in->reserved[q] != 0) return fail(MG_ERR_INVALID_ARG, "reserved option fields must be 0");
  if (in->nu1) out->nu1 = in->nu1;
  if (in->nu2) out->nu2 = in->nu2;
  if (in->max_cycles) out->max_cycles = in->max_cycles;
  if (in->inner_cycles) out->inner_cycles = in->inner_cycles;
  out->precision = in->precision;
  return MG_OK;
}

}  // namespace

extern "C" {

void mg_default_options(mg_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->nu1 = 2;
  opt->nu2 = 2;
  opt->max_cycles = 100;
  opt->precision = MG_PREC_FP64;
  opt->inner_cycles = 1;
}

mg_status mg_create(const mg_grid* grid, const double* eps_r, const uint8_t* mask,
                    const double* mask_value, const mg_bc* bc, const mg_options* opt,
                    void* cuda_stream, mg_ctx** out) {
  g_last_error.clear();
  if (!out) return fail(MG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!grid || !bc) return fail(MG_ERR_INVALID_ARG, "grid or bc is NULL");
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->h > 0.0) || !std::isfinite(grid->h))
    return fail(MG_ERR_INVALID_ARG, "grid sizes must be >= 1 and h > 0");
  for (int f = 0; f < 6; ++f) {
    if (bc->kind[f] != MG_BC_DIRICHLET && bc->kind[f] != MG_BC_NEUMANN)
      return fail(MG_ERR_INVALID_ARG, "bc kind must be MG_BC_DIRICHLET or MG_BC_NEUMANN");
    if (!std::isfinite(bc->value[f])) return fail(MG_ERR_INVALID_ARG, "non-finite bc value");
  }
  mg_options o;
  MG_TRY(normalise_options(opt, &o));
  mg_ctx* c = new (std::nothrow) mg_ctx;
  if (!c) return fail(MG_ERR_OOM, "host allocation failed");
  c->grid = *grid;
  c->bc = *bc;
  c->opt = o;
  c->stream = (cudaStream_t)cuda_stream;
  mg_status st = build(c, eps_r, mask, mask_value);
  if (st != MG_OK) {
    destroy(c);
    return st;
  }
  *out = c;
  return MG_OK;
}

mg_status mg_solve_poisson(mg_ctx* c, const double* rho, double* phi, double tol,
                           mg_stats* stats) {
  g_last_error.clear();
  if (!c || !rho || !phi) return fail(MG_ERR_INVALID_ARG, "NULL argument");
  if (!(tol >= 0.0)) return fail(MG_ERR_INVALID_ARG, "tol must be >= 0");
  Level& L0 = c->lv[0];
  const long long n = L0.b.n();
  cudaStream_t s = c->stream;
  if (L0.mask) {
    Scope sc(c, MG_KCLASS_COARSE, 0);
    mg::launch_set_masked(L0.mask, c->mask_value, n, phi, s);
  }
  // b = rho / eps0 + Dirichlet lifts, formed once per solve
  const Rhs rhs{c->b64, 1.0, false};
  {
    uint8_t dir[6];
    for (int f = 0; f < 6; ++f) dir[f] = poisson_dir(c, f);
    Scope sc(c, MG_KCLASS_COARSE, 0);
    mg::launch_rhs64(rho, 1.0 / kEps0, L0.beta64, L0.mask, L0.b, L0.ih2, dir, c->bc.value,
                     c->b64, s);
  }
  MG_TRY(check_launch());
  return solve_one(c, kPoisson, 0.0, rhs, c->b64, phi, tol, stats);
}

mg_status mg_solve_helmholtz_batch(mg_ctx* c, const double* S, double* const psi[3],
                                   const double kappa[3], double tol, mg_stats stats[3]) {
  g_last_error.clear();
  if (!c || !S || !psi || !kappa) return fail(MG_ERR_INVALID_ARG, "NULL argument");
  if (!(tol >= 0.0)) return fail(MG_ERR_INVALID_ARG, "tol must be >= 0");
  for (int j = 0; j < 3; ++j) {
    if (!psi[j]) return fail(MG_ERR_INVALID_ARG, "psi[j] is NULL");
    if (!(kappa[j] > 0.0) || !std::isfinite(kappa[j]))
      return fail(MG_ERR_INVALID_ARG, "kappa must be finite and > 0");
  }
  Level& L0 = c->lv[0];
  mg_status worst = MG_OK;
  const Rhs rhs{S, 1.0, false};
  for (int j = 0; j < 3; ++j) {
    if (L0.mask) {
      Scope sc(c, MG_KCLASS_COARSE, 0);
      mg::launch_set_masked(L0.mask, nullptr, L0.b.n(), psi[j], c->stream);
    }
    mg_status st = solve_one(c, kHelmholtz, kappa[j] * kappa[j], rhs, S, psi[j], tol,
                             stats ? &stats[j] : nullptr);
    if (st != MG_OK && st != MG_ERR_NOT_CONVERGED) return st;
    if (st != MG_OK) worst = st;
  }
  return worst;
}

mg_status mg_profile_enable(mg_ctx* c, int enable) {
  if (!c) return fail(MG_ERR_INVALID_ARG, "ctx is NULL");
  MG_CUDA(cudaStreamSynchronize(c->stream));
  harvest(c);
  c->prof = enable != 0;
  std::memset(c->acc, 0, sizeof(c->acc));
  return MG_OK;
}

mg_status mg_profile_read(mg_ctx* c, mg_kprof* out, int reset) {
  if (!c || !out) return fail(MG_ERR_INVALID_ARG, "NULL argument");
  MG_CUDA(cudaStreamSynchronize(c->stream));
  harvest(c);
  std::memcpy(out, c->acc, sizeof(c->acc));
  if (reset) std::memset(c->acc, 0, sizeof(c->acc));
  return MG_OK;
}

long long mg_launch_count(void) { return mg::launch_count(); }

mg_status mg_set_stream(mg_ctx* c, void* cuda_stream) {
  if (!c) return fail(MG_ERR_INVALID_ARG, "ctx is NULL");
  c->stream = (cudaStream_t)cuda_stream;
  return MG_OK;
}

mg_status mg_level_info(const mg_ctx* c, int level, int* nlevels, int dims[3]) {
  if (!c) return fail(MG_ERR_INVALID_ARG, "ctx is NULL");
  if (nlevels) *nlevels = (int)c->lv.size();
  if (dims) {
    if (level < 0 || level >= (int)c->lv.size()) return fail(MG_ERR_INVALID_ARG, "bad level");
    dims[0] = c->lv[level].b.nx;
    dims[1] = c->lv[level].b.ny;
    dims[2] = c->lv[level].b.nz;
  }
  return MG_OK;
}

void mg_destroy(mg_ctx* c) { destroy(c); }

const char* mg_error_string(mg_status s) {
  switch (s) {
    case MG_OK: return "success";
    case MG_ERR_INVALID_ARG: return "invalid argument";
    case MG_ERR_CUDA: return "CUDA runtime error";
    case MG_ERR_OOM: return "out of device memory";
    case MG_ERR_NOT_CONVERGED: return "not converged within max_cycles";
    case MG_ERR_NONFINITE: return "non-finite value in input or residual";
    case MG_ERR_UNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

const char* mg_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
