// Host side of libmg: context and level hierarchy, V-cycle schedules, FP64
// iterative refinement around FP32 V-cycles, the concurrent multi-problem
// driver with CUDA-graph steps, instrumentation, and the extern "C" entry
// points declared in include/mg.h.
//
// Method: geometric multigrid with red-black Gauss-Seidel smoothing for the
// second-order cell-centred discretisations of Eqs. 2 and 3 (Sec. 2 of
// arXiv:1809.08857, items (ii)-(iii)).  The paper's bottom solver (BiCGStab)
// is replaced by an exact dense inverse of the small coarsest grid.
//
// Two precision modes:
//  - FP64: V(nu1,nu2)-cycles in FP64 on natural-layout arrays, one problem
//    after the other on the context's stream.
//  - mixed: FP64 iterative refinement.  Each step forms r = b - A u in FP64
//    (fused kernel, mg_ir.cu), runs FP32 V-cycles on A e = r in red/black
//    split storage (mg_split32.cu) and adds e to u in the next fused step.
//    Several problems (the Poisson solve and the three radiative-transfer
//    solves of a time step) run concurrently, each on its own stream with its
//    own work arrays, so the FP64-bound refinement kernels of one problem
//    overlap with the HBM-bound V-cycles of the others.  Each refinement step
//    (inner V-cycles + FP64 step + norm read-back) is captured once as a CUDA
//    graph and replayed.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/mg.h"
#include "mg_diverge.h"
#include "mg_trim.h"
#include "mg_internal.h"

namespace {

constexpr double kEps0 = 8.8541878128e-12;  // F/m (CODATA 2018)
constexpr int kDenseMax = 4096;              // largest coarsest grid inverted densely
constexpr int kIrZchunkMin = 16;             // smallest tile of the refinement pass
constexpr int kMaxWork = 4;                 // concurrent problems per context
constexpr int kMaxGraphs = 8;               // cached step graphs per work slot

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

// Operator data of one level, shared by every problem of the context.
struct Level {
  mg::Box b{};
  double h = 0, ih2 = 0;
  int W = 0;                // packed row width of the split arrays
  long long ns = 0;         // entries per colour array
  uint8_t* mask = nullptr;  // null when there are no electrode cells
  // Poisson FP64 coefficients (null when eps_r == 1 everywhere)
  double* beta64 = nullptr;
  double *cx = nullptr, *cy = nullptr, *cz = nullptr, *D = nullptr;
  // level 0 only: the same as double-floats for the refinement step
  float2 *cxd = nullptr, *cyd = nullptr, *czd = nullptr, *Dd = nullptr;
  // FP32 split coefficients 1/(2 beta): Poisson (eps or mask), Helmholtz (mask only)
  float* bp[2] = {nullptr, nullptr};
  float* bh[2] = {nullptr, nullptr};
  // FP64-mode correction arrays (levels >= 1) and coarsest residual
  double *u64 = nullptr, *f64 = nullptr, *r64 = nullptr;
  // levels >= 1 of a variable-coefficient context with the face-rule coarse
  // operator: FP32 split copies of the face weights (-x, -y, -z) and diagonal
  float* fx[2] = {nullptr, nullptr};
  float* fy[2] = {nullptr, nullptr};
  float* fz[2] = {nullptr, nullptr};
  float* dg[2] = {nullptr, nullptr};
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

// FP32 arrays of one level for one problem
struct LevelWork {
  float* u32[2] = {nullptr, nullptr};
  float* f32[2] = {nullptr, nullptr};
  float* r32[2] = {nullptr, nullptr};
};

// One captured refinement step.
struct StepGraph {
  int kind = 0;
  double alpha = 0;
  int ic = 0, nu1 = 0, nu2 = 0, zc = 0, cv = 0, sz = 0;
  bool prof = false;
  const float2* b = nullptr;
  const float2* u_in = nullptr;
  float2* u_out = nullptr;
  // a stack's step: the members taking part, and per member its work slot,
  // iterate parity and alpha
  unsigned act = 0;
  std::vector<const void*> key;
  std::vector<double> keyd;
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;
  std::vector<ProfRec> recs;  // event pairs baked into the graph (profiling)
  unsigned long long stamp = 0;
};

// Everything one problem needs to run concurrently with the others (or, with
// nb > 1, the stacked FP32 level arrays and stream of nb problems whose
// V-cycles run together; see vcycle32_stack).
struct Work {
  int nb = 1;
  cudaStream_t s = nullptr;
  std::vector<LevelWork> lw;
  double* phi_tmp = nullptr;  // FP64 scratch field (warm start; allocated when needed)
  double* b64 = nullptr;      // right-hand side with lifts (allocated when needed)
  // mixed precision: the iterate as double-floats (ping-pong) and b as
  // double-floats (allocated on the first mixed-precision solve)
  float2* udf[2] = {nullptr, nullptr};
  float2* bdf = nullptr;
  double* partial = nullptr;
  // [3] ([0], [1] norms, [2] the zero-guess flag), pinned; norm_map is its
  // device-side address: the reduction kernel
  // stores the norms there itself, so no copy engine is involved (a small
  // device-to-host copy per step waits behind any bulk download in flight,
  // e.g. the previous time step's answers)
  double* norm_host = nullptr;
  double* norm_map = nullptr;
  cudaEvent_t ev = nullptr, t0 = nullptr, t1 = nullptr;
  std::vector<StepGraph> graphs;
};

}  // namespace

struct mg_ctx {
  mg_grid grid{};
  mg_bc bc{};
  mg_options opt{};
  cudaStream_t stream = nullptr;
  std::vector<Level> lv;
  double* mask_value = nullptr;
  int npartial = 0;  // partial sums allocated (the most any tile, automatic or
                     // settable, needs)
  double *gj_row = nullptr, *gj_col = nullptr;
  std::vector<Coarse> coarse;
  std::vector<Work*> work;
  std::vector<Work*> stacks;  // stacked level arrays, one per stack size in use
  cudaEvent_t fork = nullptr;
  std::vector<void*> allocs;
  std::vector<void*> host_allocs;
  unsigned long long clock = 0;
  // >= 0: every domain face of every level is the Robin face
  // n.grad u + robin_a u = 0 (the correction operator of an AMR box)
  double robin_a = -1.0;
  unsigned* efield_min = nullptr;  // mg_efield scratch (allocated on first use)
  double* efield_dt = nullptr;
  mg_unet* net = nullptr;  // warm-start network
  bool own_net = false;
  // instrumentation
  bool prof = false;
  std::vector<ProfRec> pending;
  std::vector<cudaEvent_t> pool;
  std::vector<ProfRec>* capture = nullptr;  // event pairs go into a graph
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

cudaEvent_t take_event(mg_ctx* c) {
  if (c->pool.empty()) {
    for (int q = 0; q < 16; ++q) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) == cudaSuccess) c->pool.push_back(e);
    }
  }
  if (c->pool.empty()) return nullptr;
  cudaEvent_t e = c->pool.back();
  c->pool.pop_back();
  return e;
}

// Brackets one launch: counts it and, with profiling on, times it with an
// event pair on the launching stream (inside a graph capture the pair
// becomes two event-record nodes of the graph).
struct Scope {
  mg_ctx* c;
  cudaStream_t s;
  int cls;
  double bytes;
  cudaEvent_t a = nullptr;
  Scope(mg_ctx* ctx, cudaStream_t st, int k, double by) : c(ctx), s(st), cls(k), bytes(by) {
    if (!c->capture) c->acc[cls].launches += 1;
    if (!c->prof) return;
    a = take_event(c);
    if (a) record(a);
  }
  // inside a capture, an external record makes a real event-record node
  void record(cudaEvent_t e) {
    if (c->capture) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else cudaEventRecord(e, s);
  }
  ~Scope() {
    if (!a) return;
    cudaEvent_t b = take_event(c);
    if (!b) return;
    record(b);
    (c->capture ? *c->capture : c->pending).push_back({cls, bytes, a, b});
  }
};

// Fold finished event pairs in (after the stream they ran on completed).
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

void harvest_graph(mg_ctx* c, const StepGraph& g) {
  for (const ProfRec& r : g.recs) {
    float ms = 0.0f;
    c->acc[r.cls].launches += 1;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      c->acc[r.cls].ms += ms;
      c->acc[r.cls].bytes += r.bytes;
    }
  }
}

uint8_t poisson_dir(const mg_ctx* c, int f) { return c->bc.kind[f] == MG_BC_DIRICHLET; }

// Face factor rho of face f on a level of cell size h (see Op64): Poisson
// and screened problems use the context's Dirichlet/Neumann faces; the
// Helmholtz problems Psi = 0 (rho = 1) or the Marshak condition
// n.grad Psi + a Psi = 0 with a = (sqrt(3)/2) kappa, kappa = sqrt(alpha)
// (the Eddington closure of Eq. 3, whose coefficient is 3 kappa_p / 2, in
// the Helmholtz scaling kappa = sqrt(3) kappa_p), rho = (ah/2)/(1 + ah/2).
double face_rho(const mg_ctx* c, Kind kind, double alpha, int f, double h) {
  if (c->robin_a >= 0.0) {
    const double ah2 = 0.5 * c->robin_a * h;
    return ah2 / (1.0 + ah2);
  }
  if (kind == kPoisson) return poisson_dir(c, f) ? 1.0 : 0.0;
  if (c->opt.rte_bc == MG_RTE_BC_DIRICHLET) return 1.0;
  const double ah2 = 0.5 * (0.5 * std::sqrt(3.0) * std::sqrt(alpha)) * h;
  return ah2 / (1.0 + ah2);
}

mg::Op64 op64(const mg_ctx* c, int l, Kind kind, double alpha) {
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
    op.cxd = L.cxd;
    op.cyd = L.cyd;
    op.czd = L.czd;
    op.Dd = L.Dd;
  }
  for (int f = 0; f < 6; ++f) op.rho[f] = face_rho(c, kind, alpha, f, L.h);
  return op;
}

mg::Split32 sop(const mg_ctx* c, int l, Kind kind, double alpha) {
  const Level& L = c->lv[l];
  mg::Split32 op{};
  op.b = L.b;
  op.W = L.W;
  op.ih2 = (float)L.ih2;
  float* const* beta = kind == kPoisson ? L.bp : L.bh;
  op.beta[0] = beta[0];
  op.beta[1] = beta[1];
  for (int f = 0; f < 6; ++f) op.rho[f] = (float)face_rho(c, kind, alpha, f, L.h);
  if (kind == kPoisson && L.dg[0])
    for (int col = 0; col < 2; ++col) {
      op.fx[col] = L.fx[col];
      op.fy[col] = L.fy[col];
      op.fz[col] = L.fz[col];
      op.dg[col] = L.dg[col];
    }
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

// Dense inverse of the coarsest operator for (kind, alpha), built on first
// use on the context's stream (never during a graph capture).
mg_status coarse_inverse(mg_ctx* c, Kind kind, double alpha, const double** out) {
  for (const Coarse& q : c->coarse)
    if (q.kind == kind && q.alpha == alpha) {
      *out = q.Minv;
      return MG_OK;
    }
  if (c->capture) return fail(MG_ERR_CUDA, "coarsest inverse requested during a graph capture");
  const int l = (int)c->lv.size() - 1;
  const long long n = c->lv[l].b.n();
  if (n > kDenseMax) return fail(MG_ERR_UNSUPPORTED, "coarsest grid too large for a dense inverse");
  double* M = nullptr;
  MG_TRY(c->alloc(&M, (size_t)n * n));
  mg::launch_assemble_dense(op64(c, l, kind, alpha), alpha, M, c->stream);
  mg::launch_gj_invert(M, (int)n, c->gj_row, c->gj_col, c->stream);
  MG_TRY(check_launch());
  c->coarse.push_back({kind, alpha, M});
  *out = M;
  return MG_OK;
}

// Work slot q (allocated on first use).
mg_status get_work(mg_ctx* c, int q, Work** out) {
  while ((int)c->work.size() <= q) {
    Work* w = new (std::nothrow) Work;
    if (!w) return fail(MG_ERR_OOM, "host allocation failed");
    c->work.push_back(w);
    MG_CUDA(cudaStreamCreateWithFlags(&w->s, cudaStreamNonBlocking));
    MG_CUDA(cudaEventCreateWithFlags(&w->ev, cudaEventDisableTiming));
    MG_CUDA(cudaEventCreate(&w->t0));
    MG_CUDA(cudaEventCreate(&w->t1));
    const int nlev = (int)c->lv.size();
    w->lw.resize(nlev);
    for (int l = 0; l < nlev; ++l)
      for (int col = 0; col < 2; ++col) {
        const size_t ns = (size_t)c->lv[l].ns;
        MG_TRY(c->alloc(&w->lw[l].u32[col], ns, true));
        MG_TRY(c->alloc(&w->lw[l].f32[col], ns, true));
        if (l == nlev - 1) MG_TRY(c->alloc(&w->lw[l].r32[col], ns, true));
      }
    MG_TRY(c->alloc(&w->partial, 2 * (size_t)c->npartial));
    // [0], [1]: norms; [2]: the zero-guess flag
    MG_CUDA(cudaMallocHost((void**)&w->norm_host, 3 * sizeof(double)));
    c->host_allocs.push_back(w->norm_host);
    MG_CUDA(cudaHostGetDevicePointer((void**)&w->norm_map, w->norm_host, 0));
    // the zero fills above ran on the context's stream
    MG_CUDA(cudaStreamSynchronize(c->stream));
  }
  *out = c->work[q];
  return MG_OK;
}

// Cycles on the first coarse level per cycle of the finest level.  On a
// layered medium whose interfaces cut the coarse cells (the dielectric slab),
// one V-cycle from level 1 down leaves the finest level's two-grid correction
// inexact and the fine cycle contracts by 0.16-0.23; two V-cycles there give
// 0.09 (a CPU prototype of the cycle at 64^3 and 128^3: the same rate as a
// full W-cycle, whose deeper revisits add nothing), for about 20 % more work
// per cycle.  The default stays one: with two, the mixed-precision Poisson
// solve of the 512^3 gap problem meets tol in as many refinement steps but
// lands closer to it, and there the error of the answer is 30 times its
// relative residual (3e-9 at 1e-10).
int coarse_visits(const mg_ctx* c, int l) {
  if (l != 0 || c->lv.size() < 3) return 1;
  return c->opt.coarse_visits > 1 ? c->opt.coarse_visits : 1;
}

// ---- FP64 V-cycle (natural layout) ----------------------------------------

mg_status vcycle64(mg_ctx* c, Kind kind, double alpha, int l, const double* f, double* u) {
  cudaStream_t s = c->stream;
  const int Lc = (int)c->lv.size() - 1;
  mg::Op64 op = op64(c, l, kind, alpha);
  const double n = (double)op.b.n();
  const double fb = op.cx ? 32.0 : (op.mask ? 1.0 : 0.0);  // coefficient bytes per cell
  const int cls_s = l == 0 ? MG_KCLASS_SMOOTH : MG_KCLASS_COARSE;
  if (l == Lc) {
    const double* Minv;
    MG_TRY(coarse_inverse(c, kind, alpha, &Minv));
    {
      Scope sc(c, s, MG_KCLASS_COARSE, 0);
      mg::launch_resid64(op, alpha, f, u, c->lv[l].r64, s);
    }
    {
      Scope sc(c, s, MG_KCLASS_COARSE, 0);
      mg::launch_dense_apply64(Minv, (int)c->lv[l].b.n(), c->lv[l].r64, u, s);
    }
    return check_launch();
  }
  auto smooth = [&](int sweeps) {
    for (int q = 0; q < sweeps; ++q)
      for (int col = 0; col < 2; ++col) {
        Scope sc(c, s, cls_s, n * (8.0 + 4.0 + 4.0 + fb));
        mg::launch_rbgs64(op, alpha, f, u, col, s);
      }
  };
  smooth(c->opt.nu1);
  Level& C = c->lv[l + 1];
  {
    Scope sc(c, s, l == 0 ? MG_KCLASS_RESTRICT : MG_KCLASS_COARSE, n * (16.0 + fb + 2.0));
    mg::launch_resid_restrict64(op, alpha, f, u, C.f64, C.u64, s);
  }
  for (int q = coarse_visits(c, l); q > 0; --q)
    MG_TRY(vcycle64(c, kind, alpha, l + 1, C.f64, C.u64));
  {
    Scope sc(c, s, l == 0 ? MG_KCLASS_PROLONG : MG_KCLASS_COARSE, n * (16.0 + 1.0 + fb));
    mg::launch_prolong64(op, op64(c, l + 1, kind, alpha), C.u64, u, s);
  }
  smooth(c->opt.nu2);
  return check_launch();
}

// ---- FP32 V-cycle (red/black split storage) --------------------------------

// first_zero: the level's unknown is zero on entry (the first half-sweep
// need not read the other colour).
mg_status vcycle32(mg_ctx* c, Work* w, Kind kind, double alpha, int l, bool first_zero) {
  cudaStream_t s = w->s;
  const int Lc = (int)c->lv.size() - 1;
  Level& L = c->lv[l];
  LevelWork& X = w->lw[l];
  mg::Split32 op = sop(c, l, kind, alpha);
  const float a32 = (float)alpha;
  const double n = (double)L.b.n();
  // coefficient bytes per cell of a half-sweep: the cell coefficient of both
  // colours, or (face rule) own diagonal and three faces, the other colour's
  // three faces
  const double fb = op.dg[0] ? 14.0 : (op.beta[0] ? 4.0 : 0.0);
  if (l == Lc) {
    const double* Minv;
    MG_TRY(coarse_inverse(c, kind, alpha, &Minv));
    {
      Scope sc(c, s, MG_KCLASS_COARSE, 0);
      if (op.dg[0]) mg::launch_resid32f(op, a32, cp(X.f32), cp(X.u32), mp(X.r32), s);
      else mg::launch_resid32s(op, a32, cp(X.f32), cp(X.u32), mp(X.r32), s);
    }
    {
      Scope sc(c, s, MG_KCLASS_COARSE, 0);
      mg::launch_dense_apply32s(op, Minv, cp(X.r32), mp(X.u32), s);
    }
    return check_launch();
  }
  const int cls_s = l == 0 ? MG_KCLASS_SMOOTH : MG_KCLASS_COARSE;
  auto smooth = [&](int sweeps, bool zero) {
    for (int q = 0; q < sweeps; ++q)
      for (int col = 0; col < 2; ++col) {
        const bool zo = zero && q == 0 && col == 0;
        // other colour (unless known zero) + own rhs + own write + coefficients
        Scope sc(c, s, cls_s, n * ((zo ? 0.0 : 2.0) + 2.0 + 2.0 + fb));
        if (op.dg[0])
          mg::launch_half_sweep32f(op, a32, col, X.f32[col], X.u32[col], X.u32[col ^ 1], zo,
                                   L.mask != nullptr, s);
        else
          mg::launch_half_sweep32(op, a32, col, X.f32[col], X.u32[col], X.u32[col ^ 1], zo,
                                  L.mask != nullptr, c->opt.sweep_zchunk, s);
      }
  };
  smooth(c->opt.nu1, first_zero);
  LevelWork& Y = w->lw[l + 1];
  mg::Split32 cop = sop(c, l + 1, kind, alpha);
  {
    // nu1 >= 1: the pre-smoothing ends with a black half-sweep, so only red
    // cells carry a residual.  u both colours, f red, beta both colours,
    // coarse f and u
    Scope sc(c, s, l == 0 ? MG_KCLASS_RESTRICT : MG_KCLASS_COARSE, n * (4.0 + 2.0 + fb + 1.0));
    if (op.dg[0])
      mg::launch_resid_restrict32f(op, cop, a32, cp(X.f32), cp(X.u32), mp(Y.f32), mp(Y.u32), s);
    else
      mg::launch_resid_restrict32s(op, cop, a32, cp(X.f32), cp(X.u32), mp(Y.f32), mp(Y.u32), s);
  }
  const int visits = coarse_visits(c, l);
  for (int q = 0; q < visits; ++q) MG_TRY(vcycle32(c, w, kind, alpha, l + 1, q == 0));
  {
    // nu2 >= 1: the post-smoothing starts with a red half-sweep, so only
    // black cells take the correction.  Fine black u read + write, coarse
    // e, black beta for the electrode test
    Scope sc(c, s, l == 0 ? MG_KCLASS_PROLONG : MG_KCLASS_COARSE, n * (4.0 + 0.5 + fb / 2));
    // the prolongation reads the fine level's cell coefficient only for its
    // sign (electrode cells stay untouched); on a face-rule level the
    // diagonal carries that sign
    mg::Split32 pop = op;
    if (op.dg[0]) {
      pop.beta[0] = op.dg[0];
      pop.beta[1] = op.dg[1];
    }
    mg::launch_prolong32s(pop, cop, cp(Y.u32), mp(X.u32), s);
  }
  smooth(c->opt.nu2, false);
  return check_launch();
}

// ---- stacked Helmholtz V-cycles -------------------------------------------
//
// The Helmholtz problems of one context (the three terms of Eq. 3) share the
// grid and the constant coefficient and differ in alpha = kappa_j^2 and in
// their right-hand sides.  Their FP32 V-cycles run as one stacked level: in
// every level array the problems follow one another along z (Split32::nb,
// nzp), so each half-sweep, restriction and prolongation of a level is one
// launch for all of them, and a problem that has met tol drops out through
// the active mask while the others go on.  Each problem keeps its own
// double-float iterate, b, refinement pass, norms and statistics; the
// coarsest level is solved per problem (its own dense inverse for its alpha).

// A context's Helmholtz problems are stacked if its options ask for it and the
// grid allows it: no electrode cells (the
// constant-coefficient kernels), domain faces that do not depend on alpha
// (Dirichlet radiative-transfer faces, no composite-solve Robin faces), and an
// even number of planes on every level (a cell's colour is then the same
// counted in its problem or in the stack).
bool stack_ok(const mg_ctx* c) {
  if (!c->opt.stack || c->lv[0].mask || c->robin_a >= 0.0 ||
      c->opt.rte_bc != MG_RTE_BC_DIRICHLET)
    return false;
  for (const Level& L : c->lv)
    if (L.b.nz % 2 != 0 || L.bh[0]) return false;
  return true;
}

// The stacked work of nb problems (allocated on first use).
mg_status get_stack(mg_ctx* c, int nb, Work** out) {
  for (Work* w : c->stacks)
    if (w->nb == nb) {
      *out = w;
      return MG_OK;
    }
  Work* w = new (std::nothrow) Work;
  if (!w) return fail(MG_ERR_OOM, "host allocation failed");
  c->stacks.push_back(w);
  w->nb = nb;
  MG_CUDA(cudaStreamCreateWithFlags(&w->s, cudaStreamNonBlocking));
  MG_CUDA(cudaEventCreateWithFlags(&w->ev, cudaEventDisableTiming));
  const int nlev = (int)c->lv.size();
  w->lw.resize(nlev);
  for (int l = 0; l < nlev; ++l)
    for (int col = 0; col < 2; ++col) {
      const size_t ns = (size_t)c->lv[l].ns * nb;
      MG_TRY(c->alloc(&w->lw[l].u32[col], ns, true));
      MG_TRY(c->alloc(&w->lw[l].f32[col], ns, true));
      if (l == nlev - 1) MG_TRY(c->alloc(&w->lw[l].r32[col], ns, true));
    }
  MG_CUDA(cudaStreamSynchronize(c->stream));
  *out = w;
  return MG_OK;
}

// The level-l operator of a stack of nb Helmholtz problems (its planes span
// the stack) and the stack's description (alpha[q] of member q; bit q of
// active: member q takes part).
mg::Split32 sop_stack(const mg_ctx* c, int l, const double* alpha, int nb, unsigned active,
                      mg::Stk32* st) {
  mg::Split32 op = sop(c, l, kHelmholtz, alpha[0]);
  op.b.nz *= nb;
  *st = mg::Stk32{};
  st->nb = nb;
  st->nzp = c->lv[l].b.nz;
  st->active = active;
  for (int q = 0; q < nb; ++q) st->pa[q] = (float)alpha[q];
  return op;
}

int popcount(unsigned v) {
  int k = 0;
  for (; v; v &= v - 1) ++k;
  return k;
}

// One FP32 V-cycle of the active members of a stack from level l down
// (vcycle32 for nb problems at once).
mg_status vcycle32_stack(mg_ctx* c, Work* w, const double* alpha, unsigned active, int l,
                         bool first_zero) {
  cudaStream_t s = w->s;
  const int nb = w->nb;
  const int Lc = (int)c->lv.size() - 1;
  Level& L = c->lv[l];
  LevelWork& X = w->lw[l];
  const double n = (double)L.b.n() * popcount(active);
  if (l == Lc) {
    for (int q = 0; q < nb; ++q) {
      if (!((active >> q) & 1u)) continue;
      const double* Minv;
      MG_TRY(coarse_inverse(c, kHelmholtz, alpha[q], &Minv));
      const mg::Split32 op = sop(c, l, kHelmholtz, alpha[q]);
      const long long o = (long long)q * L.ns;
      float* f[2] = {X.f32[0] + o, X.f32[1] + o};
      float* u[2] = {X.u32[0] + o, X.u32[1] + o};
      float* r[2] = {X.r32[0] + o, X.r32[1] + o};
      {
        Scope sc(c, s, MG_KCLASS_COARSE, 0);
        mg::launch_resid32s(op, (float)alpha[q], cp(f), cp(u), mp(r), s);
      }
      {
        Scope sc(c, s, MG_KCLASS_COARSE, 0);
        mg::launch_dense_apply32s(op, Minv, cp(r), mp(u), s);
      }
    }
    return check_launch();
  }
  mg::Stk32 st;
  const mg::Split32 op = sop_stack(c, l, alpha, nb, active, &st);
  const float a32 = (float)alpha[0];  // the kernels take each member's from st.pa
  const int cls_s = l == 0 ? MG_KCLASS_SMOOTH : MG_KCLASS_COARSE;
  auto smooth = [&](int sweeps, bool zero) {
    for (int q = 0; q < sweeps; ++q)
      for (int col = 0; col < 2; ++col) {
        const bool zo = zero && q == 0 && col == 0;
        Scope sc(c, s, cls_s, n * ((zo ? 0.0 : 2.0) + 2.0 + 2.0));
        mg::launch_half_sweep32(op, a32, col, X.f32[col], X.u32[col], X.u32[col ^ 1], zo, false,
                                c->opt.sweep_zchunk, s, &st);
      }
  };
  smooth(c->opt.nu1, first_zero);
  LevelWork& Y = w->lw[l + 1];
  mg::Stk32 cst;
  const mg::Split32 cop = sop_stack(c, l + 1, alpha, nb, active, &cst);
  {
    Scope sc(c, s, l == 0 ? MG_KCLASS_RESTRICT : MG_KCLASS_COARSE, n * (4.0 + 2.0 + 1.0));
    mg::launch_resid_restrict32s(op, cop, a32, cp(X.f32), cp(X.u32), mp(Y.f32), mp(Y.u32), s,
                                 &st);
  }
  const int visits = coarse_visits(c, l);
  for (int q = 0; q < visits; ++q)
    MG_TRY(vcycle32_stack(c, w, alpha, active, l + 1, q == 0));
  {
    Scope sc(c, s, l == 0 ? MG_KCLASS_PROLONG : MG_KCLASS_COARSE, n * (4.0 + 0.5));
    mg::launch_prolong32s(op, cop, cp(Y.u32), mp(X.u32), s, &st);
  }
  smooth(c->opt.nu2, false);
  return check_launch();
}

// ---- FP64 refinement step / residual norm ----------------------------------

// Operands of one refinement pass: b as double-floats (bdf) or FP64 (b64,
// then optionally written back as double-floats to bdf_out); the iterate as
// double-floats (udf_in, with the correction e of work slot w when with_e)
// or FP64 (u64); u + e written as double-floats to udf_out (nullable).
// znorm (FP64 iterate only): the same pass also sums ||b||^2, the squared
// residual of the guess that is 0 on free cells, into norm slot 0.
struct IrIo {
  const float2* bdf = nullptr;
  const double* b64 = nullptr;
  float2* bdf_out = nullptr;
  const float2* udf_in = nullptr;
  const double* u64 = nullptr;
  float2* udf_out = nullptr;
  bool with_e = false;
  bool store_r = false;
  bool znorm = false;
  double in_scale = 1.0;  // FP64 inputs (b64, u64) multiplied by this power of two on load
  bool zero_guess = false;  // first pass of a zero guess without electrodes (pointwise)
  // the correction e and the residual r in other split arrays than the work
  // slot's level 0 (a member's slice of a stack); null: the work slot's
  const float* e_ptr[2] = {nullptr, nullptr};
  float* r_ptr[2] = {nullptr, nullptr};
};

// Enqueue one fused refinement pass on level 0 and the read-back of ||r||^2
// into w->norm_host[slot] (and of ||b||^2 into norm_host[0] with znorm;
// then slot must be 1) (asynchronous).
mg_status enqueue_ir(mg_ctx* c, Work* w, cudaStream_t s, Kind kind, double alpha, const IrIo& io,
                     int slot) {
  Level& L0 = c->lv[0];
  LevelWork& X = w->lw[0];
  mg::IrArgs a{};
  a.op = op64(c, 0, kind, alpha);
  a.alpha = alpha;
  a.bdf = io.bdf;
  a.rhs = io.b64;
  a.rhs_scale = 1.0;
  a.lift = 0;
  a.beta0 = L0.beta64;
  a.bdf_out = io.bdf_out;
  a.udf_in = io.udf_in;
  a.u_in = io.u64;
  a.udf_out = io.udf_out;
  for (int col = 0; col < 2; ++col) {
    a.e[col] = io.with_e ? (io.e_ptr[col] ? io.e_ptr[col] : X.u32[col]) : nullptr;
    a.r[col] = io.store_r ? (io.r_ptr[col] ? io.r_ptr[col] : X.f32[col]) : nullptr;
  }
  a.W = L0.W;
  a.partial = w->partial;
  a.partial_z = io.znorm ? w->partial + c->npartial : nullptr;
  a.zchunk = c->opt.ir_zchunk;
  a.in_scale = io.in_scale;
  const double n = (double)L0.b.n();
  // u and b read, face arrays (or the electrode mask), e, u + e and b
  // written back, r
  const double bytes = n * (8.0 + 8.0 + (a.op.cxd ? 32.0 : (a.op.mask ? 1.0 : 0.0)) +
                            (io.with_e ? 4.0 : 0.0) + (io.udf_out ? 8.0 : 0.0) +
                            (io.bdf_out ? 8.0 : 0.0) + (io.store_r ? 4.0 : 0.0));
  int nparts;
  if (io.zero_guess) {
    // b read, b and the zero iterate written as double-floats, r written
    Scope sc(c, s, MG_KCLASS_RESID64, n * (8.0 + 8.0 + 8.0 + 4.0));
    nparts = mg::launch_first_zero(a, c->npartial, s);
  } else {
    Scope sc(c, s, MG_KCLASS_RESID64, bytes);
    nparts = mg::launch_ir_fused(a, s);
  }
  {
    Scope sc(c, s, MG_KCLASS_COARSE, 0);
    mg::launch_sum_partials(w->partial, nparts, w->norm_map + slot, s);
    if (io.znorm) mg::launch_sum_partials(a.partial_z, nparts, w->norm_map, s);
  }
  return check_launch();
}

struct Stack;

// One problem of a (possibly concurrent) solve.
struct Prob {
  mg_ctx* c;
  Kind kind;
  double alpha;
  const double* rhs;    // rho (Poisson, C/m^3) or S (Helmholtz)
  const double* faces;  // packed Dirichlet face data, or null
  double* u;            // caller's iterate
  double tol;
  mg_stats* st;
  Work* w = nullptr;
  double rhs_scale = 1.0;     // operator of kind Poisson: b = rhs * rhs_scale + lifts
  const double* b = nullptr;  // right-hand side with lifts
  float2* cur = nullptr;      // double-float iterate (mixed precision)
  float2* other = nullptr;
  int cyc = 0;
  double bnorm = 1.0, rel = 0.0;
  double rel_prev = 0.0;  // relative residual before the last step
  int ic = 0;             // inner V-cycles of the next (last enqueued) step
  int ic_last = 0;        // inner V-cycles of the step that just finished
  int vcycles = 0;        // inner V-cycles of all finished steps
  // mixed precision: the problem is solved for s u (s a power of two, 1
  // unless b's magnitude is far from 1; see rescale)
  double scale = 1.0;
  bool zero_guess = false;  // the guess is 0 and the grid has no electrode cells
  mg::Growth growth;        // divergence rule over the relative residuals
  bool diverged = false;
  int phase = 0;
  bool done = false;
  mg_status status = MG_OK;
  const StepGraph* g = nullptr;
  // member sq of a stack: its refinement steps run with the stack's
  // (waiting: ready for the stack's next step)
  Stack* stk = nullptr;
  int sq = 0;
  bool waiting = false;
};

// Helmholtz problems of one context stepping together (vcycle32_stack).
struct Stack {
  mg_ctx* c = nullptr;
  Work* w = nullptr;          // stacked level arrays, stream, step graphs
  std::vector<Prob*> m;       // members, m[q] has sq = q
  double alpha[mg::kMaxStack] = {};
  bool started = false;       // the first step has been enqueued
  bool running = false;       // a step is in flight on w->s
  unsigned stepping = 0;      // members of the step in flight
  int ic = 0;                 // its inner V-cycles
  const StepGraph* g = nullptr;
};

// Inner V-cycles of p's next refinement step (the trimming rule of mg_trim.h).
int next_inner_cycles(const Prob& p) {
  return mg::trimmed_inner_cycles(p.c->opt.inner_cycles, p.c->opt.fixed_cycles != 0, p.cyc,
                                  p.ic_last, p.rel_prev, p.rel, p.tol);
}

// kind Poisson with alpha = 0 is Eq. 2 (b = rho / eps0 + lifts); with
// rhs_scale = 1 and any alpha >= 0 it is the screened variable-coefficient
// problem alpha u - div(beta grad u) = f of mg_solve_screened.
Prob make_prob(mg_ctx* c, Kind kind, double alpha, const double* rhs, const double* faces,
               double* u, double tol, mg_stats* st, double rhs_scale = 1.0 / kEps0) {
  Prob p;
  p.c = c;
  p.kind = kind;
  p.alpha = alpha;
  p.rhs_scale = kind == kPoisson ? rhs_scale : 1.0;  // set after the call for a scaled source
  p.rhs = rhs;
  p.faces = faces;
  p.u = u;
  p.tol = tol;
  p.st = st;
  return p;
}

// Electrode values into u and the right-hand side with lifts, on stream s:
// Poisson b = rho/eps0 + lifts (screened: f + lifts); Helmholtz b = S (+
// lifts of face data).
// b = rhs * scale + the domain-face lifts of the problem kind (Dirichlet
// values of the context's bc, or the packed face data) into out, on stream s.
mg_status form_b(mg_ctx* c, Kind kind, double scale, const double* rhs, const double* faces,
                 double* out, cudaStream_t s) {
  Level& L0 = c->lv[0];
  uint8_t dir[6];
  double zero[6] = {0, 0, 0, 0, 0, 0};
  for (int f = 0; f < 6; ++f)
    dir[f] = kind == kPoisson ? poisson_dir(c, f) : c->opt.rte_bc == MG_RTE_BC_DIRICHLET;
  {
    Scope sc(c, s, MG_KCLASS_COARSE, 0);
    if (kind == kPoisson)
      mg::launch_rhs64(rhs, scale, L0.beta64, L0.mask, L0.b, L0.ih2, dir, c->bc.value, faces, out,
                       s);
    else
      mg::launch_rhs64(rhs, scale, nullptr, L0.mask, L0.b, L0.ih2, dir, zero, faces, out, s);
  }
  return check_launch();
}

mg_status prepare(Prob& p, cudaStream_t s) {
  mg_ctx* c = p.c;
  Level& L0 = c->lv[0];
  if (L0.mask) {
    Scope sc(c, s, MG_KCLASS_COARSE, 0);
    mg::launch_set_masked(L0.mask, p.kind == kPoisson ? c->mask_value : nullptr, L0.b.n(), p.u, s);
  }
  if (p.kind == kHelmholtz && !p.faces && p.rhs_scale == 1.0) {
    p.b = p.rhs;
    return check_launch();
  }
  if (!p.w->b64) MG_TRY(c->alloc(&p.w->b64, (size_t)L0.b.n()));
  MG_TRY(form_b(c, p.kind, p.rhs_scale, p.rhs, p.faces, p.w->b64, s));
  p.b = p.w->b64;
  return MG_OK;
}

// The refinement step of p: inner V-cycles on A e = r, then the fused FP64
// step u_out = u_in + e, r = b - A u_out, ||r||^2 -> host slot 1.
mg_status enqueue_step_direct(Prob& p) {
  mg_ctx* c = p.c;
  for (int q = 0; q < p.ic; ++q)
    MG_TRY(vcycle32(c, p.w, p.kind, p.alpha, 0, q == 0));
  IrIo io;
  io.bdf = p.w->bdf;
  io.udf_in = p.cur;
  io.udf_out = p.other;
  io.with_e = true;
  io.store_r = true;
  return enqueue_ir(c, p.w, p.w->s, p.kind, p.alpha, io, 1);
}

// Captures body() on w's stream into g (whose key the caller set; the option
// fields are filled here), evicting the least recently used graph of w when
// it holds kMaxGraphs; *out points at the stored graph.
template <class Body>
mg_status capture_step(mg_ctx* c, Work* w, StepGraph&& g, Body body, const StepGraph** out) {
  if ((int)w->graphs.size() >= kMaxGraphs) {  // evict the least recently used
    size_t old = 0;
    for (size_t q = 1; q < w->graphs.size(); ++q)
      if (w->graphs[q].stamp < w->graphs[old].stamp) old = q;
    cudaGraphExecDestroy(w->graphs[old].exec);
    for (const ProfRec& r : w->graphs[old].recs) {
      c->pool.push_back(r.a);
      c->pool.push_back(r.b);
    }
    w->graphs.erase(w->graphs.begin() + old);
  }
  g.nu1 = c->opt.nu1;
  g.nu2 = c->opt.nu2;
  g.zc = c->opt.ir_zchunk;
  g.cv = c->opt.coarse_visits;
  g.sz = c->opt.sweep_zchunk;
  g.prof = c->prof;
  // the event pool must not need to grow inside the capture
  if (c->prof)
    while (c->pool.size() < 1024) {
      cudaEvent_t e;
      MG_CUDA(cudaEventCreate(&e));
      c->pool.push_back(e);
    }
  const long long l0 = mg::launch_count();
  MG_CUDA(cudaStreamBeginCapture(w->s, cudaStreamCaptureModeThreadLocal));
  c->capture = &g.recs;
  mg_status st = body();
  c->capture = nullptr;
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(w->s, &graph);
  if (st != MG_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ec != cudaSuccess)
    return fail(MG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
  const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess)
    return fail(MG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
  g.launches = mg::launch_count() - l0;
  mg::add_launches(-g.launches);  // counted again at every replay
  g.stamp = ++c->clock;
  w->graphs.push_back(std::move(g));
  *out = &w->graphs.back();
  return MG_OK;
}

// Cached graph of the step for p's current (u_in, u_out) parity.
mg_status step_graph(Prob& p, const StepGraph** out) {
  mg_ctx* c = p.c;
  Work* w = p.w;
  const int ic = p.ic;
  for (StepGraph& g : w->graphs)
    if (g.kind == p.kind && g.alpha == p.alpha && g.ic == ic && g.nu1 == c->opt.nu1 &&
        g.nu2 == c->opt.nu2 && g.zc == c->opt.ir_zchunk && g.cv == c->opt.coarse_visits &&
        g.sz == c->opt.sweep_zchunk && g.prof == c->prof && g.b == w->bdf &&
        g.u_in == p.cur &&
        g.u_out == p.other) {
      g.stamp = ++c->clock;
      *out = &g;
      return MG_OK;
    }
  const double* Minv;
  MG_TRY(coarse_inverse(c, p.kind, p.alpha, &Minv));  // never inside the capture
  StepGraph g;
  g.kind = p.kind;
  g.alpha = p.alpha;
  g.ic = ic;
  g.b = w->bdf;
  g.u_in = p.cur;
  g.u_out = p.other;
  return capture_step(c, w, std::move(g), [&] { return enqueue_step_direct(p); }, out);
}

mg_status enqueue_step(Prob& p) {
  p.g = nullptr;
  if (p.stk) {  // the stack's next step takes it (solve_mixed)
    p.waiting = true;
    return MG_OK;
  }
  if (p.c->opt.no_graphs) {
    MG_TRY(enqueue_step_direct(p));
  } else {
    const StepGraph* g;
    MG_TRY(step_graph(p, &g));
    MG_CUDA(cudaGraphLaunch(g->exec, p.w->s));
    mg::add_launches(g->launches);
    p.g = g;
  }
  MG_CUDA(cudaEventRecord(p.w->ev, p.w->s));
  return MG_OK;
}

// The stack's refinement step for the members in act: ic stacked V-cycles on
// their residuals, then each member's refinement pass (u_out = u_in + e,
// r = b - A u_out into its slice of the stack's level 0, ||r||^2 into its
// host slot 1), all on the stack's stream.
mg_status enqueue_stack_direct(Stack& S, unsigned act, int ic) {
  mg_ctx* c = S.c;
  for (int v = 0; v < ic; ++v) MG_TRY(vcycle32_stack(c, S.w, S.alpha, act, 0, v == 0));
  const long long ns0 = c->lv[0].ns;
  LevelWork& X = S.w->lw[0];
  for (Prob* pp : S.m) {
    Prob& p = *pp;
    if (!((act >> p.sq) & 1u)) continue;
    IrIo io;
    io.bdf = p.w->bdf;
    io.udf_in = p.cur;
    io.udf_out = p.other;
    io.with_e = true;
    io.store_r = true;
    for (int col = 0; col < 2; ++col) {
      io.e_ptr[col] = X.u32[col] + p.sq * ns0;
      io.r_ptr[col] = X.f32[col] + p.sq * ns0;
    }
    MG_TRY(enqueue_ir(c, p.w, S.w->s, p.kind, p.alpha, io, 1));
  }
  return MG_OK;
}

// Cached graph of the stack's step (members act, ic inner V-cycles, the
// members' current iterate parity).
mg_status stack_graph(Stack& S, unsigned act, int ic, const StepGraph** out) {
  mg_ctx* c = S.c;
  Work* w = S.w;
  std::vector<const void*> key;
  std::vector<double> keyd;
  for (const Prob* p : S.m) {
    key.push_back(p->w);
    key.push_back(p->cur);
    keyd.push_back(p->alpha);
  }
  for (StepGraph& g : w->graphs)
    if (g.act == act && g.ic == ic && g.nu1 == c->opt.nu1 && g.nu2 == c->opt.nu2 &&
        g.zc == c->opt.ir_zchunk && g.cv == c->opt.coarse_visits &&
        g.sz == c->opt.sweep_zchunk && g.prof == c->prof && g.key == key && g.keyd == keyd) {
      g.stamp = ++c->clock;
      *out = &g;
      return MG_OK;
    }
  for (const Prob* p : S.m) {
    const double* Minv;
    MG_TRY(coarse_inverse(c, kHelmholtz, p->alpha, &Minv));  // never inside the capture
  }
  StepGraph g;
  g.kind = kHelmholtz;
  g.ic = ic;
  g.act = act;
  g.key = std::move(key);
  g.keyd = std::move(keyd);
  return capture_step(c, w, std::move(g), [&] { return enqueue_stack_direct(S, act, ic); }, out);
}

// Enqueue the stack's next step for the members in act (all of them wait).
mg_status enqueue_stack_step(Stack& S, unsigned act, int ic) {
  for (Prob* p : S.m)
    if ((act >> p->sq) & 1u) {
      p->ic = ic;
      // the member's first pass (or its last own work) precedes the step
      if (!S.started) MG_CUDA(cudaStreamWaitEvent(S.w->s, p->w->ev, 0));
    }
  S.started = true;
  S.g = nullptr;
  if (S.c->opt.no_graphs) {
    MG_TRY(enqueue_stack_direct(S, act, ic));
  } else {
    const StepGraph* g;
    MG_TRY(stack_graph(S, act, ic, &g));
    MG_CUDA(cudaGraphLaunch(g->exec, S.w->s));
    mg::add_launches(g->launches);
    S.g = g;
  }
  MG_CUDA(cudaEventRecord(S.w->ev, S.w->s));
  S.running = true;
  S.stepping = act;
  S.ic = ic;
  return MG_OK;
}

mg_status finish(Prob& p) {
  // a stack member's last step ran on the stack's stream
  if (p.stk && p.stk->started) MG_CUDA(cudaStreamWaitEvent(p.w->s, p.stk->w->ev, 0));
  // the iterate back to FP64 (electrode cells keep their values); without a
  // step the caller's guess stays as it was
  if (p.cyc > 0) {
    Scope sc(p.c, p.w->s, MG_KCLASS_COARSE, 0);
    mg::launch_df_to_f64(p.cur, p.c->lv[0].mask, p.u, p.c->lv[0].b.n(), 1.0 / p.scale, p.w->s);
  }
  if (p.st) MG_CUDA(cudaEventRecord(p.w->t1, p.w->s));
  p.done = true;
  if (!std::isfinite(p.rel)) {
    p.status = MG_ERR_NONFINITE;
    g_last_error = "non-finite value in input or residual";
  } else if (p.rel > p.tol) {
    p.status = p.diverged ? MG_ERR_DIVERGED : MG_ERR_NOT_CONVERGED;
    char msg[128];
    std::snprintf(msg, sizeof msg, "%s: rel. residual %.3e after %d steps",
                  p.diverged ? "diverged" : "not converged", p.rel, p.cyc);
    g_last_error = msg;
  }
  return MG_OK;
}

// The first pass of p: ||b|| (slot 0) and the residual of the guess (slot
// 1) in one pass; b and the guess become double-floats (times p.scale) on
// the way.
mg_status enqueue_first(Prob& p) {
  Work* w = p.w;
  IrIo r0;
  r0.b64 = p.b;
  r0.bdf_out = w->bdf;
  r0.u64 = p.u;
  r0.udf_out = p.cur;
  r0.store_r = true;
  r0.znorm = true;
  r0.in_scale = p.scale;
  r0.zero_guess = p.zero_guess;
  if (p.stk) {
    const long long o = p.sq * p.c->lv[0].ns;
    for (int col = 0; col < 2; ++col) r0.r_ptr[col] = p.stk->w->lw[0].f32[col] + o;
  }
  MG_TRY(enqueue_ir(p.c, w, w->s, p.kind, p.alpha, r0, 1));
  MG_CUDA(cudaEventRecord(w->ev, w->s));
  return MG_OK;
}

// Double-floats keep 48 bits only for magnitudes between about 2^-100
// (below 2^-74 the low part is dropped) and the FP32 range: a problem whose
// b is far below that (a radiative-transfer sub-box far from the source,
// with Psi ~ 1e-20) would be solved to FP32 accuracy.  The relative residual
// does not change when b and u are scaled together, so such a problem is
// solved for s u with s = 2^k bringing the RMS of b near 1 (exact: a power of
// two), and the answer divided by s at the end.  Returns the scale for an
// RMS of b (1 inside [2^-30, 2^30]).
double rescale(double bnorm, long long n) {
  const double rms = bnorm / std::sqrt((double)std::max(1LL, n));
  if (!(rms > 0.0) || !std::isfinite(rms) || (rms >= 0x1p-30 && rms <= 0x1p30)) return 1.0;
  return std::ldexp(1.0, -std::ilogb(rms));
}

// ||b|| of p in plain FP64 (the zero guess's residual with the electrode
// values kept, mg_residual_norms' kernel), on p's stream; synchronises it.
// The first pass sums squares in FP32, which underflow for |b| below about
// 1e-19, so a problem of that size shows ||b|| = 0 there.
mg_status fp64_bnorm(Prob& p, double* out) {
  mg_ctx* c = p.c;
  Work* w = p.w;
  const Level& L0 = c->lv[0];
  const int nblk = mg::resid_norms_blocks(L0.b, c->npartial);
  {
    Scope sc(c, w->s, MG_KCLASS_COARSE, 0);
    mg::launch_resid_norms64(op64(c, 0, p.kind, p.alpha), p.alpha, p.b, p.u, w->partial, nblk,
                             w->s);
    mg::launch_sum_partials(w->partial + nblk, nblk, w->norm_map, w->s);
  }
  MG_TRY(check_launch());
  MG_CUDA(cudaStreamSynchronize(w->s));
  *out = std::sqrt(w->norm_host[0]);
  return MG_OK;
}

// Host side of one finished step of p.
mg_status advance(Prob& p) {
  const double* h = p.w->norm_host;
  if (p.g) harvest_graph(p.c, *p.g);
  if (p.phase == 0) {
    p.bnorm = std::sqrt(h[0]);
    if (!std::isfinite(p.bnorm)) {
      p.rel = p.bnorm;
      return finish(p);
    }
    const long long n = p.c->lv[0].b.n();
    if (p.scale == 1.0 && (p.bnorm == 0.0 || rescale(p.bnorm, n) != 1.0)) {
      double b64 = 0.0;
      MG_TRY(fp64_bnorm(p, &b64));
      const double sc = rescale(b64, n);
      if (sc != 1.0) {  // the first pass again, on the scaled problem
        p.scale = sc;
        return enqueue_first(p);
      }
    }
    if (p.bnorm == 0.0) p.bnorm = 1.0;
    p.phase = 1;
  } else {
    std::swap(p.cur, p.other);
    ++p.cyc;
    p.vcycles += p.ic;
  }
  p.rel_prev = p.rel;
  p.rel = std::sqrt(h[1]) / p.bnorm;
  if (p.st && p.cyc < 64) p.st->hist[p.cyc] = p.rel;
  p.diverged = p.growth.push(p.rel) && p.rel > p.tol;
  if (!std::isfinite(p.rel) || p.rel <= p.tol || p.cyc >= p.c->opt.max_cycles || p.diverged)
    return finish(p);
  p.ic_last = p.ic;
  p.ic = next_inner_cycles(p);
  return enqueue_step(p);
}

// Mixed-precision solve of problems concurrently: every problem gets a work
// slot (its own stream and arrays) of its context.  Returns the worst
// status; outputs are complete on return.
mg_status solve_mixed(std::vector<Prob>& P) {
  std::vector<mg_ctx*> ctxs;
  for (Prob& p : P) {
    int slot = 0;
    for (Prob& o : P) {
      if (&o == &p) break;
      if (o.c == p.c) ++slot;
    }
    MG_TRY(get_work(p.c, slot, &p.w));
    const size_t n = (size_t)p.c->lv[0].b.n();
    if (!p.w->bdf) {
      MG_TRY(p.c->alloc(&p.w->udf[0], n));
      MG_TRY(p.c->alloc(&p.w->udf[1], n));
      MG_TRY(p.c->alloc(&p.w->bdf, n));
    }
    const double* Minv;
    MG_TRY(coarse_inverse(p.c, p.kind, p.alpha, &Minv));
    if (std::find(ctxs.begin(), ctxs.end(), p.c) == ctxs.end()) ctxs.push_back(p.c);
  }
  // the Helmholtz problems of each context that allows it step as a stack
  std::vector<Stack> stacks;
  stacks.reserve(ctxs.size());
  for (mg_ctx* c : ctxs) {
    if (!stack_ok(c)) continue;
    std::vector<Prob*> m;
    for (Prob& p : P)
      if (p.c == c && p.kind == kHelmholtz && (int)m.size() < mg::kMaxStack) m.push_back(&p);
    if (m.size() < 2) continue;
    stacks.emplace_back();
    Stack& S = stacks.back();
    S.c = c;
    S.m = m;
    MG_TRY(get_stack(c, (int)m.size(), &S.w));
    for (size_t q = 0; q < m.size(); ++q) {
      m[q]->stk = &S;
      m[q]->sq = (int)q;
      S.alpha[q] = m[q]->alpha;
    }
  }
  for (mg_ctx* c : ctxs) MG_CUDA(cudaEventRecord(c->fork, c->stream));
  for (Prob& p : P) {
    Work* w = p.w;
    MG_CUDA(cudaStreamWaitEvent(w->s, p.c->fork, 0));
    if (p.st) {
      std::memset(p.st, 0, sizeof(*p.st));
      MG_CUDA(cudaEventRecord(w->t0, w->s));
    }
    MG_TRY(prepare(p, w->s));
    p.cur = w->udf[0];
    p.other = w->udf[1];
    p.ic = p.c->opt.inner_cycles;
    // a zero guess on a grid without electrode cells (a cold start) has
    // residual b: its first pass is pointwise (checked on the device)
    if (!p.c->lv[0].mask) {
      w->norm_host[2] = 0.0;
      Scope sc(p.c, w->s, MG_KCLASS_COARSE, 0);
      mg::launch_nonzero(p.u, p.c->lv[0].b.n(), w->norm_map + 2, w->s);
    }
  }
  for (Prob& p : P) {
    if (!p.c->lv[0].mask) {
      MG_CUDA(cudaStreamSynchronize(p.w->s));
      p.zero_guess = p.w->norm_host[2] == 0.0;
    }
    // ||b|| (slot 0) and the residual of the initial guess (slot 1, r -> FP32)
    MG_TRY(enqueue_first(p));
  }
  size_t left = P.size();
  while (left) {
    bool progress = false;
    for (Prob& p : P) {
      if (p.done || p.waiting) continue;  // a waiting member is its stack's
      const cudaError_t q = cudaEventQuery(p.w->ev);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) return fail(MG_ERR_CUDA, std::string("solve: ") + cudaGetErrorString(q));
      progress = true;
      MG_TRY(advance(p));
      if (p.done) --left;
    }
    for (Stack& S : stacks) {
      if (S.running) {
        const cudaError_t q = cudaEventQuery(S.w->ev);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess)
          return fail(MG_ERR_CUDA, std::string("solve: ") + cudaGetErrorString(q));
        progress = true;
        S.running = false;
        if (S.g) harvest_graph(S.c, *S.g);
        for (Prob* p : S.m) {
          if (!((S.stepping >> p->sq) & 1u)) continue;
          p->waiting = false;
          MG_TRY(advance(*p));
          if (p->done) --left;
        }
      }
      // the next step once every member not yet done waits for it
      unsigned act = 0;
      int ic = 0;
      bool ready = true;
      for (Prob* p : S.m) {
        if (p->done) continue;
        if (!p->waiting) {
          ready = false;
          break;
        }
        act |= 1u << p->sq;
        ic = std::max(ic, p->ic);
      }
      if (ready && act) {
        progress = true;
        MG_TRY(enqueue_stack_step(S, act, ic));
      }
    }
    if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  for (Stack& S : stacks) MG_CUDA(cudaStreamSynchronize(S.w->s));
  mg_status worst = MG_OK;
  for (Prob& p : P) {
    MG_CUDA(cudaStreamSynchronize(p.w->s));
    if (p.st) {
      float ms = 0;
      MG_CUDA(cudaEventElapsedTime(&ms, p.w->t0, p.w->t1));
      p.st->cycles = p.cyc;
      p.st->vcycles = p.vcycles;
      p.st->rel_resid = p.rel;
      p.st->converged = p.rel <= p.tol;
      p.st->diverged = p.diverged;
      p.st->time_ms = ms;
    }
    if (p.status == MG_ERR_NONFINITE || (p.status != MG_OK && worst == MG_OK)) worst = p.status;
  }
  for (mg_ctx* c : ctxs) harvest(c);
  const bool sweep_late = mg::sweep_timed_out(), ir_late = mg::ir_timed_out();
  if (sweep_late || ir_late)
    return fail(MG_ERR_CUDA, sweep_late ? "a staged half-sweep gave up waiting for a plane copy"
                                        : "a staged refinement step gave up waiting for a plane copy");
  if (worst == MG_ERR_NONFINITE) g_last_error = "non-finite value in input or residual";
  return worst;
}

// FP64-mode solve of one problem on its context's stream.
mg_status solve_fp64(Prob& p) {
  mg_ctx* c = p.c;
  Work* w;
  MG_TRY(get_work(c, 0, &w));
  p.w = w;
  cudaStream_t s = c->stream;
  if (p.st) {
    std::memset(p.st, 0, sizeof(*p.st));
    MG_CUDA(cudaEventRecord(w->t0, s));
  }
  MG_TRY(prepare(p, s));
  auto norms = [&](bool with_b) -> mg_status {
    IrIo io;
    io.b64 = p.b;
    io.u64 = p.u;
    io.znorm = with_b;
    MG_TRY(enqueue_ir(c, w, s, p.kind, p.alpha, io, 1));
    MG_CUDA(cudaStreamSynchronize(s));
    harvest(c);
    return MG_OK;
  };
  MG_TRY(norms(true));
  p.bnorm = std::sqrt(w->norm_host[0]);
  if (!std::isfinite(p.bnorm)) return fail(MG_ERR_NONFINITE, "non-finite right-hand side");
  if (p.bnorm == 0.0) p.bnorm = 1.0;
  p.rel = std::sqrt(w->norm_host[1]) / p.bnorm;
  if (p.st) p.st->hist[0] = p.rel;
  p.growth.push(p.rel);
  while (std::isfinite(p.rel) && p.rel > p.tol && p.cyc < c->opt.max_cycles && !p.diverged) {
    MG_TRY(vcycle64(c, p.kind, p.alpha, 0, p.b, p.u));
    MG_TRY(norms(false));
    p.rel = std::sqrt(w->norm_host[1]) / p.bnorm;
    ++p.cyc;
    if (p.st && p.cyc < 64) p.st->hist[p.cyc] = p.rel;
    p.diverged = p.growth.push(p.rel) && p.rel > p.tol;
  }
  if (p.st) {
    MG_CUDA(cudaEventRecord(w->t1, s));
    MG_CUDA(cudaEventSynchronize(w->t1));
    float ms = 0;
    MG_CUDA(cudaEventElapsedTime(&ms, w->t0, w->t1));
    p.st->cycles = p.cyc;
    p.st->vcycles = p.cyc;
    p.st->rel_resid = p.rel;
    p.st->converged = p.rel <= p.tol;
    p.st->diverged = p.diverged;
    p.st->time_ms = ms;
  }
  if (!std::isfinite(p.rel)) return fail(MG_ERR_NONFINITE, "non-finite residual");
  if (p.rel > p.tol) {
    char msg[128];
    std::snprintf(msg, sizeof msg, "%s: rel. residual %.3e after %d cycles",
                  p.diverged ? "diverged" : "not converged", p.rel, p.cyc);
    return fail(p.diverged ? MG_ERR_DIVERGED : MG_ERR_NOT_CONVERGED, msg);
  }
  return MG_OK;
}

bool hard_error(mg_status st) {
  return st == MG_ERR_CUDA || st == MG_ERR_OOM || st == MG_ERR_UNSUPPORTED ||
         st == MG_ERR_INVALID_ARG;
}

constexpr int kMaxConcurrent = 16;  // problems in flight across contexts

mg_status solve(std::vector<Prob>& P) {
  mg_status worst = MG_OK;
  if (P.empty()) return MG_OK;
  if (P[0].c->opt.precision == MG_PREC_MIXED) {
    // waves of at most kMaxConcurrent problems, at most concurrency (<= 4) per context
    size_t q0 = 0;
    while (q0 < P.size()) {
      std::vector<Prob> part;
      std::vector<std::pair<mg_ctx*, int>> per;
      size_t q = q0;
      for (; q < P.size() && (int)part.size() < kMaxConcurrent; ++q) {
        mg_ctx* c = P[q].c;
        auto it = std::find_if(per.begin(), per.end(), [&](auto& e) { return e.first == c; });
        const int cap = std::max(1, std::min(c->opt.concurrency, kMaxWork));
        if (it != per.end() && it->second >= cap) break;
        if (it == per.end()) per.push_back({c, 1});
        else ++it->second;
        part.push_back(P[q]);
      }
      const mg_status st = solve_mixed(part);
      if (hard_error(st)) return st;
      if (st == MG_ERR_NONFINITE || (st != MG_OK && worst == MG_OK)) worst = st;
      q0 = q;
    }
    return worst;
  }
  for (Prob& p : P) {
    const mg_status st = solve_fp64(p);
    if (hard_error(st)) return st;
    if (st == MG_ERR_NONFINITE || (st != MG_OK && worst == MG_OK)) worst = st;
  }
  return worst;
}

void destroy(mg_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (Work* w : c->stacks) c->work.push_back(w);
  c->stacks.clear();
  for (Work* w : c->work) {
    if (w->s) cudaStreamSynchronize(w->s);
    for (StepGraph& g : w->graphs) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      for (const ProfRec& r : g.recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
      }
    }
    if (w->s) cudaStreamDestroy(w->s);
    if (w->ev) cudaEventDestroy(w->ev);
    if (w->t0) cudaEventDestroy(w->t0);
    if (w->t1) cudaEventDestroy(w->t1);
    delete w;
  }
  for (const ProfRec& r : c->pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  for (void* p : c->allocs) cudaFree(p);
  for (void* p : c->host_allocs) cudaFreeHost(p);
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->own_net) mg_unet_destroy(c->net);
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
  const long long nc = c->lv.back().b.n();
  if (nc > kDenseMax)
    return fail(MG_ERR_UNSUPPORTED, "grid does not coarsen to <= 4096 cells (need even sizes)");
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
      if (l == 0) {
        MG_TRY(c->alloc(&L.cxd, n));
        MG_TRY(c->alloc(&L.cyd, n));
        MG_TRY(c->alloc(&L.czd, n));
        MG_TRY(c->alloc(&L.Dd, n));
      }
    }
    for (int col = 0; col < 2; ++col) {
      if (eps_r || mask) MG_TRY(c->alloc(&L.bp[col], (size_t)L.ns, true));
      if (mask) MG_TRY(c->alloc(&L.bh[col], (size_t)L.ns, true));
    }
    if (c->opt.precision == MG_PREC_FP64) {
      if (l > 0) {
        MG_TRY(c->alloc(&L.u64, n));
        MG_TRY(c->alloc(&L.f64, n));
      }
      if (l == nlev - 1) MG_TRY(c->alloc(&L.r64, n));
    }
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
  const bool face_rule = eps_r && c->opt.coarse_op == MG_COARSE_FACE;
  for (int l = 0; l < nlev; ++l) {
    Level& L = c->lv[l];
    double rho[6];
    for (int f = 0; f < 6; ++f) rho[f] = face_rho(c, kPoisson, 0.0, f, L.h);
    if (eps_r && face_rule && l > 0) {
      // coarse operator from the finer level's face weights (levels in order)
      const Level& F = c->lv[l - 1];
      mg::launch_coarsen_faces64(F.cx, F.cy, F.cz, F.b, L.beta64, L.mask, L.b, L.ih2, rho, L.cx,
                                 L.cy, L.cz, L.D, s);
      for (int col = 0; col < 2; ++col) {
        MG_TRY(c->alloc(&L.fx[col], (size_t)L.ns, true));
        MG_TRY(c->alloc(&L.fy[col], (size_t)L.ns, true));
        MG_TRY(c->alloc(&L.fz[col], (size_t)L.ns, true));
        MG_TRY(c->alloc(&L.dg[col], (size_t)L.ns, true));
      }
      mg::launch_split_faces(L.cx, L.cy, L.cz, L.D, L.b, L.W, mp(L.fx), mp(L.fy), mp(L.fz),
                             mp(L.dg), s);
    } else if (eps_r) {
      mg::launch_faces64(L.beta64, L.mask, L.b, L.ih2, rho, L.cx, L.cy, L.cz, L.D, s);
    }
    if (eps_r && l == 0) {
      const double* src[4] = {L.cx, L.cy, L.cz, L.D};
      float2* dst[4] = {L.cxd, L.cyd, L.czd, L.Dd};
      for (int q = 0; q < 4; ++q) mg::launch_split_df(src[q], dst[q], L.b.n(), s);
    }
    if (eps_r || mask) mg::launch_split_beta(L.beta64, L.mask, sop(c, l, kPoisson, 0.0), mp(L.bp), s);
    if (mask) mg::launch_split_beta(nullptr, L.mask, sop(c, l, kHelmholtz, 0.0), mp(L.bh), s);
  }
  // the automatic tile can be shorter than the smallest settable one: room
  // for whichever grid has more CTAs
  c->npartial = std::max(mg::ir_partials(L0.b, 0), mg::ir_partials(L0.b, kIrZchunkMin));
  MG_TRY(c->alloc(&c->gj_row, (size_t)nc));
  MG_TRY(c->alloc(&c->gj_col, (size_t)nc));
  MG_CUDA(cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming));
  MG_TRY(check_launch());
  MG_CUDA(cudaStreamSynchronize(s));
  return MG_OK;
}

mg_status normalise_options(const mg_options* in, mg_options* out) {
  mg_default_options(out);
  if (!in) return MG_OK;
  if (in->nu1 < 0 || in->nu2 < 0 || in->max_cycles < 0 || in->inner_cycles < 0 ||
      in->concurrency < 0)
    return fail(MG_ERR_INVALID_ARG, "negative option");
  if (in->precision != MG_PREC_FP64 && in->precision != MG_PREC_MIXED)
    return fail(MG_ERR_INVALID_ARG, "unknown precision");
  if (in->no_graphs != 0 && in->no_graphs != 1)
    return fail(MG_ERR_INVALID_ARG, "no_graphs must be 0 or 1");
  if (in->rte_bc != MG_RTE_BC_DIRICHLET && in->rte_bc != MG_RTE_BC_MARSHAK)
    return fail(MG_ERR_INVALID_ARG, "rte_bc must be MG_RTE_BC_DIRICHLET or MG_RTE_BC_MARSHAK");
  if (in->ir_zchunk != 0 && in->ir_zchunk < kIrZchunkMin)
    return fail(MG_ERR_INVALID_ARG, "ir_zchunk must be 0 (automatic) or >= 16");
  if (in->coarse_op != MG_COARSE_FACE && in->coarse_op != MG_COARSE_CELL)
    return fail(MG_ERR_INVALID_ARG, "coarse_op must be MG_COARSE_FACE or MG_COARSE_CELL");
  if (in->nu1) out->nu1 = in->nu1;
  if (in->nu2) out->nu2 = in->nu2;
  if (in->max_cycles) out->max_cycles = in->max_cycles;
  if (in->inner_cycles) out->inner_cycles = in->inner_cycles;
  if (in->concurrency) out->concurrency = in->concurrency;
  out->precision = in->precision;
  out->no_graphs = in->no_graphs;
  out->rte_bc = in->rte_bc;
  out->ir_zchunk = in->ir_zchunk;
  out->coarse_op = in->coarse_op;
  if (in->fixed_cycles != 0 && in->fixed_cycles != 1)
    return fail(MG_ERR_INVALID_ARG, "fixed_cycles must be 0 or 1");
  out->fixed_cycles = in->fixed_cycles;
  if (in->coarse_visits < 0 || in->coarse_visits > 2)
    return fail(MG_ERR_INVALID_ARG, "coarse_visits must be 0, 1 or 2");
  out->coarse_visits = in->coarse_visits;
  if (in->sweep_zchunk != 0 && in->sweep_zchunk != -1 && in->sweep_zchunk != 8 &&
      in->sweep_zchunk != 16 && in->sweep_zchunk != 32)
    return fail(MG_ERR_INVALID_ARG, "sweep_zchunk must be 0, -1, 8, 16 or 32");
  out->sweep_zchunk = in->sweep_zchunk;
  if (in->stack != 0 && in->stack != 1) return fail(MG_ERR_INVALID_ARG, "stack must be 0 or 1");
  out->stack = in->stack;
  return MG_OK;
}

mg_status check_ctx_tol(const mg_ctx* c, double tol) {
  if (!c) return fail(MG_ERR_INVALID_ARG, "ctx is NULL");
  if (!(tol >= 0.0)) return fail(MG_ERR_INVALID_ARG, "tol must be >= 0");
  return MG_OK;
}

mg_status check_helmholtz_args(const double* S, double* const psi[3], const double kappa[3]) {
  if (!S || !psi || !kappa) return fail(MG_ERR_INVALID_ARG, "NULL argument");
  for (int j = 0; j < 3; ++j) {
    if (!psi[j]) return fail(MG_ERR_INVALID_ARG, "psi[j] is NULL");
    if (!(kappa[j] > 0.0) || !std::isfinite(kappa[j]))
      return fail(MG_ERR_INVALID_ARG, "kappa must be finite and > 0");
  }
  return MG_OK;
}

}  // namespace

// ---- composite AMR hierarchy ---------------------------------------------
//
// Fast adaptive composite (FAC) iteration on a ratio-2 hierarchy of boxes.
// Every iteration, for each level l from the base upwards: the composite
// residual of all levels >= l (finest first: coarse-fine ghosts, residual
// with refluxing, children's residuals averaged onto covered cells), a
// correction solve on every box of level l (inner V-cycles from zero; the
// base box with its domain faces, a refined box with Robin faces that stand
// in for its coarse-fine ghosts), and the correction added to the box and,
// by trilinear interpolation, to every box refining it.  The residual is
// FP64; corrections are FP32 V-cycles (mixed) or FP64 V-cycles, so the
// iteration converges to the FP64 composite solution either way.

namespace {

// Face factor rho of a refined box's correction operator on its finest
// level: Robin faces n.grad e + a e = 0 with a h / 2 = rho / (1 - rho), i.e.
// the ghost (1 - 2 rho) e = (2/3) e, close to the coarse-fine ghost of a
// smooth correction whose coarse part is zero, (2/3) e_1 - (1/5) e_2.  It
// only affects the convergence rate of the iteration, not its fixed point.
constexpr double kBoxRho = 1.0 / 6.0;
constexpr int kMaxChildren = 254;

struct AmrBox {
  int level = 0, parent = -1;
  int lo[3] = {0, 0, 0}, n[3] = {0, 0, 0};
  int fo[3] = {0, 0, 0};  // footprint lower corner in the parent's cells
  double h = 0.0;
  mg_ctx* ctx = nullptr;
  std::vector<int> children;
  int child0 = 0;
  uint8_t* cov = nullptr;  // 0 valid, k + 1 covered by child k, 255 valid next to a
                           // covered cell (null: no children)
  double* b = nullptr;     // right-hand side with lifts
  double* r = nullptr;     // composite residual
  double* ghost = nullptr; // level >= 1: coarse-fine ghosts, packed per face
  double* delta = nullptr; // level >= 1 with children: increment passed on
  double* e64 = nullptr;   // FP64 mode: correction
  long long poff = 0;      // first partial sum of this box
  unsigned* special = nullptr;  // valid boundary cells and cells next to a covered cell
  unsigned nspecial = 0;
  mg::Box box() const { return mg::Box{n[0], n[1], n[2]}; }
};

}  // namespace

struct mg_amr {
  mg_options opt{};
  cudaStream_t stream = nullptr;
  std::vector<AmrBox> box;  // 0: base box; then the refined boxes in the caller's order
  int nlev = 1;
  mg::AmrDev* dev = nullptr;       // box descriptors on the device
  mg::AmrDev* dev_host = nullptr;  // pinned staging copy
  int* child_list = nullptr;
  double* partial = nullptr;  // [2][npartial]: r^2 and zero-guess r^2 per block
  long long npartial = 0;
  double* norm_host = nullptr;  // [2], pinned, written by the reduction kernel
  double* norm_map = nullptr;   // its device-side address
  cudaEvent_t ev = nullptr, upload = nullptr, t0 = nullptr, t1 = nullptr;
  std::vector<void*> allocs;
  std::vector<void*> host_allocs;

  template <class T>
  mg_status alloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return MG_OK;
    MG_CUDA(cudaMalloc((void**)p, sizeof(T) * count));
    allocs.push_back(*p);
    return MG_OK;
  }
};

namespace {

// double-float (hi, lo) of a host double
float2 df_host(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

void amr_destroy(mg_amr* a) {
  if (!a) return;
  if (a->stream) cudaStreamSynchronize(a->stream);
  for (AmrBox& B : a->box) destroy(B.ctx);
  for (void* p : a->allocs) cudaFree(p);
  for (void* p : a->host_allocs) cudaFreeHost(p);
  for (cudaEvent_t e : {a->ev, a->upload, a->t0, a->t1})
    if (e) cudaEventDestroy(e);
  delete a;
}

bool box_inside(const int lo[3], const int hi[3], const int olo[3], const int ohi[3]) {
  for (int d = 0; d < 3; ++d)
    if (lo[d] < olo[d] || hi[d] > ohi[d]) return false;
  return true;
}

bool box_overlap(const int lo[3], const int hi[3], const int olo[3], const int ohi[3]) {
  for (int d = 0; d < 3; ++d)
    if (lo[d] >= ohi[d] || olo[d] >= hi[d]) return false;
  return true;
}

// Levels, parents, footprints and the nesting rules (host only).
mg_status amr_layout(mg_amr* a, const mg_grid* g, int nbox, const mg_amr_box* boxes) {
  a->box.resize((size_t)nbox + 1);
  if ((long long)g->nx * g->ny * g->nz >= (1ll << 31))
    return fail(MG_ERR_UNSUPPORTED, "base grid with 2^31 cells or more");
  AmrBox& B0 = a->box[0];
  B0.n[0] = g->nx;
  B0.n[1] = g->ny;
  B0.n[2] = g->nz;
  B0.h = g->h;
  for (int q = 1; q <= nbox; ++q) {
    const mg_amr_box& in = boxes[q - 1];
    AmrBox& B = a->box[q];
    if (in.level < 1 || in.level > 20)
      return fail(MG_ERR_INVALID_ARG, "refined box level must be in 1..20");
    B.level = in.level;
    B.h = g->h / (double)(1 << in.level);
    if ((long long)in.n[0] * in.n[1] * in.n[2] >= (1ll << 31))
      return fail(MG_ERR_UNSUPPORTED, "refined box with 2^31 cells or more");
    for (int d = 0; d < 3; ++d) {
      if (in.n[d] < 2 || (in.n[d] & 1) || (in.lo[d] & 1))
        return fail(MG_ERR_INVALID_ARG, "refined box corners and sizes must be even, sizes >= 2");
      B.lo[d] = in.lo[d];
      B.n[d] = in.n[d];
    }
    a->nlev = std::max(a->nlev, B.level + 1);
  }
  for (int q = 1; q <= nbox; ++q) {
    AmrBox& B = a->box[q];
    int flo[3], fhi[3], glo[3], ghi[3];
    // the footprint grown by one parent cell must lie inside the parent, by
    // two when the parent is a refined box (its own ghosts read its two
    // outermost cell layers, which must stay valid)
    const int margin = B.level == 1 ? 1 : 2;
    int mlo[3], mhi[3];
    for (int d = 0; d < 3; ++d) {
      flo[d] = B.lo[d] / 2;
      fhi[d] = (B.lo[d] + B.n[d]) / 2;
      glo[d] = flo[d] - 1;
      ghi[d] = fhi[d] + 1;
      mlo[d] = flo[d] - margin;
      mhi[d] = fhi[d] + margin;
    }
    for (int p = 0; p <= nbox; ++p) {
      const AmrBox& P = a->box[p];
      if (P.level != B.level - 1) continue;
      int phi[3];
      for (int d = 0; d < 3; ++d) phi[d] = P.lo[d] + P.n[d];
      if (!box_inside(mlo, mhi, P.lo, phi)) continue;
      if (B.parent >= 0) return fail(MG_ERR_INVALID_ARG, "refined box inside two parents");
      B.parent = p;
    }
    if (B.parent < 0)
      return fail(MG_ERR_INVALID_ARG,
                  "refined box: footprint grown by one cell (two inside a refined box) not "
                  "inside a box of the level below");
    AmrBox& P = a->box[B.parent];
    for (int d = 0; d < 3; ++d) B.fo[d] = flo[d] - P.lo[d];
    P.children.push_back(q);
    if ((int)P.children.size() > kMaxChildren)
      return fail(MG_ERR_UNSUPPORTED, "more than 254 refined boxes inside one box");
    for (int o = 1; o <= nbox; ++o) {
      const AmrBox& O = a->box[o];
      if (o == q || O.level != B.level) continue;
      int olo[3], ohi[3];
      for (int d = 0; d < 3; ++d) {
        olo[d] = O.lo[d] / 2;
        ohi[d] = (O.lo[d] + O.n[d]) / 2;
      }
      if (box_overlap(glo, ghi, olo, ohi))
        return fail(MG_ERR_INVALID_ARG,
                    "refined boxes of one level must be at least one parent cell apart");
    }
  }
  return MG_OK;
}

// Electrode cells may not lie under, or next to, a refined box.
mg_status amr_check_mask(mg_amr* a, const uint8_t* mask) {
  if (!mask) return MG_OK;
  const AmrBox& B0 = a->box[0];
  const mg::Box b = B0.box();
  std::vector<uint8_t> m((size_t)b.n());
  MG_CUDA(cudaMemcpy(m.data(), mask, m.size(), cudaMemcpyDeviceToHost));
  for (int q : B0.children) {
    const AmrBox& B = a->box[q];
    for (int k = B.fo[2] - 1; k < B.fo[2] + B.n[2] / 2 + 1; ++k)
      for (int j = B.fo[1] - 1; j < B.fo[1] + B.n[1] / 2 + 1; ++j)
        for (int i = B.fo[0] - 1; i < B.fo[0] + B.n[0] / 2 + 1; ++i)
          if (m[((size_t)k * b.ny + j) * b.nx + i])
            return fail(MG_ERR_INVALID_ARG, "electrode cell under or next to a refined box");
  }
  return MG_OK;
}

// Context of a refined box: its own grid and coefficient, Robin faces.
mg_status amr_box_ctx(mg_amr* a, AmrBox& B, const double* eps, const mg_options& o) {
  mg_ctx* c = new (std::nothrow) mg_ctx;
  if (!c) return fail(MG_ERR_OOM, "host allocation failed");
  c->grid.nx = B.n[0];
  c->grid.ny = B.n[1];
  c->grid.nz = B.n[2];
  c->grid.h = B.h;
  for (int f = 0; f < 6; ++f) {
    c->bc.kind[f] = MG_BC_NEUMANN;
    c->bc.value[f] = 0.0;
  }
  c->opt = o;
  c->opt.rte_bc = MG_RTE_BC_DIRICHLET;
  c->stream = a->stream;
  c->robin_a = 2.0 * (kBoxRho / (1.0 - kBoxRho)) / B.h;
  const mg_status st = build(c, eps, nullptr, nullptr);
  if (st != MG_OK) {
    destroy(c);
    return st;
  }
  B.ctx = c;
  return MG_OK;
}

// Device arrays of every box, the child list and the partial sums.
mg_status amr_alloc(mg_amr* a) {
  std::vector<int> clist;
  for (AmrBox& B : a->box) {
    const mg::Box b = B.box();
    const size_t n = (size_t)b.n();
    MG_TRY(a->alloc(&B.b, n));
    MG_TRY(a->alloc(&B.r, n));
    if (B.level > 0) MG_TRY(a->alloc(&B.ghost, (size_t)mg::face_count(b)));
    if (B.level > 0 && !B.children.empty()) MG_TRY(a->alloc(&B.delta, n));
    if (a->opt.precision == MG_PREC_FP64) MG_TRY(a->alloc(&B.e64, n));
    B.child0 = (int)clist.size();
    for (int k : B.children) clist.push_back(k);
    std::vector<uint8_t> cov_host;
    if (!B.children.empty()) {
      std::vector<uint8_t>& cov = cov_host;
      cov.assign(n, 0);
      for (size_t t = 0; t < B.children.size(); ++t) {
        const AmrBox& K = a->box[B.children[t]];
        for (int k = 0; k < K.n[2] / 2; ++k)
          for (int j = 0; j < K.n[1] / 2; ++j)
            for (int i = 0; i < K.n[0] / 2; ++i)
              cov[((size_t)(K.fo[2] + k) * b.ny + K.fo[1] + j) * b.nx + K.fo[0] + i] =
                  (uint8_t)(t + 1);
      }
      // valid cells with a covered face neighbour take the refluxed row
      const long long st[3] = {1, b.nx, (long long)b.nx * b.ny};
      for (int k = 0; k < b.nz; ++k)
        for (int j = 0; j < b.ny; ++j)
          for (int i = 0; i < b.nx; ++i) {
            const size_t c = ((size_t)k * b.ny + j) * b.nx + i;
            if (cov[c]) continue;
            const int x[3] = {i, j, k}, m[3] = {b.nx, b.ny, b.nz};
            for (int d = 0; d < 3; ++d) {
              if (x[d] > 0 && cov[c - st[d]] && cov[c - st[d]] != 255) cov[c] = 255;
              if (x[d] + 1 < m[d] && cov[c + st[d]] && cov[c + st[d]] != 255) cov[c] = 255;
            }
          }
      MG_TRY(a->alloc(&B.cov, n));
      MG_CUDA(cudaMemcpy(B.cov, cov.data(), n, cudaMemcpyHostToDevice));
    }
    // cells that take the general row: valid cells on the box boundary and
    // valid cells next to a covered cell
    {
      std::vector<unsigned> sp;
      for (int k = 0; k < b.nz; ++k)
        for (int j = 0; j < b.ny; ++j)
          for (int i = 0; i < b.nx; ++i) {
            const size_t c = ((size_t)k * b.ny + j) * b.nx + i;
            const uint8_t kc = B.cov ? cov_host[c] : 0;
            const bool edge = i == 0 || j == 0 || k == 0 || i == b.nx - 1 || j == b.ny - 1 ||
                              k == b.nz - 1;
            if (kc == 255 || (kc == 0 && edge)) sp.push_back((unsigned)c);
          }
      B.nspecial = (unsigned)sp.size();
      MG_TRY(a->alloc(&B.special, sp.size()));
      if (!sp.empty())
        MG_CUDA(cudaMemcpy(B.special, sp.data(), sizeof(unsigned) * sp.size(),
                           cudaMemcpyHostToDevice));
    }
    B.poff = a->npartial;
    a->npartial += mg::amr_resid_blocks(b, B.nspecial);
  }
  if (!clist.empty()) {
    MG_TRY(a->alloc(&a->child_list, clist.size()));
    MG_CUDA(cudaMemcpy(a->child_list, clist.data(), sizeof(int) * clist.size(),
                       cudaMemcpyHostToDevice));
  }
  MG_TRY(a->alloc(&a->partial, 2 * (size_t)a->npartial));
  MG_TRY(a->alloc(&a->dev, a->box.size()));
  MG_CUDA(cudaMallocHost((void**)&a->dev_host, sizeof(mg::AmrDev) * a->box.size()));
  a->host_allocs.push_back(a->dev_host);
  MG_CUDA(cudaMallocHost((void**)&a->norm_host, 2 * sizeof(double)));
  a->host_allocs.push_back(a->norm_host);
  MG_CUDA(cudaHostGetDevicePointer((void**)&a->norm_map, a->norm_host, 0));
  MG_CUDA(cudaEventCreateWithFlags(&a->ev, cudaEventDisableTiming));
  MG_CUDA(cudaEventCreateWithFlags(&a->upload, cudaEventDisableTiming));
  MG_CUDA(cudaEventCreate(&a->t0));
  MG_CUDA(cudaEventCreate(&a->t1));
  MG_CUDA(cudaEventRecord(a->upload, a->stream));
  return MG_OK;
}

// Operator kind, alpha and right-hand-side scale of an AMR solve.
mg_status amr_kind(const mg_amr* a, int kind, double param, Kind* k, double* alpha,
                   double* scale) {
  switch (kind) {
    case MG_PROBLEM_POISSON:
      *k = kPoisson;
      *alpha = 0.0;
      *scale = 1.0 / kEps0;
      return MG_OK;
    case MG_PROBLEM_SCREENED:
      if (!(param >= 0.0) || !std::isfinite(param))
        return fail(MG_ERR_INVALID_ARG, "alpha must be finite and >= 0");
      *k = kPoisson;
      *alpha = param;
      *scale = 1.0;
      return MG_OK;
    case MG_PROBLEM_HELMHOLTZ:
      if (!(param > 0.0) || !std::isfinite(param))
        return fail(MG_ERR_INVALID_ARG, "kappa must be finite and > 0");
      if (a->opt.rte_bc != MG_RTE_BC_DIRICHLET)
        return fail(MG_ERR_UNSUPPORTED, "AMR Helmholtz solves support Psi = 0 faces only");
      *k = kHelmholtz;
      *alpha = param * param;
      *scale = 1.0;
      return MG_OK;
    default:
      return fail(MG_ERR_INVALID_ARG, "unknown problem kind");
  }
}

// Box descriptors for this call's iterate (the staging copy is reused once
// the previous upload has left it).
mg_status amr_upload(mg_amr* a, Kind kind, const double* const* u) {
  MG_CUDA(cudaEventSynchronize(a->upload));
  for (size_t q = 0; q < a->box.size(); ++q) {
    const AmrBox& B = a->box[q];
    mg::AmrDev& d = a->dev_host[q];
    d = mg::AmrDev{};
    d.b = B.box();
    for (int e = 0; e < 3; ++e) d.fo[e] = B.fo[e];
    d.parent = B.parent;
    d.child0 = B.child0;
    d.ih2 = 1.0 / (B.h * B.h);
    d.u = u[q];
    d.beta = kind == kPoisson ? B.ctx->lv[0].beta64 : nullptr;
    d.ghost = B.ghost;
    d.cov = B.cov;
  }
  MG_CUDA(cudaMemcpyAsync(a->dev, a->dev_host, sizeof(mg::AmrDev) * a->box.size(),
                          cudaMemcpyHostToDevice, a->stream));
  MG_CUDA(cudaEventRecord(a->upload, a->stream));
  return MG_OK;
}

// b of every box: rhs * scale plus the base box's domain-face lifts.
mg_status amr_rhs(mg_amr* a, Kind kind, double scale, const double* const* rhs) {
  const double zero[6] = {0, 0, 0, 0, 0, 0};
  for (size_t q = 0; q < a->box.size(); ++q) {
    AmrBox& B = a->box[q];
    const Level& L = B.ctx->lv[0];
    uint8_t dir[6] = {0, 0, 0, 0, 0, 0};
    if (q == 0)
      for (int f = 0; f < 6; ++f) dir[f] = kind == kPoisson ? poisson_dir(B.ctx, f) : 1;
    mg::launch_rhs64(rhs[q], scale, kind == kPoisson ? L.beta64 : nullptr, L.mask, L.b, L.ih2,
                     dir, q == 0 && kind == kPoisson ? B.ctx->bc.value : zero, nullptr, B.b,
                     a->stream);
  }
  return check_launch();
}

// Composite residual of every box of level >= lmin, finest level first;
// with norm, ||r||^2 over the valid cells into norm_host[1] (and the
// zero-guess ||b||^2 into norm_host[0] with znorm), asynchronously.  With
// split_base the base box's residual goes straight to the FP32 split
// right-hand side of its correction solve (mixed precision).
mg_status amr_pass(mg_amr* a, Kind kind, double alpha, int lmin, bool norm, bool znorm,
                   bool split_base = false) {
  cudaStream_t s = a->stream;
  LevelWork* X0 = nullptr;
  if (split_base && lmin == 0) {
    Work* w;
    MG_TRY(get_work(a->box[0].ctx, 0, &w));
    X0 = &w->lw[0];
  }
  for (int lev = a->nlev - 1; lev >= lmin; --lev)
    for (size_t q = 0; q < a->box.size(); ++q) {
      AmrBox& B = a->box[q];
      if (B.level != lev) continue;
      const mg::Box b = B.box();
      if (lev > 0) mg::launch_amr_ghost(a->dev, (int)q, b, B.ghost, s);
      const Level& L = B.ctx->lv[0];
      mg::AmrResArgs ra{};
      ra.alpha = alpha;
      if (kind == kPoisson) {
        ra.cx = L.cx;
        ra.cy = L.cy;
        ra.cz = L.cz;
        ra.cxd = L.cxd;
        ra.cyd = L.cyd;
        ra.czd = L.czd;
        ra.Dd = L.Dd;
      }
      ra.ih2d = df_host(L.ih2);
      ra.dint = df_host(6.0 * L.ih2 + alpha);
      ra.nalpha = df_host(-alpha);
      ra.has_alpha = alpha != 0.0;
      ra.mask = L.mask;
      for (int f = 0; f < 6; ++f) ra.rho[f] = q == 0 ? face_rho(B.ctx, kind, alpha, f, B.h) : 0.0;
      ra.b = B.b;
      ra.r = B.r;
      const bool split = q == 0 && X0;
      if (split) {
        ra.f32[0] = X0->f32[0];
        ra.f32[1] = X0->f32[1];
        ra.W = L.W;
      }
      ra.partial = norm ? a->partial + B.poff : nullptr;
      ra.partial_z = znorm ? a->partial + a->npartial + B.poff : nullptr;
      ra.special = B.special;
      ra.nspecial = B.nspecial;
      mg::launch_amr_resid(a->dev, a->child_list, (int)q, b, ra, s);
      for (int k : B.children) {
        const AmrBox& K = a->box[k];
        mg::launch_amr_average(K.box(), K.fo, K.r, b, B.r, split ? X0->f32[0] : nullptr,
                               split ? X0->f32[1] : nullptr, L.W, s);
      }
    }
  if (norm) {
    mg::launch_sum_partials(a->partial, (int)a->npartial, a->norm_map + 1, s);
    if (znorm) mg::launch_sum_partials(a->partial + a->npartial, (int)a->npartial, a->norm_map, s);
  }
  return check_launch();
}

// Correction solve on box q from its residual, added to the box and passed
// on to every box refining it.
mg_status amr_correct(mg_amr* a, Kind kind, double alpha, int q, double* const* u,
                      bool rhs_split) {
  AmrBox& B = a->box[q];
  mg_ctx* c = B.ctx;
  cudaStream_t s = a->stream;
  const Level& L = c->lv[0];
  const float* e0 = nullptr;
  const float* e1 = nullptr;
  const double* e64 = nullptr;
  if (a->opt.precision == MG_PREC_MIXED) {
    Work* w;
    MG_TRY(get_work(c, 0, &w));
    // the coarsest inverse is built on the context's stream: before the fork
    const double* Minv;
    MG_TRY(coarse_inverse(c, kind, alpha, &Minv));
    LevelWork& X = w->lw[0];
    if (!rhs_split) mg::launch_amr_split(L.b, L.W, B.r, X.f32[0], X.f32[1], s);
    MG_CUDA(cudaEventRecord(a->ev, s));
    MG_CUDA(cudaStreamWaitEvent(w->s, a->ev, 0));
    for (int ic = 0; ic < a->opt.inner_cycles; ++ic)
      MG_TRY(vcycle32(c, w, kind, alpha, 0, ic == 0));
    MG_CUDA(cudaEventRecord(w->ev, w->s));
    MG_CUDA(cudaStreamWaitEvent(s, w->ev, 0));
    e0 = X.u32[0];
    e1 = X.u32[1];
  } else {
    MG_CUDA(cudaMemsetAsync(B.e64, 0, sizeof(double) * (size_t)L.b.n(), s));
    for (int ic = 0; ic < a->opt.inner_cycles; ++ic)
      MG_TRY(vcycle64(c, kind, alpha, 0, B.r, B.e64));
    e64 = B.e64;
  }
  mg::launch_amr_add(L.b, L.W, e0, e1, e64, L.mask, u[q], nullptr, s);
  // children from the correction, deeper boxes from their parent's increment
  std::vector<int> todo;
  for (int k : B.children) {
    AmrBox& K = a->box[k];
    mg::launch_amr_prolong(L.b, L.W, e0, e1, e64, K.box(), K.fo, u[k], K.delta, s);
    if (!K.children.empty()) todo.push_back(k);
  }
  for (size_t t = 0; t < todo.size(); ++t) {
    const AmrBox& P = a->box[todo[t]];
    for (int k : P.children) {
      AmrBox& K = a->box[k];
      mg::launch_amr_prolong(P.box(), 0, nullptr, nullptr, P.delta, K.box(), K.fo, u[k], K.delta,
                             s);
      if (!K.children.empty()) todo.push_back(k);
    }
  }
  return check_launch();
}

mg_status check_amr_arrays(const mg_amr* a, const void* const* p) {
  if (!p) return fail(MG_ERR_INVALID_ARG, "NULL argument");
  for (size_t q = 0; q < a->box.size(); ++q)
    if (!p[q]) return fail(MG_ERR_INVALID_ARG, "NULL box array");
  return MG_OK;
}

mg_status amr_solve(mg_amr* a, int kind_in, double param, const double* const* rhs,
                    double* const* u, double tol, mg_stats* st) {
  Kind kind;
  double alpha, scale;
  MG_TRY(amr_kind(a, kind_in, param, &kind, &alpha, &scale));
  MG_TRY(check_amr_arrays(a, (const void* const*)rhs));
  MG_TRY(check_amr_arrays(a, (const void* const*)u));
  if (!(tol >= 0.0)) return fail(MG_ERR_INVALID_ARG, "tol must be >= 0");
  cudaStream_t s = a->stream;
  if (st) {
    std::memset(st, 0, sizeof(*st));
    MG_CUDA(cudaEventRecord(a->t0, s));
  }
  const Level& L0 = a->box[0].ctx->lv[0];
  if (L0.mask)
    mg::launch_set_masked(L0.mask, kind == kPoisson ? a->box[0].ctx->mask_value : nullptr,
                          L0.b.n(), u[0], s);
  MG_TRY(amr_upload(a, kind, u));
  MG_TRY(amr_rhs(a, kind, scale, rhs));
  const bool mixed = a->opt.precision == MG_PREC_MIXED;
  MG_TRY(amr_pass(a, kind, alpha, 0, true, true, mixed));
  MG_CUDA(cudaStreamSynchronize(s));
  double bnorm = std::sqrt(a->norm_host[0]);
  double rel = std::isfinite(bnorm) ? std::sqrt(a->norm_host[1]) / (bnorm > 0.0 ? bnorm : 1.0)
                                    : bnorm;
  if (bnorm == 0.0) bnorm = 1.0;
  if (st) st->hist[0] = rel;
  int cyc = 0;
  mg::Growth growth;
  growth.push(rel);
  bool diverged = false;
  while (std::isfinite(rel) && rel > tol && cyc < a->opt.max_cycles && !diverged) {
    for (int l = 0; l < a->nlev; ++l) {
      if (l > 0) MG_TRY(amr_pass(a, kind, alpha, l, false, false));
      for (size_t q = 0; q < a->box.size(); ++q)
        if (a->box[q].level == l)
          MG_TRY(amr_correct(a, kind, alpha, (int)q, u, q == 0 && mixed));
    }
    MG_TRY(amr_pass(a, kind, alpha, 0, true, false, mixed));
    MG_CUDA(cudaStreamSynchronize(s));
    rel = std::sqrt(a->norm_host[1]) / bnorm;
    ++cyc;
    if (st && cyc < 64) st->hist[cyc] = rel;
    diverged = growth.push(rel) && rel > tol;
  }
  // covered cells: the mean of their children, finest level first
  for (int lev = a->nlev - 1; lev >= 1; --lev)
    for (size_t q = 0; q < a->box.size(); ++q) {
      const AmrBox& B = a->box[q];
      if (B.level != lev) continue;
      mg::launch_amr_average(B.box(), B.fo, u[q], a->box[B.parent].box(), u[B.parent], nullptr,
                             nullptr, 0, s);
    }
  MG_TRY(check_launch());
  if (mixed && mg::sweep_timed_out())
    return fail(MG_ERR_CUDA, "a staged half-sweep gave up waiting for a plane copy");
  if (st) {
    MG_CUDA(cudaEventRecord(a->t1, s));
    MG_CUDA(cudaEventSynchronize(a->t1));
    float ms = 0.0f;
    MG_CUDA(cudaEventElapsedTime(&ms, a->t0, a->t1));
    st->cycles = cyc;
    st->vcycles = cyc * a->opt.inner_cycles;  // per box of every level
    st->rel_resid = rel;
    st->converged = rel <= tol;
    st->diverged = diverged;
    st->time_ms = ms;
  }
  if (!std::isfinite(rel)) return fail(MG_ERR_NONFINITE, "non-finite value in input or residual");
  if (rel > tol) {
    char msg[128];
    std::snprintf(msg, sizeof msg, "%s: rel. residual %.3e after %d iterations",
                  diverged ? "diverged" : "not converged", rel, cyc);
    return fail(diverged ? MG_ERR_DIVERGED : MG_ERR_NOT_CONVERGED, msg);
  }
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
  opt->concurrency = 4;
  opt->no_graphs = 0;
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
  mg::sweep_kernels_ready();
  mg::ir_tma_ready();
  *out = c;
  return MG_OK;
}

mg_status mg_solve_poisson(mg_ctx* c, const double* rho, double* phi, double tol,
                           mg_stats* stats) {
  g_last_error.clear();
  MG_TRY(check_ctx_tol(c, tol));
  if (!rho || !phi) return fail(MG_ERR_INVALID_ARG, "NULL argument");
  std::vector<Prob> P;
  P.push_back(make_prob(c, kPoisson, 0.0, rho, nullptr, phi, tol, stats));
  return solve(P);
}

mg_status mg_efield(mg_ctx* c, const double* phi, const double* J, double* E, double* dt) {
  g_last_error.clear();
  if (!c || !phi) return fail(MG_ERR_INVALID_ARG, "NULL ctx or phi");
  if (dt && !J) return fail(MG_ERR_INVALID_ARG, "dt needs J");
  const Level& L0 = c->lv[0];
  if (L0.b.ny > 65535 || L0.b.nz > 65535)
    return fail(MG_ERR_UNSUPPORTED, "mg_efield needs ny, nz <= 65535");
  if (!c->efield_min) {
    MG_TRY(c->alloc(&c->efield_min, 1));
    MG_TRY(c->alloc(&c->efield_dt, 1));
  }
  uint8_t dir[6];
  for (int f = 0; f < 6; ++f) dir[f] = poisson_dir(c, f);
  mg::launch_efield(phi, L0.mask, L0.b, L0.h, dir, c->bc.value, J, E, kEps0, c->efield_min,
                    dt ? c->efield_dt : nullptr, c->stream);
  MG_TRY(check_launch());
  if (dt) {
    MG_CUDA(cudaMemcpyAsync(dt, c->efield_dt, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    MG_CUDA(cudaStreamSynchronize(c->stream));
  }
  return MG_OK;
}

mg_status mg_solve_screened(mg_ctx* c, double alpha, const double* f, double* u, double tol,
                            mg_stats* stats) {
  g_last_error.clear();
  MG_TRY(check_ctx_tol(c, tol));
  if (!f || !u) return fail(MG_ERR_INVALID_ARG, "NULL argument");
  if (!(alpha >= 0.0) || !std::isfinite(alpha))
    return fail(MG_ERR_INVALID_ARG, "alpha must be finite and >= 0");
  std::vector<Prob> P;
  P.push_back(make_prob(c, kPoisson, alpha, f, nullptr, u, tol, stats, 1.0));
  return solve(P);
}

mg_status mg_solve_helmholtz_batch(mg_ctx* c, const double* S, double* const psi[3],
                                   const double kappa[3], double tol, mg_stats stats[3]) {
  g_last_error.clear();
  MG_TRY(check_ctx_tol(c, tol));
  MG_TRY(check_helmholtz_args(S, psi, kappa));
  std::vector<Prob> P;
  for (int j = 0; j < 3; ++j)
    P.push_back(make_prob(c, kHelmholtz, kappa[j] * kappa[j], S, nullptr, psi[j], tol,
                          stats ? &stats[j] : nullptr));
  return solve(P);
}

mg_status mg_solve_photoionization(mg_ctx* c, const double* S, double* const psi[3],
                                   const double kappa[3], const double amp[3], double tol,
                                   mg_stats stats[3]) {
  g_last_error.clear();
  MG_TRY(check_ctx_tol(c, tol));
  MG_TRY(check_helmholtz_args(S, psi, kappa));
  if (!amp) return fail(MG_ERR_INVALID_ARG, "NULL amplitudes");
  for (int j = 0; j < 3; ++j)
    if (!std::isfinite(amp[j])) return fail(MG_ERR_INVALID_ARG, "amplitudes must be finite");
  std::vector<Prob> P;
  for (int j = 0; j < 3; ++j) {
    P.push_back(make_prob(c, kHelmholtz, kappa[j] * kappa[j], S, nullptr, psi[j], tol,
                          stats ? &stats[j] : nullptr));
    P.back().rhs_scale = amp[j];
  }
  return solve(P);
}

mg_status mg_solve_set(mg_ctx* c, const double* rho, double* phi, const double* S,
                       double* const psi[3], const double kappa[3], double tol,
                       mg_stats stats[4]) {
  g_last_error.clear();
  MG_TRY(check_ctx_tol(c, tol));
  if (!rho || !phi) return fail(MG_ERR_INVALID_ARG, "NULL argument");
  MG_TRY(check_helmholtz_args(S, psi, kappa));
  std::vector<Prob> P;
  P.push_back(make_prob(c, kPoisson, 0.0, rho, nullptr, phi, tol, stats ? &stats[0] : nullptr));
  for (int j = 0; j < 3; ++j)
    P.push_back(make_prob(c, kHelmholtz, kappa[j] * kappa[j], S, nullptr, psi[j], tol,
                          stats ? &stats[1 + j] : nullptr));
  return solve(P);
}

mg_status mg_solve_batch(const mg_problem* probs, int nprob, double tol, mg_stats* stats) {
  g_last_error.clear();
  if (nprob < 0 || (nprob > 0 && !probs)) return fail(MG_ERR_INVALID_ARG, "bad problem list");
  if (!(tol >= 0.0)) return fail(MG_ERR_INVALID_ARG, "tol must be >= 0");
  std::vector<Prob> P;
  for (int q = 0; q < nprob; ++q) {
    const mg_problem& pr = probs[q];
    if (!pr.ctx || !pr.rhs || !pr.u) return fail(MG_ERR_INVALID_ARG, "NULL ctx, rhs or u");
    if (pr.ctx->opt.precision != probs[0].ctx->opt.precision)
      return fail(MG_ERR_INVALID_ARG, "all contexts of a batch need the same precision mode");
    for (int o = 0; o < q; ++o)
      if (probs[o].u == pr.u) return fail(MG_ERR_INVALID_ARG, "two problems share one u array");
    if (pr.kind == MG_PROBLEM_POISSON) {
      P.push_back(make_prob(pr.ctx, kPoisson, 0.0, pr.rhs, pr.faces, pr.u, tol,
                            stats ? &stats[q] : nullptr));
    } else if (pr.kind == MG_PROBLEM_HELMHOLTZ) {
      if (!(pr.kappa > 0.0) || !std::isfinite(pr.kappa))
        return fail(MG_ERR_INVALID_ARG, "kappa must be finite and > 0");
      if (pr.faces && pr.ctx->opt.rte_bc == MG_RTE_BC_MARSHAK)
        return fail(MG_ERR_INVALID_ARG, "face data needs Dirichlet faces (rte_bc is Marshak)");
      P.push_back(make_prob(pr.ctx, kHelmholtz, pr.kappa * pr.kappa, pr.rhs, pr.faces, pr.u, tol,
                            stats ? &stats[q] : nullptr));
    } else if (pr.kind == MG_PROBLEM_SCREENED) {
      if (!(pr.alpha >= 0.0) || !std::isfinite(pr.alpha))
        return fail(MG_ERR_INVALID_ARG, "alpha must be finite and >= 0");
      P.push_back(make_prob(pr.ctx, kPoisson, pr.alpha, pr.rhs, pr.faces, pr.u, tol,
                            stats ? &stats[q] : nullptr, 1.0));
    } else {
      return fail(MG_ERR_INVALID_ARG, "unknown problem kind");
    }
  }
  return solve(P);
}

mg_status mg_subbox_bc(const mg_ctx* parent, const double* parent_u, const int origin[3],
                       const int dims[3], double* faces) {
  g_last_error.clear();
  if (!parent || !parent_u || !origin || !dims || !faces)
    return fail(MG_ERR_INVALID_ARG, "NULL argument");
  const mg::Box pb = parent->lv[0].b;
  const int pn[3] = {pb.nx, pb.ny, pb.nz};
  for (int a = 0; a < 3; ++a) {
    if (dims[a] < 2 || dims[a] % 2) return fail(MG_ERR_INVALID_ARG, "sub-box sizes must be even, >= 2");
    // the interpolation stencil needs one parent cell outside each face
    if (origin[a] < 1 || origin[a] + dims[a] / 2 > pn[a] - 1)
      return fail(MG_ERR_INVALID_ARG, "sub-box must lie at least one parent cell inside the parent");
  }
  mg::launch_subbox_bc(parent_u, pb, origin[0], origin[1], origin[2],
                       mg::Box{dims[0], dims[1], dims[2]}, faces, parent->stream);
  MG_TRY(check_launch());
  return MG_OK;
}

long long mg_face_count(int nx, int ny, int nz) {
  if (nx < 1 || ny < 1 || nz < 1) return 0;
  return mg::face_count(mg::Box{nx, ny, nz});
}

mg_status mg_set_options(mg_ctx* c, const mg_options* opt) {
  g_last_error.clear();
  if (!c || !opt) return fail(MG_ERR_INVALID_ARG, "NULL argument");
  mg_options o;
  MG_TRY(normalise_options(opt, &o));
  if (o.precision != c->opt.precision)
    return fail(MG_ERR_INVALID_ARG, "the precision mode is fixed at mg_create");
  if (o.rte_bc != c->opt.rte_bc)
    return fail(MG_ERR_INVALID_ARG, "rte_bc is fixed at mg_create");
  if (o.coarse_op != c->opt.coarse_op)
    return fail(MG_ERR_INVALID_ARG, "coarse_op is fixed at mg_create");
  c->opt = o;
  return MG_OK;
}

mg_status mg_autotune(mg_ctx* c, const double* rho, const double* S, const double kappa[3],
                      double tol, mg_options* best, double* best_ms) {
  g_last_error.clear();
  MG_TRY(check_ctx_tol(c, tol));
  if (!rho || !S || !kappa || !best) return fail(MG_ERR_INVALID_ARG, "NULL argument");
  const size_t n = (size_t)c->lv[0].b.n();
  double* scratch = nullptr;
  MG_CUDA(cudaMalloc((void**)&scratch, 4 * n * sizeof(double)));
  double* phi = scratch;
  double* psi[3] = {scratch + n, scratch + 2 * n, scratch + 3 * n};
  const mg_options keep = c->opt;
  const int sweeps[4][2] = {{1, 1}, {2, 1}, {2, 2}, {3, 3}};
  const int inner_mixed[4] = {1, 2, 3, 4};
  const int n_inner = c->opt.precision == MG_PREC_MIXED ? 4 : 1;
  double best_t = 1e300;
  mg_options best_o = keep;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  mg_status st = MG_OK;
  if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess)
    st = fail(MG_ERR_CUDA, "cudaEventCreate failed");
  // device time of one candidate: the faster of two runs from zero (the
  // first builds its graphs); false if it does not reach tol
  auto time_opts = [&](const mg_options& o, double* t_out) -> bool {
    c->opt = o;
    double t_min = 1e300;
    for (int rep = 0; rep < 2 && st == MG_OK; ++rep) {
      if (cudaMemsetAsync(scratch, 0, 4 * n * sizeof(double), c->stream) != cudaSuccess ||
          cudaEventRecord(t0, c->stream) != cudaSuccess) {
        st = fail(MG_ERR_CUDA, "autotune launch failed");
        break;
      }
      const mg_status sv = mg_solve_set(c, rho, phi, S, psi, kappa, tol, nullptr);
      cudaEventRecord(t1, c->stream);
      cudaEventSynchronize(t1);
      float ms = 0;
      cudaEventElapsedTime(&ms, t0, t1);
      if (sv == MG_ERR_NOT_CONVERGED || sv == MG_ERR_DIVERGED) return false;  // rejected
      if (sv != MG_OK) {
        st = sv;
        break;
      }
      t_min = std::min(t_min, (double)ms);
    }
    *t_out = t_min;
    return st == MG_OK;
  };
  auto consider = [&](const mg_options& o) {
    double t;
    if (time_opts(o, &t) && t < best_t) {
      best_t = t;
      best_o = o;
    }
  };
  for (int a = 0; a < 4 && st == MG_OK; ++a)
    for (int b = 0; b < n_inner && st == MG_OK; ++b) {
      mg_options o = keep;
      o.nu1 = sweeps[a][0];
      o.nu2 = sweeps[a][1];
      o.inner_cycles = c->opt.precision == MG_PREC_MIXED ? inner_mixed[b] : 1;
      consider(o);
    }
  // then, for the best candidate (mixed mode), the tile of the refinement
  // pass and the z planes per CTA of the staged half-sweep
  if (st == MG_OK && best_t < 1e300 && keep.precision == MG_PREC_MIXED) {
    const int zcs[4] = {16, 32, 64, 128};
    const mg_options base = best_o;
    for (int z = 0; z < 4 && st == MG_OK; ++z) {
      if (zcs[z] >= c->lv[0].b.nz) continue;
      mg_options o = base;
      o.ir_zchunk = zcs[z];
      consider(o);
    }
    const int szs[2] = {16, 32};
    const mg_options base2 = best_o;
    for (int z = 0; z < 2 && st == MG_OK; ++z) {
      if (base2.sweep_zchunk == szs[z]) continue;
      mg_options o = base2;
      o.sweep_zchunk = szs[z];
      consider(o);
    }
  }
  c->opt = st == MG_OK ? best_o : keep;
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaStreamSynchronize(c->stream);
  cudaFree(scratch);
  if (st != MG_OK) return st;
  if (best_t >= 1e300) return fail(MG_ERR_NOT_CONVERGED, "no candidate converged");
  *best = best_o;
  if (best_ms) *best_ms = best_t;
  return MG_OK;
}

mg_status mg_warmstart_attach(mg_ctx* c, mg_unet* net) {
  if (!c) return fail(MG_ERR_INVALID_ARG, "ctx is NULL");
  if (c->own_net) mg_unet_destroy(c->net);
  c->net = net;
  c->own_net = false;
  return MG_OK;
}

mg_status mg_warmstart_load(mg_ctx* c, const char* path) {
  if (!c || !path) return fail(MG_ERR_INVALID_ARG, "NULL argument");
  mg_unet* net = nullptr;
  MG_TRY(mg_unet_create(0, &net));
  const mg_status st = mg_unet_load(net, path);
  if (st != MG_OK) {
    mg_unet_destroy(net);
    return st;
  }
  if (c->own_net) mg_unet_destroy(c->net);
  c->net = net;
  c->own_net = true;
  return MG_OK;
}

// r = b - A phi in FP64 (natural layout) for the Poisson problem of rho, via
// work slot 0 (b formed there); electrode cells of phi are set first.
mg_status poisson_residual(mg_ctx* c, const double* rho, double* phi, double* r, Prob* pout) {
  cudaStream_t s = c->stream;
  Prob p = make_prob(c, kPoisson, 0.0, rho, nullptr, phi, 0.0, nullptr);
  MG_TRY(get_work(c, 0, &p.w));
  MG_TRY(prepare(p, s));
  if (r) {
    Scope sc(c, s, MG_KCLASS_COARSE, 0);
    mg::launch_resid64(op64(c, 0, kPoisson, 0.0), 0.0, p.b, phi, r, s);
  }
  MG_TRY(check_launch());
  if (pout) *pout = p;
  return MG_OK;
}

mg_status mg_poisson_residual(mg_ctx* c, const double* rho, double* phi, double* r) {
  g_last_error.clear();
  if (!c || !rho || !phi || !r) return fail(MG_ERR_INVALID_ARG, "NULL argument");
  return poisson_residual(c, rho, phi, r, nullptr);
}

mg_status mg_residual_norms(mg_ctx* c, int kind, double param, const double* rhs,
                            const double* u, double norms[2]) {
  g_last_error.clear();
  if (!c || !rhs || !u || !norms) return fail(MG_ERR_INVALID_ARG, "NULL argument");
  Kind k = kPoisson;
  double alpha = 0.0, scale = 1.0 / kEps0;
  if (kind == MG_PROBLEM_HELMHOLTZ) {
    if (!(param > 0.0) || !std::isfinite(param))
      return fail(MG_ERR_INVALID_ARG, "kappa must be finite and > 0");
    k = kHelmholtz;
    alpha = param * param;
    scale = 1.0;
  } else if (kind == MG_PROBLEM_SCREENED) {
    if (!(param >= 0.0) || !std::isfinite(param))
      return fail(MG_ERR_INVALID_ARG, "alpha must be finite and >= 0");
    alpha = param;
    scale = 1.0;
  } else if (kind != MG_PROBLEM_POISSON) {
    return fail(MG_ERR_INVALID_ARG, "unknown problem kind");
  }
  cudaStream_t s = c->stream;
  Work* w;
  MG_TRY(get_work(c, 0, &w));
  const Level& L0 = c->lv[0];
  if (!w->b64) MG_TRY(c->alloc(&w->b64, (size_t)L0.b.n()));
  MG_TRY(form_b(c, k, scale, rhs, nullptr, w->b64, s));
  const int nblk = mg::resid_norms_blocks(L0.b, c->npartial);
  {
    Scope sc(c, s, MG_KCLASS_COARSE, 0);
    mg::launch_resid_norms64(op64(c, 0, k, alpha), alpha, w->b64, u, w->partial, nblk, s);
    mg::launch_sum_partials(w->partial, nblk, w->norm_map + 1, s);
    mg::launch_sum_partials(w->partial + nblk, nblk, w->norm_map, s);
  }
  MG_TRY(check_launch());
  MG_CUDA(cudaStreamSynchronize(s));
  norms[0] = std::sqrt(w->norm_host[1]);
  norms[1] = std::sqrt(w->norm_host[0]);
  return MG_OK;
}

mg_status mg_warmstart_predict(mg_ctx* c, const double* rho, const double* phi_prev,
                               double* phi_guess, int* used_net) {
  g_last_error.clear();
  if (!c || !rho || !phi_prev || !phi_guess) return fail(MG_ERR_INVALID_ARG, "NULL argument");
  if (!c->net) return fail(MG_ERR_INVALID_ARG, "no warm-start network attached");
  const mg::Box b = c->lv[0].b;
  cudaStream_t s = c->stream;
  // the network sees the residual of the previous potential, r = A (phi_n - phi_prev)
  MG_CUDA(cudaMemcpyAsync(phi_guess, phi_prev, sizeof(double) * b.n(), cudaMemcpyDeviceToDevice, s));
  Prob p;
  MG_TRY(get_work(c, 0, &p.w));
  if (!p.w->phi_tmp) MG_TRY(c->alloc(&p.w->phi_tmp, (size_t)b.n()));
  double* r = p.w->phi_tmp;
  MG_TRY(poisson_residual(c, rho, phi_guess, r, &p));
  MG_TRY(mg_unet_predict(c->net, r, phi_guess, phi_guess, 1, b.nz, b.ny, b.nx, s));
  // plain multigrid judges the guess: both candidates get the same nu1 FP64
  // red-black Gauss-Seidel sweeps (the network's BF16 noise is high-frequency
  // and would otherwise dominate its residual), then their FP64 residuals
  // are compared; the better smoothed candidate is the guess
  double* prev_s = r;  // the network input is no longer needed
  MG_CUDA(cudaMemcpyAsync(prev_s, phi_prev, sizeof(double) * b.n(), cudaMemcpyDeviceToDevice, s));
  const mg::Op64 op = op64(c, 0, kPoisson, 0.0);
  for (double* u : {phi_guess, prev_s})
    for (int q = 0; q < c->opt.nu1; ++q)
      for (int col = 0; col < 2; ++col) {
        Scope sc(c, s, MG_KCLASS_COARSE, 0);
        mg::launch_rbgs64(op, 0.0, p.b, u, col, s);
      }
  IrIo io;
  io.b64 = p.b;
  io.u64 = phi_guess;
  MG_TRY(enqueue_ir(c, p.w, s, kPoisson, 0.0, io, 0));
  io.u64 = prev_s;
  MG_TRY(enqueue_ir(c, p.w, s, kPoisson, 0.0, io, 1));
  MG_CUDA(cudaStreamSynchronize(s));
  const double r_net = p.w->norm_host[0], r_prev = p.w->norm_host[1];
  const bool use = std::isfinite(r_net) && r_net <= r_prev;
  if (!use)
    MG_CUDA(cudaMemcpyAsync(phi_guess, prev_s, sizeof(double) * b.n(), cudaMemcpyDeviceToDevice, s));
  MG_CUDA(cudaStreamSynchronize(s));
  if (used_net) *used_net = use ? 1 : 0;
  return MG_OK;
}

mg_status mg_profile_enable(mg_ctx* c, int enable) {
  if (!c) return fail(MG_ERR_INVALID_ARG, "ctx is NULL");
  MG_CUDA(cudaStreamSynchronize(c->stream));
  for (Work* w : c->work) MG_CUDA(cudaStreamSynchronize(w->s));
  harvest(c);
  c->prof = enable != 0;
  std::memset(c->acc, 0, sizeof(c->acc));
  return MG_OK;
}

mg_status mg_profile_read(mg_ctx* c, mg_kprof* out, int reset) {
  if (!c || !out) return fail(MG_ERR_INVALID_ARG, "NULL argument");
  MG_CUDA(cudaStreamSynchronize(c->stream));
  for (Work* w : c->work) MG_CUDA(cudaStreamSynchronize(w->s));
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
    case MG_ERR_DIVERGED: return "diverged: the residual grew over three cycles";
  }
  return "unknown status";
}

mg_status mg_amr_create(const mg_grid* base, int nbox, const mg_amr_box* boxes,
                        const double* const* eps_r, const uint8_t* mask, const double* mask_value,
                        const mg_bc* bc, const mg_options* opt, void* cuda_stream, mg_amr** out) {
  g_last_error.clear();
  if (!out) return fail(MG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!base || !bc) return fail(MG_ERR_INVALID_ARG, "base grid or bc is NULL");
  if (nbox < 0 || (nbox > 0 && !boxes)) return fail(MG_ERR_INVALID_ARG, "bad box list");
  if (base->nx < 1 || base->ny < 1 || base->nz < 1 || !(base->h > 0.0) || !std::isfinite(base->h))
    return fail(MG_ERR_INVALID_ARG, "grid sizes must be >= 1 and h > 0");
  mg_options o;
  MG_TRY(normalise_options(opt, &o));
  mg_amr* a = new (std::nothrow) mg_amr;
  if (!a) return fail(MG_ERR_OOM, "host allocation failed");
  a->opt = o;
  a->stream = (cudaStream_t)cuda_stream;
  mg_status st = amr_layout(a, base, nbox, boxes);
  if (st == MG_OK) st = amr_check_mask(a, mask);
  if (st == MG_OK)
    st = mg_create(base, eps_r ? eps_r[0] : nullptr, mask, mask_value, bc, &o, cuda_stream,
                   &a->box[0].ctx);
  for (int q = 1; st == MG_OK && q <= nbox; ++q)
    st = amr_box_ctx(a, a->box[q], eps_r ? eps_r[q] : nullptr, o);
  if (st == MG_OK) st = amr_alloc(a);
  if (st != MG_OK) {
    const std::string msg = g_last_error;
    amr_destroy(a);
    g_last_error = msg;
    return st;
  }
  *out = a;
  return MG_OK;
}

mg_status mg_amr_solve(mg_amr* amr, int kind, double param, const double* const* rhs,
                       double* const* u, double tol, mg_stats* stats) {
  g_last_error.clear();
  if (!amr) return fail(MG_ERR_INVALID_ARG, "amr is NULL");
  return amr_solve(amr, kind, param, rhs, u, tol, stats);
}

mg_status mg_amr_residual(mg_amr* amr, int kind, double param, const double* const* rhs,
                          const double* const* u, double* const* r, double* norm) {
  g_last_error.clear();
  if (!amr) return fail(MG_ERR_INVALID_ARG, "amr is NULL");
  Kind k;
  double alpha, scale;
  MG_TRY(amr_kind(amr, kind, param, &k, &alpha, &scale));
  MG_TRY(check_amr_arrays(amr, (const void* const*)rhs));
  MG_TRY(check_amr_arrays(amr, (const void* const*)u));
  MG_TRY(check_amr_arrays(amr, (const void* const*)r));
  MG_TRY(amr_upload(amr, k, u));
  MG_TRY(amr_rhs(amr, k, scale, rhs));
  MG_TRY(amr_pass(amr, k, alpha, 0, true, false));
  for (size_t q = 0; q < amr->box.size(); ++q)
    MG_CUDA(cudaMemcpyAsync(r[q], amr->box[q].r, sizeof(double) * (size_t)amr->box[q].box().n(),
                            cudaMemcpyDeviceToDevice, amr->stream));
  if (norm) {
    MG_CUDA(cudaStreamSynchronize(amr->stream));
    *norm = std::sqrt(amr->norm_host[1]);
  }
  return MG_OK;
}

void mg_amr_destroy(mg_amr* amr) { amr_destroy(amr); }

const char* mg_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
