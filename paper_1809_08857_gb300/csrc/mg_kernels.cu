// Device kernels of libmg: operator setup, red-black Gauss-Seidel smoothing,
// fused residual + restriction, trilinear prolongation + correction,
// coarsest-grid dense solve and the FP64 iterative-refinement residual.
//
// Discretisation: Sec. 2 items (ii)-(iii) of arXiv:1809.08857 (second-order
// cell-centred finite volumes for Eqs. 2 and 3); smoother: red-black
// Gauss-Seidel (Sec. 2 item (ii)).
#include <algorithm>

#include "mg_internal.h"

namespace mg {

namespace {

constexpr int kThreads = 256;

__host__ __device__ inline long long cidx(const Box& b, int i, int j, int k) {
  return ((long long)k * b.ny + j) * b.nx + i;
}

inline unsigned blocks_for(long long n, int threads = kThreads) {
  return (unsigned)((n + threads - 1) / threads);
}

// ---- FP64 operator rows ---------------------------------------------------

__device__ __forceinline__ bool masked(const Op64& op, long long c) {
  if (op.D) return op.D[c] < 0.0;
  return op.mask != nullptr && op.mask[c] != 0;
}

// (A u)_c = diag * u_c - off, diag without alpha.  `ld(n)` returns the value
// of in-box neighbour n.
template <class Load>
__device__ __forceinline__ void row(const Op64& op, int i, int j, int k, long long c, Load ld,
                                    double& diag, double& off) {
  const int nx = op.b.nx, ny = op.b.ny, nz = op.b.nz;
  const long long sy = nx, sz = (long long)nx * ny;
  if (op.cx) {
    double o = 0.0;
    if (i > 0) o += op.cx[c] * ld(c - 1);
    if (i < nx - 1) o += op.cx[c + 1] * ld(c + 1);
    if (j > 0) o += op.cy[c] * ld(c - sy);
    if (j < ny - 1) o += op.cy[c + sy] * ld(c + sy);
    if (k > 0) o += op.cz[c] * ld(c - sz);
    if (k < nz - 1) o += op.cz[c + sz] * ld(c + sz);
    diag = op.D[c];
    off = o;
  } else {
    double o = 0.0, d = 0.0;
    if (i > 0) { d += 1.0; o += ld(c - 1); } else d += 2.0 * op.rho[0];
    if (i < nx - 1) { d += 1.0; o += ld(c + 1); } else d += 2.0 * op.rho[1];
    if (j > 0) { d += 1.0; o += ld(c - sy); } else d += 2.0 * op.rho[2];
    if (j < ny - 1) { d += 1.0; o += ld(c + sy); } else d += 2.0 * op.rho[3];
    if (k > 0) { d += 1.0; o += ld(c - sz); } else d += 2.0 * op.rho[4];
    if (k < nz - 1) { d += 1.0; o += ld(c + sz); } else d += 2.0 * op.rho[5];
    diag = d * op.ih2;
    off = o * op.ih2;
  }
}

template <class T>
__device__ __forceinline__ T divide(T a, T b) { return a / b; }

// ---- setup kernels --------------------------------------------------------

__device__ __forceinline__ double hmean(double a, double b) { return 2.0 * a * b / (a + b); }

// weight of the face between c and its in-box neighbour n (unscaled)
__device__ __forceinline__ double face_w(const double* beta, const uint8_t* mask, long long c,
                                         long long n) {
  const bool mc = mask && mask[c], mn = mask && mask[n];
  const double bc = beta ? beta[c] : 1.0, bn = beta ? beta[n] : 1.0;
  if (!mc && !mn) return hmean(bc, bn);
  if (!mc) return bc;
  if (!mn) return bn;
  return 0.0;
}

__global__ void k_faces64(const double* beta, const uint8_t* mask, Box b, double ih2,
                          Val6 rho, double* cx, double* cy, double* cz, double* D) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= b.n()) return;
  const int i = (int)(c % b.nx);
  const long long jk = c / b.nx;
  const int j = (int)(jk % b.ny), k = (int)(jk / b.ny);
  const long long sy = b.nx, sz = (long long)b.nx * b.ny;
  const bool mc = mask && mask[c];
  const double bc = beta ? beta[c] : 1.0;
  const double wb = mc ? 0.0 : 2.0 * bc;  // domain face, times its factor rho
  double wxm = i > 0 ? face_w(beta, mask, c, c - 1) : wb * rho.v[0];
  double wym = j > 0 ? face_w(beta, mask, c, c - sy) : wb * rho.v[2];
  double wzm = k > 0 ? face_w(beta, mask, c, c - sz) : wb * rho.v[4];
  double wxp = i < b.nx - 1 ? face_w(beta, mask, c, c + 1) : wb * rho.v[1];
  double wyp = j < b.ny - 1 ? face_w(beta, mask, c, c + sy) : wb * rho.v[3];
  double wzp = k < b.nz - 1 ? face_w(beta, mask, c, c + sz) : wb * rho.v[5];
  cx[c] = wxm * ih2;
  cy[c] = wym * ih2;
  cz[c] = wzm * ih2;
  D[c] = mc ? -1.0
            : wxm * ih2 + wxp * ih2 + wym * ih2 + wyp * ih2 + wzm * ih2 + wzp * ih2;
}

// ---- face-based coarse operator ------------------------------------------
//
// Weight of the coarse face between C - e_a and C along axis a (C_a >= 1),
// from the fine level's face weights w (cx, cy or cz: w[c] is the face between
// c and c - e_a, already divided by h_f^2): on each of the 4 fine lines that
// cross the coarse face (the transverse children), the path between the two
// coarse centres passes half of fine cell 2C_a - 1, the fine face 2C_a and
// half of fine cell 2C_a, i.e. the fine faces 2C_a - 1, 2C_a, 2C_a + 1 in
// series with weights 1/4, 1/2, 1/4 (a zero weight, a face between two
// electrode cells, blocks the line); the lines conduct in parallel (their
// mean); the factor 1/4 takes 1/h_f^2 to 1/h_c^2.  For a coefficient that
// is constant on the 4 x 3 cells involved this is the fine rule itself.
__device__ double coarse_face_series(const double* __restrict__ w, const Box& fb, int axis,
                                     int I, int J, int K) {
  double sum = 0.0;
  for (int q = 0; q < 4; ++q) {
    int i = 2 * I, j = 2 * J, k = 2 * K;
    long long st;
    if (axis == 0) { j += q & 1; k += q >> 1; st = 1; }
    else if (axis == 1) { i += q & 1; k += q >> 1; st = fb.nx; }
    else { i += q & 1; j += q >> 1; st = (long long)fb.nx * fb.ny; }
    const long long c = cidx(fb, i, j, k);  // fine cell 2C_a on this line
    const double w1 = w[c - st], w2 = w[c], w3 = w[c + st];
    if (w1 > 0.0 && w2 > 0.0 && w3 > 0.0) sum += 1.0 / (0.25 / w1 + 0.5 / w2 + 0.25 / w3);
  }
  return 0.25 * 0.25 * sum;
}

// Coarse face weights and diagonal (the layout of k_faces64) by the face rule
// above between free coarse cells; a face towards a coarse electrode cell and
// a domain face follow the cell rule of k_faces64 on the coarse cell
// coefficient bc (the mean of the free children, k_coarsen) and mask mc.
__global__ void k_coarsen_faces64(const double* __restrict__ fcx, const double* __restrict__ fcy,
                                  const double* __restrict__ fcz, Box fb,
                                  const double* __restrict__ bc, const uint8_t* __restrict__ mc,
                                  Box cb, double ih2c, Val6 rho, double* cx, double* cy,
                                  double* cz, double* D) {
  const long long C = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (C >= cb.n()) return;
  const int I = (int)(C % cb.nx);
  const long long JK = C / cb.nx;
  const int J = (int)(JK % cb.ny), K = (int)(JK / cb.ny);
  const long long sy = cb.nx, sz = (long long)cb.nx * cb.ny;
  const bool m = mc && mc[C];
  const double wb = m ? 0.0 : 2.0 * (bc ? bc[C] : 1.0);
  // face towards the in-box coarse neighbour N, whose face with C is face
  // (axis, A) in the numbering of coarse_face_series
  auto face = [&](long long N, int axis, int A, int B, int Cc) {
    if (m || (mc && mc[N])) return face_w(bc, mc, C, N) * ih2c;
    return coarse_face_series(axis == 0 ? fcx : (axis == 1 ? fcy : fcz), fb, axis, A, B, Cc);
  };
  const double wxm = I > 0 ? face(C - 1, 0, I, J, K) : wb * rho.v[0] * ih2c;
  const double wxp = I < cb.nx - 1 ? face(C + 1, 0, I + 1, J, K) : wb * rho.v[1] * ih2c;
  const double wym = J > 0 ? face(C - sy, 1, I, J, K) : wb * rho.v[2] * ih2c;
  const double wyp = J < cb.ny - 1 ? face(C + sy, 1, I, J + 1, K) : wb * rho.v[3] * ih2c;
  const double wzm = K > 0 ? face(C - sz, 2, I, J, K) : wb * rho.v[4] * ih2c;
  const double wzp = K < cb.nz - 1 ? face(C + sz, 2, I, J, K + 1) : wb * rho.v[5] * ih2c;
  cx[C] = wxm;
  cy[C] = wym;
  cz[C] = wzm;
  D[C] = m ? -1.0 : wxm + wxp + wym + wyp + wzm + wzp;
}

__global__ void k_split_df(const double* __restrict__ in, float2* __restrict__ out, long long n) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const double v = in[c];
  const float hi = __double2float_rn(v);
  out[c] = make_float2(hi, __double2float_rn(v - (double)hi));
}

// A coarse cell is an electrode cell when at least this many of its 8
// children are.  With "all 8" a thin electrode (a needle tip a few cells
// wide) vanishes from the coarse levels, the coarse operators lose its
// Dirichlet coupling and their corrections overshoot next to it: the
// mixed-precision cycle diverged on the needle-plane gap at 768^3 and above.
// 3 of 8 converged best among 1, 2, 3, 4 and 8 (0.16-0.22 per refinement step
// with one inner V-cycle at 192^3 and 896^3).  The rule shapes only the coarse
// operators, not the answer.
constexpr int kCoarseElectrodeChildren = 3;

// coarse electrode rule as above; beta = mean of the free children
__global__ void k_coarsen(const double* bf, const uint8_t* mf, Box fb, double* bcoarse,
                          uint8_t* mcoarse) {
  Box cb{fb.nx / 2, fb.ny / 2, fb.nz / 2};
  long long C = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (C >= cb.n()) return;
  const int I = (int)(C % cb.nx);
  const long long JK = C / cb.nx;
  const int J = (int)(JK % cb.ny), K = (int)(JK / cb.ny);
  double s = 0.0;
  int nfree = 0;
  for (int q = 0; q < 8; ++q) {
    long long n = cidx(fb, 2 * I + (q & 1), 2 * J + ((q >> 1) & 1), 2 * K + (q >> 2));
    if (mf && mf[n]) continue;
    s += bf ? bf[n] : 1.0;
    ++nfree;
  }
  if (mcoarse) mcoarse[C] = 8 - nfree >= kCoarseElectrodeChildren;
  if (bcoarse) bcoarse[C] = nfree ? s / nfree : 1.0;
}

// Dense matrix of the homogeneous coarsest-level operator (plus alpha) over
// all cells; electrode rows/columns are the identity.  M must be zeroed.
__global__ void k_assemble_dense(Op64 op, double alpha, double* M) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = op.b.n();
  if (c >= n) return;
  if (masked(op, c)) { M[c * n + c] = 1.0; return; }
  const int i = (int)(c % op.b.nx);
  const long long jk = c / op.b.nx;
  const int j = (int)(jk % op.b.ny), k = (int)(jk / op.b.ny);
  // off-diagonal weight of neighbour m = coefficient of u_m in `off`
  auto put = [&](long long m) {
    double diag, off;
    row(op, i, j, k, c, [&](long long q) { return q == m ? 1.0 : 0.0; }, diag, off);
    if (!masked(op, m)) M[c * n + m] = -off;
  };
  const long long sy = op.b.nx, sz = (long long)op.b.nx * op.b.ny;
  if (i > 0) put(c - 1);
  if (i < op.b.nx - 1) put(c + 1);
  if (j > 0) put(c - sy);
  if (j < op.b.ny - 1) put(c + sy);
  if (k > 0) put(c - sz);
  if (k < op.b.nz - 1) put(c + sz);
  double diag, off;
  row(op, i, j, k, c, [](long long) { return 0.0; }, diag, off);
  M[c * n + c] = diag + alpha;
}

// In-place Gauss-Jordan inversion, pivot p: (1) save the pivot row scaled by
// 1/a and the pivot column; (2) eliminate.  No pivoting (the matrix is SPD).
__global__ void k_gj_save(const double* M, int n, int p, double* rowp, double* colp) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double a = M[(size_t)p * n + p];
  rowp[t] = t == p ? 1.0 / a : M[(size_t)p * n + t] / a;
  colp[t] = M[(size_t)t * n + p];
}

__global__ void k_gj_elim(double* M, int n, int p, const double* rowp, const double* colp) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  if (i == p) {
    M[t] = rowp[j];
  } else if (j == p) {
    M[t] = -colp[i] * rowp[p];
  } else {
    M[t] -= colp[i] * rowp[j];
  }
}

// ---- solve kernels --------------------------------------------------------

// b = f * scale + Dirichlet lifts 2 beta_c g / h^2, with g = bval[face] or,
// when faces != nullptr, the packed per-face-cell values.
// One row (j = blockIdx.y, k = blockIdx.z) per grid row, x across threads:
// no 64-bit index division per cell.
__global__ void k_rhs64(const double* f, double scale, const double* beta, const uint8_t* mask,
                        Box b, double ih2, Dir6 dir, Val6 bval, const double* faces,
                        double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, k = blockIdx.z;
  if (i >= b.nx) return;
  const long long c = cidx(b, i, j, k);
  if (mask && mask[c]) { out[c] = 0.0; return; }
  double v = f[c] * scale;
  const double bc = beta ? beta[c] : 1.0;
  auto g = [&](int face) -> double {
    if (!faces) return bval.v[face];
    long long q;
    if (face < 2) q = (long long)k * b.ny + j;
    else if (face < 4) q = (long long)k * b.nx + i;
    else q = (long long)j * b.nx + i;
    return faces[face_offset(b, face) + q];
  };
  if (i == 0 && dir.d[0]) v += 2.0 * bc * ih2 * g(0);
  if (i == b.nx - 1 && dir.d[1]) v += 2.0 * bc * ih2 * g(1);
  if (j == 0 && dir.d[2]) v += 2.0 * bc * ih2 * g(2);
  if (j == b.ny - 1 && dir.d[3]) v += 2.0 * bc * ih2 * g(3);
  if (k == 0 && dir.d[4]) v += 2.0 * bc * ih2 * g(4);
  if (k == b.nz - 1 && dir.d[5]) v += 2.0 * bc * ih2 * g(5);
  out[c] = v;
}

// Dirichlet data of a refined sub-box (ratio 2) from the parent solution:
// trilinear interpolation of the parent's cell-centred values at the fine
// face centres of the sub-box boundary.  The sub-box covers parent cells
// [o, o + n/2) per axis; one thread per face point.
__global__ void k_subbox_bc(const double* __restrict__ pu, Box pb, int ox, int oy, int oz,
                            Box sb, double* faces) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = face_offset(sb, 5) + (long long)sb.nx * sb.ny;
  if (t >= total) return;
  int f = 0;
  while (f < 5 && t >= face_offset(sb, f + 1)) ++f;
  const long long q = t - face_offset(sb, f);
  // parent-grid coordinates (in parent cells, cell centres at integers + 1/2)
  // of the face point; fine cell (i,j,k) centre = o + (i + 1/2)/2
  double px, py, pz;
  if (f < 2) {
    const int j = (int)(q % sb.ny), k = (int)(q / sb.ny);
    px = ox + (f == 0 ? 0.0 : 0.5 * sb.nx);
    py = oy + 0.5 * (j + 0.5);
    pz = oz + 0.5 * (k + 0.5);
  } else if (f < 4) {
    const int i = (int)(q % sb.nx), k = (int)(q / sb.nx);
    px = ox + 0.5 * (i + 0.5);
    py = oy + (f == 2 ? 0.0 : 0.5 * sb.ny);
    pz = oz + 0.5 * (k + 0.5);
  } else {
    const int i = (int)(q % sb.nx), j = (int)(q / sb.nx);
    px = ox + 0.5 * (i + 0.5);
    py = oy + 0.5 * (j + 0.5);
    pz = oz + (f == 4 ? 0.0 : 0.5 * sb.nz);
  }
  // lower parent cell index and weight along each axis
  const double sx = px - 0.5, sy = py - 0.5, sz = pz - 0.5;
  const int I = (int)floor(sx), J = (int)floor(sy), K = (int)floor(sz);
  const double wx = sx - I, wy = sy - J, wz = sz - K;
  double v = 0.0;
  for (int c = 0; c < 8; ++c) {
    const int a = c & 1, bb = (c >> 1) & 1, cc = c >> 2;
    const double w = (a ? wx : 1.0 - wx) * (bb ? wy : 1.0 - wy) * (cc ? wz : 1.0 - wz);
    v += w * pu[cidx(pb, I + a, J + bb, K + cc)];
  }
  faces[t] = v;
}

__global__ void k_set_masked(const uint8_t* mask, const double* value, long long n, double* u) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  if (mask[c]) u[c] = value ? value[c] : 0.0;
}

template <class Op, class T>
__global__ void k_rbgs(Op op, T alpha, const T* __restrict__ f, T* u, int color) {
  const int nx = op.b.nx, ny = op.b.ny, nz = op.b.nz;
  const int nxh = (nx + 1) >> 1;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nxh * ny * nz) return;
  const int ti = (int)(t % nxh);
  const long long jk = t / nxh;
  const int j = (int)(jk % ny), k = (int)(jk / ny);
  const int i = 2 * ti + ((j + k + color) & 1);
  if (i >= nx) return;
  const long long c = cidx(op.b, i, j, k);
  if (masked(op, c)) return;
  T diag, off;
  row(op, i, j, k, c, [&](long long q) { return u[q]; }, diag, off);
  u[c] = divide<T>(f[c] + off, diag + alpha);
}

template <class Op, class T>
__global__ void k_resid_restrict(Op op, T alpha, const T* __restrict__ f,
                                 const T* __restrict__ u, T* fc, T* uc) {
  Box cb{op.b.nx / 2, op.b.ny / 2, op.b.nz / 2};
  long long C = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (C >= cb.n()) return;
  const int I = (int)(C % cb.nx);
  const long long JK = C / cb.nx;
  const int J = (int)(JK % cb.ny), K = (int)(JK / cb.ny);
  T s = 0;
  for (int q = 0; q < 8; ++q) {
    const int i = 2 * I + (q & 1), j = 2 * J + ((q >> 1) & 1), k = 2 * K + (q >> 2);
    const long long c = cidx(op.b, i, j, k);
    if (masked(op, c)) continue;
    T diag, off;
    row(op, i, j, k, c, [&](long long n) { return u[n]; }, diag, off);
    s += f[c] - ((diag + alpha) * u[c] - off);
  }
  fc[C] = s * (T)0.125;
  if (uc) uc[C] = 0;
}

template <class Op, class T>
__global__ void k_resid(Op op, T alpha, const T* __restrict__ f, const T* __restrict__ u, T* r) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= op.b.n()) return;
  const int i = (int)(c % op.b.nx);
  const long long jk = c / op.b.nx;
  const int j = (int)(jk % op.b.ny), k = (int)(jk / op.b.ny);
  if (masked(op, c)) { r[c] = 0; return; }
  T diag, off;
  row(op, i, j, k, c, [&](long long n) { return u[n]; }, diag, off);
  r[c] = f[c] - ((diag + alpha) * u[c] - off);
}

// coarse value with the homogeneous face ghost (1 - 2 rho) across domain
// faces (rho of the coarse level)
template <class T>
__device__ __forceinline__ T cval(const T* ec, const Box& cb, const double* rho, int I, int J,
                                  int K) {
  T s = 1;
  if (I < 0) { I = 0; s *= (T)(1.0 - 2.0 * rho[0]); }
  if (I >= cb.nx) { I = cb.nx - 1; s *= (T)(1.0 - 2.0 * rho[1]); }
  if (J < 0) { J = 0; s *= (T)(1.0 - 2.0 * rho[2]); }
  if (J >= cb.ny) { J = cb.ny - 1; s *= (T)(1.0 - 2.0 * rho[3]); }
  if (K < 0) { K = 0; s *= (T)(1.0 - 2.0 * rho[4]); }
  if (K >= cb.nz) { K = cb.nz - 1; s *= (T)(1.0 - 2.0 * rho[5]); }
  return s * ec[cidx(cb, I, J, K)];
}

template <class Op, class T>
__global__ void k_prolong(Op op, Op cop, const T* __restrict__ ec, T* uf) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= op.b.n()) return;
  if (masked(op, c)) return;
  const int i = (int)(c % op.b.nx);
  const long long jk = c / op.b.nx;
  const int j = (int)(jk % op.b.ny), k = (int)(jk / op.b.ny);
  Box cb{op.b.nx / 2, op.b.ny / 2, op.b.nz / 2};
  const int I = i >> 1, J = j >> 1, K = k >> 1;
  const int si = (i & 1) ? 1 : -1, sj = (j & 1) ? 1 : -1, sk = (k & 1) ? 1 : -1;
  T v = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int a = q & 1, bb = (q >> 1) & 1, cc = q >> 2;
    const T w = (a ? (T)0.25 : (T)0.75) * (bb ? (T)0.25 : (T)0.75) * (cc ? (T)0.25 : (T)0.75);
    v += w * cval(ec, cb, cop.rho, I + a * si, J + bb * sj, K + cc * sk);
  }
  uf[c] += v;
}

// u += Minv r, one warp per row
template <class T>
__global__ void k_dense_apply(const double* __restrict__ Minv, int n, const T* __restrict__ r,
                              T* u) {
  const int warp = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  double s = 0.0;
  for (int col = lane; col < n; col += 32) s += Minv[(size_t)warp * n + col] * (double)r[col];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) u[warp] += (T)s;
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) ws[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = lane < kThreads / 32 ? ws[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

// FP64 norms of a field's residual, plain FP64 arithmetic on the natural
// layout (independent of the double-float refinement pass): per block, the
// sum over free cells of (f - A u)^2 into part[block] and of the residual of
// the guess that is 0 on free cells and u on electrode cells (the norm of b
// with the electrode lifts) into part[nblk + block].  Grid-stride.
__global__ void k_resid_norms64(Op64 op, double alpha, const double* __restrict__ f,
                                const double* __restrict__ u, double* part, int nblk) {
  const long long n = op.b.n();
  double s = 0.0, sb = 0.0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    if (masked(op, c)) continue;
    const int i = (int)(c % op.b.nx);
    const long long jk = c / op.b.nx;
    const int j = (int)(jk % op.b.ny), k = (int)(jk / op.b.ny);
    double diag, off, offb;
    row(op, i, j, k, c, [&](long long q) { return u[q]; }, diag, off);
    row(op, i, j, k, c, [&](long long q) { return masked(op, q) ? u[q] : 0.0; }, diag, offb);
    const double r = f[c] - ((diag + alpha) * u[c] - off);
    const double rb = f[c] + offb;
    s += r * r;
    sb += rb * rb;
  }
  s = block_sum(s);
  __syncthreads();  // block_sum's shared scratch is reused
  sb = block_sum(sb);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s;
    part[nblk + blockIdx.x] = sb;
  }
}

__global__ void k_sum_partials(const double* partial, int n, double* out) {
  double s = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) s += partial[t];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

}  // namespace

// ---- launch wrappers ------------------------------------------------------

namespace {
long long g_launches = 0;
}
long long launch_count() { return g_launches; }
void add_launches(long long k) { g_launches += k; }

static Dir6 to_dir(const uint8_t d[6]) {
  Dir6 r;
  for (int q = 0; q < 6; ++q) r.d[q] = d[q];
  return r;
}

void launch_faces64(const double* beta, const uint8_t* mask, Box b, double ih2,
                    const double rho[6], double* cx, double* cy, double* cz, double* D,
                    cudaStream_t s) {
  Val6 r;
  for (int f = 0; f < 6; ++f) r.v[f] = rho[f];
  k_faces64<<<blocks_for(b.n()), kThreads, 0, s>>>(beta, mask, b, ih2, r, cx, cy, cz, D);
  add_launches(1);
}

void launch_coarsen_faces64(const double* fcx, const double* fcy, const double* fcz, Box fb,
                            const double* beta_c, const uint8_t* mask_c, Box cb, double ih2c,
                            const double rho[6], double* cx, double* cy, double* cz, double* D,
                            cudaStream_t s) {
  Val6 r;
  for (int f = 0; f < 6; ++f) r.v[f] = rho[f];
  k_coarsen_faces64<<<blocks_for(cb.n()), kThreads, 0, s>>>(fcx, fcy, fcz, fb, beta_c, mask_c, cb,
                                                             ih2c, r, cx, cy, cz, D);
  add_launches(1);
}

void launch_split_df(const double* in, float2* out, long long n, cudaStream_t s) {
  k_split_df<<<blocks_for(n), kThreads, 0, s>>>(in, out, n);
  add_launches(1);
}

void launch_coarsen(const double* beta_f, const uint8_t* mask_f, Box fb, double* beta_c,
                    uint8_t* mask_c, cudaStream_t s) {
  Box cb{fb.nx / 2, fb.ny / 2, fb.nz / 2};
  k_coarsen<<<blocks_for(cb.n()), kThreads, 0, s>>>(beta_f, mask_f, fb, beta_c, mask_c);
  add_launches(1);
}

void launch_assemble_dense(Op64 op, double alpha, double* M, cudaStream_t s) {
  const long long n = op.b.n();
  cudaMemsetAsync(M, 0, sizeof(double) * n * n, s);
  k_assemble_dense<<<blocks_for(n), kThreads, 0, s>>>(op, alpha, M);
  add_launches(1);
}

void launch_gj_invert(double* M, int n, double* rowp, double* colp, cudaStream_t s) {
  for (int p = 0; p < n; ++p) {
    k_gj_save<<<blocks_for(n), kThreads, 0, s>>>(M, n, p, rowp, colp);
    add_launches(1);
    k_gj_elim<<<blocks_for((long long)n * n), kThreads, 0, s>>>(M, n, p, rowp, colp);
    add_launches(1);
  }
}

void launch_rhs64(const double* f, double scale, const double* beta, const uint8_t* mask,
                  Box b, double ih2, const uint8_t dir[6], const double bval[6],
                  const double* faces, double* out, cudaStream_t s) {
  Val6 v;
  for (int q = 0; q < 6; ++q) v.v[q] = bval[q];
  dim3 g(blocks_for(b.nx), b.ny, b.nz);
  k_rhs64<<<g, kThreads, 0, s>>>(f, scale, beta, mask, b, ih2, to_dir(dir), v, faces, out);
  add_launches(1);
}

void launch_subbox_bc(const double* parent_u, Box pb, int ox, int oy, int oz, Box sb,
                      double* faces, cudaStream_t s) {
  k_subbox_bc<<<blocks_for(face_count(sb)), kThreads, 0, s>>>(parent_u, pb, ox, oy, oz, sb,
                                                               faces);
  add_launches(1);
}

void launch_set_masked(const uint8_t* mask, const double* value, long long n, double* u,
                       cudaStream_t s) {
  k_set_masked<<<blocks_for(n), kThreads, 0, s>>>(mask, value, n, u);
  add_launches(1);
}

void launch_rbgs64(const Op64& op, double alpha, const double* f, double* u, int color,
                   cudaStream_t s) {
  const long long t = (long long)((op.b.nx + 1) / 2) * op.b.ny * op.b.nz;
  k_rbgs<Op64, double><<<blocks_for(t), kThreads, 0, s>>>(op, alpha, f, u, color);
  add_launches(1);
}

void launch_resid_restrict64(const Op64& op, double alpha, const double* f, const double* u,
                             double* fc, double* uc, cudaStream_t s) {
  Box cb{op.b.nx / 2, op.b.ny / 2, op.b.nz / 2};
  k_resid_restrict<Op64, double><<<blocks_for(cb.n()), kThreads, 0, s>>>(op, alpha, f, u, fc, uc);
  add_launches(1);
}

void launch_prolong64(const Op64& fop, const Op64& cop, const double* ec, double* uf,
                      cudaStream_t s) {
  k_prolong<Op64, double><<<blocks_for(fop.b.n()), kThreads, 0, s>>>(fop, cop, ec, uf);
  add_launches(1);
}

void launch_resid64(const Op64& op, double alpha, const double* f, const double* u, double* r,
                    cudaStream_t s) {
  k_resid<Op64, double><<<blocks_for(op.b.n()), kThreads, 0, s>>>(op, alpha, f, u, r);
  add_launches(1);
}

void launch_dense_apply64(const double* Minv, int n, const double* r, double* u,
                          cudaStream_t s) {
  k_dense_apply<double><<<blocks_for((long long)n * 32), kThreads, 0, s>>>(Minv, n, r, u);
  add_launches(1);
}

int resid_norms_blocks(const Box& b, int cap) {
  const long long want = (b.n() + kThreads - 1) / kThreads;
  return (int)std::max(1LL, std::min<long long>(want, std::min(cap, 152 * 8)));
}

void launch_resid_norms64(const Op64& op, double alpha, const double* f, const double* u,
                          double* part, int nblk, cudaStream_t s) {
  k_resid_norms64<<<nblk, kThreads, 0, s>>>(op, alpha, f, u, part, nblk);
  add_launches(1);
}

void launch_sum_partials(const double* partial, int n, double* out, cudaStream_t s) {
  k_sum_partials<<<1, kThreads, 0, s>>>(partial, n, out);
  add_launches(1);
}

}  // namespace mg
