// Electric field and dielectric relaxation time after a Poisson solve.
//
// The paper's scheme (Sec. 1; the coarse step of Sec. 3) advances the
// elliptic updates on the time scale Delta t_E = eps0 |E| / |J|, the
// relaxation time that a first-order truncation of Ampere's law gives.  This
// pass forms E = -grad phi at cell centres and the minimum of eps0 |E| / |J|
// over the free cells in one read of phi and J.
//
// E: centred differences (phi(c - 1) - phi(c + 1)) / (2h) per axis, with the
// ghost value of the domain face outside the box (Dirichlet value g: 2g -
// phi_c, Neumann: phi_c) and the electrode value at the centre of a masked
// neighbour (the same values the operator of Eq. 2 uses).  Electrode cells
// get E = 0.  E is FP64 (one FP64 add and multiply per component, the same
// arithmetic as the definition); the ratio that only selects a time step is
// formed in FP32 from E and J narrowed on the integer pipe, which keeps the
// FP64 pipe of GB300 (about 1/57 of the FP32 rate) at six operations per cell.
#include <cfloat>

#include "df.cuh"
#include "mg_internal.h"

namespace mg {

namespace {

constexpr int kT = 256;

// FP32 minimum of a block (every thread passes its value).
__device__ __forceinline__ float block_min(float v) {
  __shared__ float w[kT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < kT / 32 ? w[threadIdx.x] : FLT_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;
}

// One thread per cell along x (grid-stride over rows): blockIdx covers (x
// blocks, rows); the per-block minimum goes to partial[block].
__global__ void __launch_bounds__(kT) k_efield(const double* __restrict__ phi,
                                               const uint8_t* __restrict__ mask, Box b,
                                               double inv2h, Dir6 dir, Val6 g,
                                               const double* __restrict__ J,
                                               double* __restrict__ E, float eps0,
                                               float* __restrict__ partial) {
  using namespace df;
  const long long n = b.n();
  const long long sy = b.nx, sz = (long long)b.nx * b.ny;
  const long long rows = (long long)b.ny * b.nz;
  float best = FLT_MAX;
  for (long long row = blockIdx.y; row < rows; row += gridDim.y) {
    const int j = (int)(row % b.ny), k = (int)(row / b.ny);
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i >= b.nx) continue;
    const long long c = row * b.nx + i;
    const bool m = mask && mask[c];
    const double pc = phi[c];
    // neighbour value or the face ghost
    auto nb = [&](bool inside, long long q, int f) {
      if (inside) return phi[q];
      return dir.d[f] ? 2.0 * g.v[f] - pc : pc;
    };
    double ex = 0.0, ey = 0.0, ez = 0.0;
    if (!m) {
      ex = (nb(i > 0, c - 1, 0) - nb(i < b.nx - 1, c + 1, 1)) * inv2h;
      ey = (nb(j > 0, c - sy, 2) - nb(j < b.ny - 1, c + sy, 3)) * inv2h;
      ez = (nb(k > 0, c - sz, 4) - nb(k < b.nz - 1, c + sz, 5)) * inv2h;
    }
    if (E) {
      E[c] = ex;
      E[n + c] = ey;
      E[2 * n + c] = ez;
    }
    if (J && !m) {
      const float jx = narrow(J[c]), jy = narrow(J[n + c]), jz = narrow(J[2 * n + c]);
      const float fx = narrow(ex), fy = narrow(ey), fz = narrow(ez);
      const float j2 = fmaf(jx, jx, fmaf(jy, jy, jz * jz));
      const float e2 = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
      if (j2 > 0.0f) best = fminf(best, eps0 * sqrtf(e2) * rsqrtf(j2));
    }
  }
  best = block_min(best);
  if (threadIdx.x == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = best;
}

__global__ void k_min_partials(const float* __restrict__ partial, int n, double* out) {
  float v = FLT_MAX;
  for (int t = threadIdx.x; t < n; t += kT) v = fminf(v, partial[t]);
  v = block_min(v);
  if (threadIdx.x == 0) *out = v == FLT_MAX ? __longlong_as_double(0x7ff0000000000000ll) : (double)v;
}

}  // namespace

int efield_partials(const Box& b) {
  const int gx = (b.nx + kT - 1) / kT;
  const long long rows = (long long)b.ny * b.nz;
  const long long gy = rows < 4096 ? rows : 4096;
  return (int)(gx * gy);
}

void launch_efield(const double* phi, const uint8_t* mask, Box b, double h, const uint8_t dir[6],
                   const double gval[6], const double* J, double* E, double eps0, float* partial,
                   double* dt_out, cudaStream_t s) {
  const int gx = (b.nx + kT - 1) / kT;
  const long long rows = (long long)b.ny * b.nz;
  const int gy = (int)(rows < 4096 ? rows : 4096);
  Dir6 d;
  Val6 g;
  for (int f = 0; f < 6; ++f) {
    d.d[f] = dir[f];
    g.v[f] = gval[f];
  }
  k_efield<<<dim3(gx, gy), kT, 0, s>>>(phi, mask, b, 0.5 / h, d, g, J, E, (float)eps0, partial);
  add_launches(1);
  if (J && dt_out) {
    k_min_partials<<<1, kT, 0, s>>>(partial, gx * gy, dt_out);
    add_launches(1);
  }
}

}  // namespace mg
