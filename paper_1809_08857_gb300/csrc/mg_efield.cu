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

// FP32 minimum of a block (every thread passes its value; the result is
// valid in thread 0).
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

// One thread per cell: blockIdx = (x block, j, k).  The block minimum of the
// ratio (a non-negative FP32 number, whose bit pattern orders like an
// unsigned integer) goes to *min_bits by atomicMin.
__global__ void __launch_bounds__(kT) k_efield(const double* __restrict__ phi,
                                               const uint8_t* __restrict__ mask, Box b,
                                               double inv2h, Dir6 dir, Val6 g,
                                               const double* __restrict__ J,
                                               double* __restrict__ E, float eps0,
                                               unsigned* __restrict__ min_bits) {
  using namespace df;
  const long long n = b.n();
  const long long sy = b.nx, sz = (long long)b.nx * b.ny;
  const int i = blockIdx.x * kT + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  float best = FLT_MAX;
  if (i < b.nx) {
    const long long c = ((long long)k * b.ny + j) * b.nx + i;
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
  if (!J) return;  // whole grid
  best = block_min(best);
  if (threadIdx.x == 0 && best < FLT_MAX) atomicMin(min_bits, __float_as_uint(best));
}

__global__ void k_min_init(unsigned* min_bits) { *min_bits = __float_as_uint(FLT_MAX); }

__global__ void k_min_final(const unsigned* min_bits, double* out) {
  const float v = __uint_as_float(*min_bits);
  *out = v == FLT_MAX ? __longlong_as_double(0x7ff0000000000000ll) : (double)v;
}

}  // namespace

void launch_efield(const double* phi, const uint8_t* mask, Box b, double h, const uint8_t dir[6],
                   const double gval[6], const double* J, double* E, double eps0,
                   unsigned* min_bits, double* dt_out, cudaStream_t s) {
  Dir6 d;
  Val6 g;
  for (int f = 0; f < 6; ++f) {
    d.d[f] = dir[f];
    g.v[f] = gval[f];
  }
  if (J) {
    k_min_init<<<1, 1, 0, s>>>(min_bits);
    add_launches(1);
  }
  const dim3 grid((b.nx + kT - 1) / kT, b.ny, b.nz);
  k_efield<<<grid, kT, 0, s>>>(phi, mask, b, 0.5 / h, d, g, J, E, (float)eps0, min_bits);
  add_launches(1);
  if (J && dt_out) {
    k_min_final<<<1, 1, 0, s>>>(min_bits, dt_out);
    add_launches(1);
  }
}

}  // namespace mg
