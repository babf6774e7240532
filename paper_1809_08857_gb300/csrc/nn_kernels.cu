// Kernels of the learned warm start: a 3D U-Net on BF16 activations with
// FP32 accumulation (the network maps (rho_n, phi_{n-1}) to phi_n - phi_{n-1},
// motivated by the infrequent elliptic re-solves of Sec. 2.2).
//
// Layout: activations channels-last [N][D][H][W][C] in BF16, C a multiple of
// 16; 3x3x3 conv weights [Cout][27][Cin] (tap t = (kd*3 + kh)*3 + kw) in
// BF16 with an FP32 master copy.
//
// conv3d forward is an implicit GEMM on the tensor cores (mma.sync
// m16n8k16 bf16 -> fp32): M = output voxels, N = Cout, K = 27 Cin.  A CTA owns
// a 16 x 4 x 2 (w, h, d) block of output voxels and all output channels; for
// each 16-channel input chunk it stages the (18 x 6 x 4) halo tile and the 27
// taps of weights in shared memory (rows padded to 48 bytes so the ldmatrix
// row groups hit distinct banks), then every warp multiplies two w-rows of 16
// voxels against all output channels, tap by tap.  The input gradient is the
// same kernel with flipped, transposed weights.
#include <cuda_bf16.h>
#include <stdint.h>

#include "nn_internal.h"

namespace mg {
namespace nn {

namespace {

constexpr int TW = 16, TH = 4, TD = 2;            // output voxel tile
constexpr int HW = TW + 2, HH = TH + 2, HD = TD + 2;  // halo tile
constexpr int HALO = HW * HH * HD;                // 432 voxels
constexpr int ROWB = 48;                          // bytes per 16-channel row in smem
constexpr int kConvThreads = 128;                 // 4 warps x 2 w-rows = 8 rows

inline unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                        uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r0), "=r"(r1)
               : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float* c, uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// NF = Cout / 8 output-channel fragments.
template <int NF>
__global__ void __launch_bounds__(kConvThreads) k_conv3d(ConvArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* halo = smem;                       // HALO rows of ROWB bytes
  unsigned char* wsm = smem + HALO * ROWB;          // [27][NF*8] rows of ROWB bytes
  const int Co = NF * 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // tile origin
  const int tiles_w = (a.W + TW - 1) / TW, tiles_h = (a.H + TH - 1) / TH;
  int bid = blockIdx.x;
  const int tw = bid % tiles_w;
  bid /= tiles_w;
  const int th = bid % tiles_h;
  bid /= tiles_h;
  const int tiles_d = (a.D + TD - 1) / TD;
  const int td = bid % tiles_d;
  const int n = bid / tiles_d;
  const int w0 = tw * TW, h0 = th * TH, d0 = td * TD;

  float acc[2][NF][4];
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[m][f][q] = 0.0f;

  const int nchunks = (a.C1 + a.C2) / 16;
  for (int ch = 0; ch < nchunks; ++ch) {
    // input chunk: channels [16 ch, 16 ch + 16) of concat(x1, x2)
    const bool first = ch * 16 < a.C1;
    const __nv_bfloat16* src = first ? a.x1 : a.x2;
    const int cs = first ? a.C1 : a.C2;
    const int c0 = first ? ch * 16 : ch * 16 - a.C1;
    // halo tile: 432 voxels x 32 bytes, as 16-byte pieces
    for (int q = threadIdx.x; q < HALO * 2; q += kConvThreads) {
      const int v = q >> 1, half = q & 1;
      const int hx = v % HW, hy = (v / HW) % HH, hz = v / (HW * HH);
      const int x = w0 + hx - 1, y = h0 + hy - 1, z = d0 + hz - 1;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (x >= 0 && x < a.W && y >= 0 && y < a.H && z >= 0 && z < a.D) {
        const long long vox = (((long long)n * a.D + z) * a.H + y) * a.W + x;
        val = *reinterpret_cast<const uint4*>(src + vox * cs + c0 + half * 8);
      }
      *reinterpret_cast<uint4*>(halo + v * ROWB + half * 16) = val;
    }
    // weights of this chunk: [tap][co] rows of 16 input channels
    for (int q = threadIdx.x; q < 27 * Co * 2; q += kConvThreads) {
      const int half = q & 1, r = q >> 1;
      const int co = r % Co, tap = r / Co;
      const uint4 val = *reinterpret_cast<const uint4*>(
          a.w + ((long long)co * 27 + tap) * (a.C1 + a.C2) + ch * 16 + half * 8);
      *reinterpret_cast<uint4*>(wsm + (tap * Co + co) * ROWB + half * 16) = val;
    }
    __syncthreads();
    // this warp's two w-rows: rows 2 warp, 2 warp + 1 of the 8 (h, d) rows
#pragma unroll 1
    for (int tap = 0; tap < 27; ++tap) {
      const int kw = tap % 3, kh = (tap / 3) % 3, kd = tap / 9;
      uint32_t af[2][4];
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const int row = warp * 2 + m;
        const int hy = row % TH, hz = row / TH;
        // ldmatrix x4: matrices (rows 0-7, k 0-7), (rows 8-15, k 0-7),
        // (rows 0-7, k 8-15), (rows 8-15, k 8-15); lane gives one row address
        const int mj = lane >> 3, rr = lane & 7;
        const int wx = rr + 8 * (mj & 1);
        const int v = ((hz + kd) * HH + (hy + kh)) * HW + (wx + kw);
        ldsm_x4(smem_u32(halo + v * ROWB + (mj >> 1) * 16), af[m][0], af[m][1], af[m][2],
                af[m][3]);
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        uint32_t b0, b1;
        // x2: matrices (co 8f..8f+7, k 0-7), (co 8f..8f+7, k 8-15)
        const int mj = (lane >> 3) & 1, rr = lane & 7;
        ldsm_x2(smem_u32(wsm + (tap * Co + f * 8 + rr) * ROWB + mj * 16), b0, b1);
#pragma unroll
        for (int m = 0; m < 2; ++m)
          mma_bf16(acc[m][f], af[m][0], af[m][1], af[m][2], af[m][3], b0, b1);
      }
    }
    __syncthreads();
  }
  // epilogue: bias, ReLU, BF16, store (two outputs split by channel)
  const int g = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const int row = warp * 2 + m;
    const int y = h0 + row % TH, z = d0 + row / TH;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int x = w0 + g + 8 * half;
      if (x >= a.W || y >= a.H || z >= a.D) continue;
      const long long vox = (((long long)n * a.D + z) * a.H + y) * a.W + x;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const int co = f * 8 + tq * 2;
        float v0 = acc[m][f][half * 2 + 0], v1 = acc[m][f][half * 2 + 1];
        if (a.bias) {
          v0 += a.bias[co];
          v1 += a.bias[co + 1];
        }
        if (a.relu) {
          v0 = fmaxf(v0, 0.0f);
          v1 = fmaxf(v1, 0.0f);
        }
        const __nv_bfloat162 pr = __floats2bfloat162_rn(v0, v1);
        if (co < a.O1)
          *reinterpret_cast<__nv_bfloat162*>(a.y1 + vox * a.Ys1 + a.Yo1 + co) = pr;
        else
          *reinterpret_cast<__nv_bfloat162*>(a.y2 + vox * a.Ys2 + a.Yo2 + (co - a.O1)) = pr;
      }
    }
  }
}

// W'[ci][t][co] = W[co][26 - t][ci]: weights of the input-gradient conv.
__global__ void k_flip_weights(const __nv_bfloat16* w, int Co, int Ci, __nv_bfloat16* wt) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)Co * 27 * Ci) return;
  const int ci = (int)(q % Ci);
  const int t = (int)((q / Ci) % 27);
  const int co = (int)(q / (27LL * Ci));
  wt[((long long)ci * 27 + (26 - t)) * Co + co] = w[q];
}

// dY <- dY * [Y > 0] (ReLU backward on the stored post-activation output)
__global__ void k_relu_bwd(const __nv_bfloat16* y, __nv_bfloat16* dy, long long n) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  if (!(__bfloat162float(y[q]) > 0.0f)) dy[q] = __float2bfloat16(0.0f);
}

// 2x average pooling (D, H, W even) and its backward
__global__ void k_pool(const __nv_bfloat16* x, int N, int D, int H, int W, int C,
                       __nv_bfloat16* y) {
  const int d2 = D / 2, h2 = H / 2, w2 = W / 2;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)N * d2 * h2 * w2 * C) return;
  const int c = (int)(q % C);
  long long v = q / C;
  const int x0 = (int)(v % w2);
  v /= w2;
  const int y0 = (int)(v % h2);
  v /= h2;
  const int z0 = (int)(v % d2);
  const int n = (int)(v / d2);
  float s = 0.0f;
  for (int k = 0; k < 8; ++k) {
    const long long vox =
        (((long long)n * D + 2 * z0 + (k >> 2)) * H + 2 * y0 + ((k >> 1) & 1)) * W + 2 * x0 + (k & 1);
    s += __bfloat162float(x[vox * C + c]);
  }
  y[q] = __float2bfloat16(0.125f * s);
}

__global__ void k_pool_bwd(const __nv_bfloat16* dy, int N, int D, int H, int W, int C,
                           __nv_bfloat16* dx, int acc) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)N * D * H * W * C) return;
  const int c = (int)(q % C);
  long long v = q / C;
  const int x = (int)(v % W);
  v /= W;
  const int y = (int)(v % H);
  v /= H;
  const int z = (int)(v % D);
  const int n = (int)(v / D);
  const long long p = (((long long)n * (D / 2) + z / 2) * (H / 2) + y / 2) * (W / 2) + x / 2;
  const float v0 = acc ? __bfloat162float(dx[q]) : 0.0f;
  dx[q] = __float2bfloat16(v0 + 0.125f * __bfloat162float(dy[p * C + c]));
}

// nearest 2x upsampling (output D, H, W) and its backward (sum of children)
__global__ void k_up(const __nv_bfloat16* x, int N, int D, int H, int W, int C,
                     __nv_bfloat16* y) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)N * D * H * W * C) return;
  const int c = (int)(q % C);
  long long v = q / C;
  const int xx = (int)(v % W);
  v /= W;
  const int yy = (int)(v % H);
  v /= H;
  const int z = (int)(v % D);
  const int n = (int)(v / D);
  const long long p = (((long long)n * (D / 2) + z / 2) * (H / 2) + yy / 2) * (W / 2) + xx / 2;
  y[q] = x[p * C + c];
}

__global__ void k_up_bwd(const __nv_bfloat16* dy, int N, int D, int H, int W, int C,
                         __nv_bfloat16* dx) {
  const int d2 = D / 2, h2 = H / 2, w2 = W / 2;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)N * d2 * h2 * w2 * C) return;
  const int c = (int)(q % C);
  long long v = q / C;
  const int x0 = (int)(v % w2);
  v /= w2;
  const int y0 = (int)(v % h2);
  v /= h2;
  const int z0 = (int)(v % d2);
  const int n = (int)(v / d2);
  float s = 0.0f;
  for (int k = 0; k < 8; ++k) {
    const long long vox =
        (((long long)n * D + 2 * z0 + (k >> 2)) * H + 2 * y0 + ((k >> 1) & 1)) * W + 2 * x0 + (k & 1);
    s += __bfloat162float(dy[vox * C + c]);
  }
  dx[q] = __float2bfloat16(s);
}

// dW[co][t][ci] += sum_v dY[v][co] X[v + off(t)][ci]: one CTA per (tap, voxel
// split); each thread owns a 4 x 4 block of (co, ci); voxels are staged in
// shared memory 32 at a time.  FP32 CUDA cores, FP32 atomics per CTA.
template <int CO, int CI>
__global__ void __launch_bounds__(256) k_wgrad(const __nv_bfloat16* __restrict__ dy,
                                               const __nv_bfloat16* __restrict__ x1, int C1,
                                               const __nv_bfloat16* __restrict__ x2, int C2,
                                               int N, int D, int H, int W, float* dw,
                                               int splits) {
  constexpr int VB = 32;
  constexpr int BCO = CO / 4, BCI = CI / 4;  // 4 x 4 (co, ci) blocks
  constexpr int NB = (BCO * BCI + 255) / 256;
  __shared__ float sdy[VB][CO];
  __shared__ float sx[VB][CI + 1];
  const int tap = blockIdx.x;
  const int kw = tap % 3 - 1, kh = (tap / 3) % 3 - 1, kd = tap / 9 - 1;
  const long long nvox = (long long)N * D * H * W;
  const long long per = (nvox + splits - 1) / splits;
  const long long v0 = blockIdx.y * per, v1 = min(nvox, v0 + per);
  float acc[NB][4][4] = {};
  for (long long vb = v0; vb < v1; vb += VB) {
    for (int q = threadIdx.x; q < VB * (CO + CI); q += 256) {
      const int r = q / (CO + CI), c = q % (CO + CI);
      const long long v = vb + r;
      float val = 0.0f;
      if (v < v1) {
        if (c < CO) {
          val = __bfloat162float(dy[v * CO + c]);
        } else {
          long long t = v;
          const int xx = (int)(t % W);
          t /= W;
          const int yy = (int)(t % H);
          t /= H;
          const int zz = (int)(t % D);
          const int nn = (int)(t / D);
          const int xs = xx + kw, ys = yy + kh, zs = zz + kd;
          if (xs >= 0 && xs < W && ys >= 0 && ys < H && zs >= 0 && zs < D) {
            const long long src = (((long long)nn * D + zs) * H + ys) * W + xs;
            const int ci = c - CO;
            val = ci < C1 ? __bfloat162float(x1[src * C1 + ci])
                          : __bfloat162float(x2[src * C2 + ci - C1]);
          }
        }
      }
      if (c < CO) sdy[r][c] = val;
      else sx[r][c - CO] = val;
    }
    __syncthreads();
#pragma unroll
    for (int nb = 0; nb < NB; ++nb) {
      const int blk = threadIdx.x + nb * 256;
      if (blk < BCO * BCI) {
        const int bo = blk / BCI, bi = blk % BCI;
#pragma unroll 4
        for (int r = 0; r < VB; ++r) {
          float dv[4], xv[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            dv[q] = sdy[r][bo * 4 + q];
            xv[q] = sx[r][bi * 4 + q];
          }
#pragma unroll
          for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[nb][p][q] = fmaf(dv[p], xv[q], acc[nb][p][q]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int nb = 0; nb < NB; ++nb) {
    const int blk = threadIdx.x + nb * 256;
    if (blk < BCO * BCI) {
      const int bo = blk / BCI, bi = blk % BCI;
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          atomicAdd(&dw[((long long)(bo * 4 + p) * 27 + tap) * CI + bi * 4 + q], acc[nb][p][q]);
    }
  }
}

// db[c] += sum_v dY[v][c]
__global__ void k_bias_grad(const __nv_bfloat16* dy, long long nvox, int C, float* db) {
  const int c = blockIdx.y;
  float s = 0.0f;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nvox;
       v += (long long)gridDim.x * blockDim.x)
    s += __bfloat162float(dy[v * C + c]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&db[c], s);
}

// 1x1x1 head: out[v] = sum_c x[v][c] w[c] + b (FP32 output)
__global__ void k_head(const __nv_bfloat16* x, int C, const float* w, const float* b,
                       long long nvox, float* out) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvox) return;
  float s = b[0];
  for (int c = 0; c < C; ++c) s = fmaf(__bfloat162float(x[v * C + c]), w[c], s);
  out[v] = s;
}

// head backward: dx[v][c] = g[v] w[c]; dw[c] += sum_v g[v] x[v][c]; db += sum g
__global__ void k_head_bwd(const __nv_bfloat16* x, int C, const float* w, const float* g,
                           long long nvox, __nv_bfloat16* dx, float* dw, float* db) {
  __shared__ float part[64];
  if (threadIdx.x < 64) part[threadIdx.x] = 0.0f;
  __syncthreads();
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < nvox) {
    const float gv = g[v];
    for (int c = 0; c < C; ++c) {
      dx[v * C + c] = __float2bfloat16(gv * w[c]);
      atomicAdd(&part[c], gv * __bfloat162float(x[v * C + c]));
    }
    atomicAdd(&part[C], gv);
  }
  __syncthreads();
  if (threadIdx.x < C) atomicAdd(&dw[threadIdx.x], part[threadIdx.x]);
  if (threadIdx.x == C) atomicAdd(db, part[C]);
}

// MSE: loss += sum (p - t)^2 / n; g = 2 (p - t) / n
__global__ void k_mse(const float* p, const float* t, long long n, float* g, float* loss) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float e = 0.0f;
  if (v < n) {
    const float d = p[v] - t[v];
    g[v] = 2.0f * d / (float)n;
    e = d * d / (float)n;
  }
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, e);
}

// Adam on FP32 master weights (bias-corrected), then the BF16 copy.
__global__ void k_adam(float* w, float* m, float* v, const float* g, long long n, float lr,
                       float b1, float b2, float eps, float c1, float c2, __nv_bfloat16* w16) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const float gq = g[q];
  const float mq = b1 * m[q] + (1.0f - b1) * gq;
  const float vq = b2 * v[q] + (1.0f - b2) * gq * gq;
  m[q] = mq;
  v[q] = vq;
  const float wq = w[q] - lr * (mq / c1) / (sqrtf(vq / c2) + eps);
  w[q] = wq;
  if (w16) w16[q] = __float2bfloat16(wq);
}

__global__ void k_f32_to_bf16(const float* x, long long n, __nv_bfloat16* y) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) y[q] = __float2bfloat16(x[q]);
}

// network input [v][16]: channel 0 = a[v] * sa, channel 1 = b[v] * sb (FP64
// fields), channels 2..15 zero
__global__ void k_pack_input(const double* a, double sa, const double* b, double sb,
                             long long nvox, __nv_bfloat16* x) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvox) return;
  __nv_bfloat16 z = __float2bfloat16(0.0f);
  __nv_bfloat16 row[16];
  row[0] = __float2bfloat16((float)(a[v] * sa));
  row[1] = __float2bfloat16((float)(b[v] * sb));
  for (int c = 2; c < 16; ++c) row[c] = z;
  uint4* dst = reinterpret_cast<uint4*>(x + v * 16);
  dst[0] = *reinterpret_cast<uint4*>(&row[0]);
  dst[1] = *reinterpret_cast<uint4*>(&row[8]);
}

// phi_guess = phi_prev + scale * delta (FP32 network output)
__global__ void k_apply_delta(const double* prev, const float* delta, double scale, long long n,
                              double* out) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) out[v] = prev[v] + scale * (double)delta[v];
}

__global__ void k_target(const double* phi, const double* prev, double scale, long long n,
                         float* t) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) t[v] = (float)((phi[v] - prev[v]) * scale);
}

}  // namespace

// ---- launchers ------------------------------------------------------------

size_t conv_smem_bytes(int cout) { return (size_t)(HALO + 27 * cout) * ROWB; }

bool conv_supported(int cin_total, int cout) {
  return cin_total % 16 == 0 && cin_total > 0 &&
         (cout == 16 || cout == 32 || cout == 48 || cout == 64 || cout == 96);
}

cudaError_t launch_conv3d(const ConvArgs& a, int cout, cudaStream_t s) {
  const long long tiles = (long long)a.N * ((a.D + TD - 1) / TD) * ((a.H + TH - 1) / TH) *
                          ((a.W + TW - 1) / TW);
  const size_t sm = conv_smem_bytes(cout);
  static bool attr_done[13] = {};
  const int nf = cout / 8;
  auto go = [&](auto kernel) {
    if (!attr_done[nf]) {
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm + 1024);
      attr_done[nf] = true;
    }
    kernel<<<(unsigned)tiles, kConvThreads, sm, s>>>(a);
  };
  switch (nf) {
    case 2: go(k_conv3d<2>); break;
    case 4: go(k_conv3d<4>); break;
    case 6: go(k_conv3d<6>); break;
    case 8: go(k_conv3d<8>); break;
    case 12: go(k_conv3d<12>); break;
    default: return cudaErrorInvalidValue;
  }
  add_launches(1);
  return cudaGetLastError();
}

void launch_flip_weights(const __nv_bfloat16* w, int co, int ci, __nv_bfloat16* wt,
                         cudaStream_t s) {
  k_flip_weights<<<nblk((long long)co * 27 * ci), 256, 0, s>>>(w, co, ci, wt);
  add_launches(1);
}

void launch_relu_bwd(const __nv_bfloat16* y, __nv_bfloat16* dy, long long n, cudaStream_t s) {
  k_relu_bwd<<<nblk(n), 256, 0, s>>>(y, dy, n);
  add_launches(1);
}

void launch_pool(const __nv_bfloat16* x, int N, int D, int H, int W, int C, __nv_bfloat16* y,
                 cudaStream_t s) {
  k_pool<<<nblk((long long)N * (D / 2) * (H / 2) * (W / 2) * C), 256, 0, s>>>(x, N, D, H, W, C, y);
  add_launches(1);
}

void launch_pool_bwd(const __nv_bfloat16* dy, int N, int D, int H, int W, int C,
                     __nv_bfloat16* dx, int acc, cudaStream_t s) {
  k_pool_bwd<<<nblk((long long)N * D * H * W * C), 256, 0, s>>>(dy, N, D, H, W, C, dx, acc);
  add_launches(1);
}

void launch_up(const __nv_bfloat16* x, int N, int D, int H, int W, int C, __nv_bfloat16* y,
               cudaStream_t s) {
  k_up<<<nblk((long long)N * D * H * W * C), 256, 0, s>>>(x, N, D, H, W, C, y);
  add_launches(1);
}

void launch_up_bwd(const __nv_bfloat16* dy, int N, int D, int H, int W, int C, __nv_bfloat16* dx,
                   cudaStream_t s) {
  k_up_bwd<<<nblk((long long)N * (D / 2) * (H / 2) * (W / 2) * C), 256, 0, s>>>(dy, N, D, H, W, C,
                                                                                dx);
  add_launches(1);
}

cudaError_t launch_wgrad(const __nv_bfloat16* dy, int co, const __nv_bfloat16* x1, int c1,
                         const __nv_bfloat16* x2, int c2, int N, int D, int H, int W, float* dw,
                         cudaStream_t s) {
  const long long nvox = (long long)N * D * H * W;
  int splits = (int)std::min<long long>(4096, (nvox + 1023) / 1024);
  if (splits < 1) splits = 1;
  dim3 g(27, splits);
  const int ci = c1 + c2;
#define WG(CO_, CI_)                                                                       \
  if (co == CO_ && ci == CI_) {                                                            \
    k_wgrad<CO_, CI_><<<g, 256, 0, s>>>(dy, x1, c1, x2, c2, N, D, H, W, dw, splits);       \
    add_launches(1);                                                                       \
    return cudaGetLastError();                                                             \
  }
  WG(16, 16) WG(32, 16) WG(32, 32) WG(48, 32) WG(48, 48) WG(64, 48) WG(64, 64)
  WG(48, 64) WG(48, 96) WG(32, 48) WG(32, 64) WG(16, 32)
#undef WG
  return cudaErrorInvalidValue;
}

void launch_bias_grad(const __nv_bfloat16* dy, long long nvox, int C, float* db, cudaStream_t s) {
  dim3 g((unsigned)std::min<long long>(1024, (nvox + 255) / 256), C);
  k_bias_grad<<<g, 256, 0, s>>>(dy, nvox, C, db);
  add_launches(1);
}

void launch_head(const __nv_bfloat16* x, int C, const float* w, const float* b, long long nvox,
                 float* out, cudaStream_t s) {
  k_head<<<nblk(nvox), 256, 0, s>>>(x, C, w, b, nvox, out);
  add_launches(1);
}

void launch_head_bwd(const __nv_bfloat16* x, int C, const float* w, const float* g,
                     long long nvox, __nv_bfloat16* dx, float* dw, float* db, cudaStream_t s) {
  k_head_bwd<<<nblk(nvox), 256, 0, s>>>(x, C, w, g, nvox, dx, dw, db);
  add_launches(1);
}

void launch_mse(const float* p, const float* t, long long n, float* g, float* loss,
                cudaStream_t s) {
  k_mse<<<nblk(n), 256, 0, s>>>(p, t, n, g, loss);
  add_launches(1);
}

void launch_adam(float* w, float* m, float* v, const float* g, long long n, float lr, float b1,
                 float b2, float eps, int step, __nv_bfloat16* w16, cudaStream_t s) {
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  k_adam<<<nblk(n), 256, 0, s>>>(w, m, v, g, n, lr, b1, b2, eps, c1, c2, w16);
  add_launches(1);
}

void launch_f32_to_bf16(const float* x, long long n, __nv_bfloat16* y, cudaStream_t s) {
  k_f32_to_bf16<<<nblk(n), 256, 0, s>>>(x, n, y);
  add_launches(1);
}

void launch_pack_input(const double* a, double sa, const double* b, double sb, long long nvox,
                       __nv_bfloat16* x, cudaStream_t s) {
  k_pack_input<<<nblk(nvox), 256, 0, s>>>(a, sa, b, sb, nvox, x);
  add_launches(1);
}

void launch_target(const double* phi, const double* prev, double scale, long long n, float* t,
                   cudaStream_t s) {
  k_target<<<nblk(n), 256, 0, s>>>(phi, prev, scale, n, t);
  add_launches(1);
}

void launch_apply_delta(const double* prev, const float* delta, double scale, long long n,
                        double* out, cudaStream_t s) {
  k_apply_delta<<<nblk(n), 256, 0, s>>>(prev, delta, scale, n, out);
  add_launches(1);
}

}  // namespace nn
}  // namespace mg
