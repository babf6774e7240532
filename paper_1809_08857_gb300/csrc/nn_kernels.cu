// Kernels of the learned warm start: a 3D U-Net on BF16 activations with
// FP32 accumulation (the network maps (rho_n, phi_{n-1}) to phi_n - phi_{n-1},
// motivated by the infrequent elliptic re-solves of Sec. 2.2).
//
// Layout: activations channels-last [N][D][H][W][C] in BF16, C a multiple of
// 16; 3x3x3 conv weights [Cout][27][Cin] (tap t = (kd*3 + kh)*3 + kw) in
// BF16 with an FP32 master copy.
//
// conv3d forward is an implicit GEMM on the tcgen05 tensor cores (BF16 x
// BF16 -> FP32 accumulators in tensor memory, operands staged in shared
// memory by the tensor memory accelerator, one producer and one MMA-issuing
// thread per CTA; a persistent form with a ring of stages and two
// accumulators for large grids): M = output voxels, N = Cout, K = 27 Cin.
// The input gradient is the same kernel with flipped, transposed weights;
// the weight gradient is a second tcgen05 GEMM over voxels.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <algorithm>
#include <stdint.h>

#include "nn_internal.h"

namespace mg {
namespace nn {

namespace {

// Output tile of a CTA: MT UMMA M-tiles of 8 (w) x 16 (h) voxels at d0 ..
// d0 + MT - 1 (MT = 2: 256 voxels sharing the weights staged in shared
// memory; MT = 1 on small grids, for more CTAs).
constexpr int TW = 8, TH = 16;
constexpr int HW = TW + 2, HH = TH + 2;  // halo tile rows
constexpr int kConvThreads = 128;                     // 4 warps: TMEM lane quarters
constexpr int kMmaM = 128;                            // rows (voxels) of one MMA
constexpr long long kWaitIters = 1ll << 24;           // bound of an mbarrier wait (tries)
constexpr unsigned long long kWaitNs = 2000000000ull; // and its time limit (2 s)
constexpr int kMaxStages = 2;                         // shared-memory stages of the K loop

__host__ __device__ constexpr int round1k(int b) { return (b + 1023) / 1024 * 1024; }

// Shared-memory plan of one stage: the two 8-channel halves of the halo
// (each [voxel] x 16 B, padded to 1 KB) and the chunk's weights
// [tap][half][co] x 16 B.
template <int N, int MT>
struct ConvPlan {
  static constexpr int kHalo = HW * HH * (MT + 2);         // halo voxels
  static constexpr int kHalfBytes = round1k(kHalo * 16);   // one channel half
  static constexpr int kHaloTx = 2 * kHalo * 16;           // bytes the two halo loads bring
  static constexpr int kWBytes = 27 * 2 * N * 16;          // weights of a 16-channel chunk
  static constexpr int kStage = 2 * kHalfBytes + round1k(kWBytes);
  static constexpr int smem(int stages) { return stages * kStage + 1024; }  // + alignment slack
  // TMEM columns: MT accumulators, each starting on a multiple of 32
  // columns; the allocation is a power of two >= 32
  static constexpr int kTile = (N + 31) / 32 * 32;
  static constexpr int kAlloc = MT * kTile <= 32 ? 32 : MT * kTile <= 64 ? 64
                                : MT * kTile <= 128 ? 128 : MT * kTile <= 256 ? 256 : 512;
};

// Set when a CTA gave up waiting on an mbarrier (its outputs are not written).
__device__ unsigned g_conv_timeout = 0;

inline unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of the tensor-core MMA for an operand in
// the K-major layout without swizzle: 8-row x 16-byte core matrices whose
// rows are 16 bytes apart; lbo = byte distance between the two core
// matrices adjacent in K, sbo = between those adjacent in M (or N); bits
// 46-47 carry the descriptor version of this architecture (1).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3ffffu) >> 4) | ((uint64_t)((lbo & 0x3ffffu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3ffffu) >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 accumulator,
// both operands K-major, M x N.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n) {
  return (1u << 4)      // D: FP32
         | (1u << 7)    // A: BF16
         | (1u << 10)   // B: BF16
         | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the mbarrier phase with the given parity; false after kWaitIters
// unsuccessful tries or limit_ns nanoseconds, whichever comes first.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity,
                                          unsigned long long limit_ns = kWaitNs) {
  unsigned long long t0 = 0;
  for (long long it = 0; it < kWaitIters; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63) == 0) {
      const unsigned long long t = now_ns();
      if (it == 0) t0 = t;
      else if (t - t0 > limit_ns) return false;
    }
  }
  return false;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar),
               "r"(bytes)
               : "memory");
}

// Tiled tensor loads (global -> shared), completing on an mbarrier.
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, uint32_t mbar,
                                            int c0, int c1, int c2, int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(mbar), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
      "r"(c4)
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, uint32_t mbar,
                                            int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(mbar), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}

// The MT x 27 MMAs of one 16-channel chunk.  The A view of tap (kw, kh, kd)
// for M-tile s starts kw + HW (kh + HH (kd + s)) 16-byte rows into the halo
// and tap t's weights t 2 N rows into the chunk's weights, so every
// descriptor is the chunk's first one plus a compile-time count of 16-byte
// units in its address field (no carry: shared addresses stay below 256 KB);
// the unrolled loop issues each MMA after one add per operand.
template <int N, int MT, int kTileCols>
__device__ __forceinline__ void conv_chunk_mmas(uint32_t acc, uint32_t halo, uint32_t wsm,
                                                uint32_t half_bytes, uint32_t idesc,
                                                bool accumulate) {
  const uint64_t a0 = smem_desc(halo, half_bytes, HW * 16);
  const uint64_t b0 = smem_desc(wsm, N * 16, 128);
#pragma unroll
  for (int s = 0; s < MT; ++s)
#pragma unroll
    for (int tap = 0; tap < 27; ++tap) {
      const int kw = tap % 3, kh = (tap / 3) % 3, kd = tap / 9;
      mma_f16(acc + (uint32_t)(s * kTileCols), a0 + (uint64_t)(kw + HW * (kh + HH * (kd + s))),
              b0 + (uint64_t)(tap * 2 * N), idesc, (accumulate || tap > 0) ? 1u : 0u);
    }
}

// Tiled tensor store (shared -> global) of a 5D box, as one bulk group.
__device__ __forceinline__ void tma_store_5d(const CUtensorMap* map, uint32_t src, int c0, int c1,
                                             int c2, int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group"
      " [%0, {%2, %3, %4, %5, %6}], [%1];\n" ::"l"(reinterpret_cast<uint64_t>(map)),
      "r"(src), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
      : "memory");
}

// 3D convolution (3x3x3, pad 1) as an implicit GEMM on the fifth-generation
// tensor cores: M = output voxels, N = Cout, K = 27 taps x Cin, in chunks
// of 16 input channels.
//
// Staging: for every chunk the producer thread (warp 0) issues three tiled
// tensor loads into a free stage: the halo tile of each 8-channel half
// ([voxel] x 16 B, voxels w-fastest; out-of-range voxels are zero-filled by
// the copy engine, which is the convolution's zero padding) and the chunk's
// weights [tap][half][co] x 16 B (a 4D view of the [co][tap][ci] weights).
// The A operand of tap (kw, kh, kd) is the halo itself seen from offset
// (kw, kh, kd): 8 voxels along w form a core matrix (contiguous 16-byte
// rows), the next h row is one halo row further (sbo), the other channel
// half one padded half-plane further (lbo).
//
// The number of stages S (1 or 2) is a launch argument: with two or more
// waves of CTAs one stage per CTA is faster (more CTAs per SM hide each
// other's load latency: 348 against 463 us for 32 -> 32 channels on 128^3),
// on small grids two (26 against 36 us for 96 -> 48 on 2 x 16^3).
//
// MMA: one thread (warp 1) waits for a stage's loads, issues its MT x 27
// MMAs into the MT TMEM accumulators (128 lanes = voxels, Cout columns) and
// commits them to the stage's "empty" barrier, which frees the stage for the
// producer; after the last chunk it commits to the "done" barrier.  Every
// wait is bounded; a CTA that gives up sets g_conv_timeout, waits (bounded)
// for its copies and MMAs still in flight and writes nothing.
//
// Epilogue: the four warps read their TMEM lane quarters with tcgen05.ld and
// apply bias and ReLU.  With tma_out (every output channel slice 16-byte
// aligned), the BF16 tile is staged in the first stage's shared memory
// ([z][y][x][channel], one region per output) and written by one tiled
// tensor store per output, which also clips the tile at the volume's edge:
// each output byte crosses to L2 once, where per-thread stores of a voxel's
// channels sent every 32-byte sector as eight partial writes.  Otherwise
// each thread stores its voxel's channels itself.
template <int N, int MT>
__global__ void __launch_bounds__(kConvThreads)
    k_conv3d(ConvArgs a, const __grid_constant__ CUtensorMap map_x1,
             const __grid_constant__ CUtensorMap map_x2, const __grid_constant__ CUtensorMap map_w,
             const __grid_constant__ CUtensorMap map_y1,
             const __grid_constant__ CUtensorMap map_y2, int S, int tma_out) {
  using P = ConvPlan<N, MT>;
  constexpr int TD = MT;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[2 * kMaxStages + 1];  // full[], empty[], done
  __shared__ uint32_t tmem_slot;
  __shared__ int issued_s, committed_s, fail_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tiles_w = (a.W + TW - 1) / TW, tiles_h = (a.H + TH - 1) / TH;
  const int tiles_d = (a.D + TD - 1) / TD;
  int bid = blockIdx.x;
  const int tw = bid % tiles_w;
  bid /= tiles_w;
  const int th = bid % tiles_h;
  bid /= tiles_h;
  const int td = bid % tiles_d;
  const int n = bid / tiles_d;
  const int w0 = tw * TW, h0 = th * TH, d0 = td * TD;
  const int nchunks = (a.C1 + a.C2) / 16;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const unsigned long long lim = a.wait_ns ? a.wait_ns : kWaitNs;
  const uint32_t bar0 = smem_u32(&bars[0]);
  auto full = [&](int st) { return bar0 + 8u * (uint32_t)st; };
  auto empty = [&](int st) { return bar0 + 8u * (uint32_t)(kMaxStages + st); };
  const uint32_t done_bar = bar0 + 8u * (uint32_t)(2 * kMaxStages);

  if (tid == 0) {
    for (int i = 0; i < 2 * kMaxStages + 1; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0 + 8u * i) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    issued_s = 0;
    committed_s = 0;
    fail_s = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(P::kAlloc)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (tid == 0) {
    // producer: chunk ch goes to stage ch % S once the MMAs of chunk ch - S
    // (that stage's previous use, phase ch / S - 1 of its empty barrier) are done
    for (int ch = 0; ch < nchunks; ++ch) {
      const int st = ch % S;
      if (ch >= S && !mbar_wait(empty(st), (uint32_t)((ch / S - 1) & 1), lim)) {
        atomicExch(&fail_s, 1);
        break;
      }
      if (*(volatile int*)&fail_s) break;
      const uint32_t halo = base + (uint32_t)(st * P::kStage);
      const uint32_t wsm = halo + 2u * P::kHalfBytes;
      const bool first = ch * 16 < a.C1;
      const CUtensorMap* mx = first ? &map_x1 : &map_x2;
      const int c0 = first ? ch * 16 : ch * 16 - a.C1;
      mbar_expect_tx(full(st), (uint32_t)(P::kHaloTx + P::kWBytes) + (ch == 0 ? a.stall_bytes : 0u));
      tma_load_5d(halo, mx, full(st), c0, w0 - 1, h0 - 1, d0 - 1, n);
      tma_load_5d(halo + P::kHalfBytes, mx, full(st), c0 + 8, w0 - 1, h0 - 1, d0 - 1, n);
      tma_load_4d(wsm, &map_w, full(st), 0, 0, 2 * ch, 0);
      issued_s = ch + 1;
    }
  } else if (tid == 32) {
    // MMA issue: chunk ch waits for phase ch / S of its stage's full barrier
    const uint32_t idesc = instr_desc(kMmaM, N);
    for (int ch = 0; ch < nchunks; ++ch) {
      const int st = ch % S;
      if (!mbar_wait(full(st), (uint32_t)((ch / S) & 1), lim)) {
        atomicExch(&fail_s, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t halo = base + (uint32_t)(st * P::kStage);
      conv_chunk_mmas<N, TD, P::kTile>(tmem, halo, halo + 2u * P::kHalfBytes, P::kHalfBytes, idesc,
                                       ch > 0);
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              empty(st))
          : "memory");
      committed_s = ch + 1;
    }
    if (!*(volatile int*)&fail_s)
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              done_bar)
          : "memory");
  }
  __syncwarp();
  // every thread: wait for the last MMAs (bounded; skipped once a role gave up)
  bool ok = !*(volatile int*)&fail_s && mbar_wait(done_bar, 0, lim);
  ok = __syncthreads_and(ok) && !fail_s;
  if (!ok && tid == 0) {
    atomicExch(&g_conv_timeout, 1u);
    // bounded waits for the copies and MMAs still in flight
    for (int ch = issued_s - S < 0 ? 0 : issued_s - S; ch < issued_s; ++ch)
      mbar_wait(full(ch % S), (uint32_t)((ch / S) & 1), lim);
    if (committed_s > 0)
      mbar_wait(empty((committed_s - 1) % S), (uint32_t)(((committed_s - 1) / S) & 1), lim);
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

  if (ok) {
    // epilogue: TMEM lane 32 warp + lane = voxel (w = m % 8, h = m / 8)
    const int m = warp * 32 + lane;
    const int x = w0 + (m % TW), y = h0 + m / TW;
    const int O2 = N - a.O1;
    unsigned char* stg = smem_raw + (base - smem_u32(smem_raw));  // stage 0, free now
    unsigned char* stg2 = stg + TD * kMmaM * a.O1 * 2;
#pragma unroll 1
    for (int s = 0; s < TD; ++s) {
      const int z = d0 + s;
      const bool in = x < a.W && y < a.H && z < a.D;
      const long long vox = (((long long)n * a.D + z) * a.H + y) * a.W + x;
#pragma unroll 1
      for (int cb = 0; cb < N; cb += 16) {
        uint32_t r[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(s * P::kTile + cb);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
            "%12,%13,%14,%15}, [%16];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
              "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
              "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        uint32_t pk[8];
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          const int co = cb + j;
          float v0 = __uint_as_float(r[j]), v1 = __uint_as_float(r[j + 1]);
          if (a.bias) {
            v0 += a.bias[co];
            v1 += a.bias[co + 1];
          }
          if (a.relu) {
            v0 = fmaxf(v0, 0.0f);
            v1 = fmaxf(v1, 0.0f);
          }
          const __nv_bfloat162 pr = __floats2bfloat162_rn(v0, v1);
          pk[j / 2] = *reinterpret_cast<const uint32_t*>(&pr);
        }
        if (tma_out) {
          // the 16 channels lie in one output (O1 is a multiple of 16)
          uint4* d = cb < a.O1
                         ? reinterpret_cast<uint4*>(stg + ((s * kMmaM + m) * a.O1 + cb) * 2)
                         : reinterpret_cast<uint4*>(stg2 + ((s * kMmaM + m) * O2 + cb - a.O1) * 2);
          d[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
          d[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        } else if (in) {
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            const int co = cb + j;
            if (co < a.O1)
              *reinterpret_cast<uint32_t*>(a.y1 + vox * a.Ys1 + a.Yo1 + co) = pk[j / 2];
            else
              *reinterpret_cast<uint32_t*>(a.y2 + vox * a.Ys2 + a.Yo2 + (co - a.O1)) = pk[j / 2];
          }
        }
      }
    }
    if (tma_out) {
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        tma_store_5d(&map_y1, base, a.Yo1, w0, h0, d0, n);
        if (O2 > 0)
          tma_store_5d(&map_y2, base + (uint32_t)(TD * kMmaM * a.O1 * 2), a.Yo2, w0, h0, d0, n);
        asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
        asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
      }
    }
  } else if (tid == 0) {
    atomicExch(&g_conv_timeout, 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(P::kAlloc)
                 : "memory");
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

// Persistent form of k_conv3d for large grids (two M-tiles per tile, Cout
// <= 64): about one CTA per SM walks its tiles (blockIdx.x, + gridDim.x,
// ...) with three roles.  Warp 0 (one thread) fills a ring of S shared-
// memory stages with each chunk's halo (and weights, unless they are
// resident); warp 1 allocates TMEM and one thread issues the MMAs into two
// accumulators used in turn, so the MMAs of one tile run while the four
// epilogue warps (2..5, TMEM lane quarters warp % 4) drain the other: they
// read it back, apply bias and ReLU, stage the BF16 tile in shared memory
// and one of them writes it with tiled tensor stores.  With RW the weights
// of all chunks are loaded once per CTA.  Barriers: full/empty per stage,
// acc_full (MMA commit) and acc_empty (128 epilogue arrivals) per
// accumulator, one for the resident weights; every wait is bounded.
constexpr int kPThreads = 192;
constexpr int kPMaxStages = 4;

template <int N, bool RW>
struct PPlan {
  static constexpr int MT = 2;
  static constexpr int kHalo = HW * HH * (MT + 2);
  static constexpr int kHalfBytes = round1k(kHalo * 16);
  static constexpr int kHaloTx = 2 * kHalo * 16;
  static constexpr int kWBytes = 27 * 2 * N * 16;              // one chunk's weights
  static constexpr int kStage = 2 * kHalfBytes + (RW ? 0 : round1k(kWBytes));
  static constexpr int kStg = MT * kMmaM * N * 2;                // BF16 output tile
  static constexpr int kTile = (N + 31) / 32 * 32;
  static constexpr int kAcc = MT * kTile;                        // columns of one accumulator
  static constexpr int kAlloc = 2 * kAcc <= 32 ? 32 : 2 * kAcc <= 64 ? 64
                                : 2 * kAcc <= 128 ? 128 : 2 * kAcc <= 256 ? 256 : 512;
  // bytes for S stages and nchunks resident chunks of weights
  static constexpr int smem(int S, int nchunks) {
    return S * kStage + (RW ? round1k(nchunks * kWBytes) : 0) + kStg + 1024;
  }
};

template <int N, bool RW>
__global__ void __launch_bounds__(kPThreads, 1)
    k_conv3d_p(ConvArgs a, const __grid_constant__ CUtensorMap map_x1,
               const __grid_constant__ CUtensorMap map_x2, const __grid_constant__ CUtensorMap map_w,
               const __grid_constant__ CUtensorMap map_y1,
               const __grid_constant__ CUtensorMap map_y2, int S) {
  using P = PPlan<N, RW>;
  constexpr int MT = P::MT;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // full[4], empty[4], acc_full[2], acc_empty[2], weights
  __shared__ __align__(8) uint64_t bars[2 * kPMaxStages + 5];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tiles_w = (a.W + TW - 1) / TW, tiles_h = (a.H + TH - 1) / TH;
  const int tiles_d = (a.D + MT - 1) / MT;
  const long long tiles = (long long)a.N * tiles_d * tiles_h * tiles_w;
  const int nch = (a.C1 + a.C2) / 16;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t wreg = base + (uint32_t)(S * P::kStage);                  // resident weights
  const uint32_t stg = wreg + (uint32_t)(RW ? round1k(nch * P::kWBytes) : 0);  // output tile
  const uint32_t bar0 = smem_u32(&bars[0]);
  auto full = [&](int st) { return bar0 + 8u * (uint32_t)st; };
  auto empty = [&](int st) { return bar0 + 8u * (uint32_t)(kPMaxStages + st); };
  auto acc_full = [&](int b) { return bar0 + 8u * (uint32_t)(2 * kPMaxStages + b); };
  auto acc_empty = [&](int b) { return bar0 + 8u * (uint32_t)(2 * kPMaxStages + 2 + b); };
  const uint32_t wbar = bar0 + 8u * (uint32_t)(2 * kPMaxStages + 4);
  auto tile_origin = [&](long long t, int& w0, int& h0, int& d0, int& n) {
    w0 = (int)(t % tiles_w) * TW;
    t /= tiles_w;
    h0 = (int)(t % tiles_h) * TH;
    t /= tiles_h;
    d0 = (int)(t % tiles_d) * MT;
    n = (int)(t / tiles_d);
  };

  if (tid == 0) {
    for (int i = 0; i < 2 * kPMaxStages + 5; ++i) {
      const bool epi = i == 2 * kPMaxStages + 2 || i == 2 * kPMaxStages + 3;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar0 + 8u * i),
                   "r"(epi ? 128 : 1)
                   : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    fail_s = 0;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(P::kAlloc)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  auto failed = [&]() { return *(volatile int*)&fail_s != 0; };
  auto give_up = [&]() { atomicExch(&fail_s, 1); };

  if (tid == 0) {
    // ---- producer
    long long q = 0;
    if (RW) {
      mbar_expect_tx(wbar, (uint32_t)(nch * P::kWBytes));
      for (int ch = 0; ch < nch; ++ch)
        tma_load_4d(wreg + (uint32_t)(ch * P::kWBytes), &map_w, wbar, 0, 0, 2 * ch, 0);
    }
    for (long long t = blockIdx.x; t < tiles && !failed(); t += gridDim.x) {
      int w0, h0, d0, n;
      tile_origin(t, w0, h0, d0, n);
      for (int ch = 0; ch < nch; ++ch, ++q) {
        const int st = (int)(q % S);
        if (q >= S && !mbar_wait(empty(st), (uint32_t)((q / S - 1) & 1))) {
          give_up();
          break;
        }
        const uint32_t halo = base + (uint32_t)(st * P::kStage);
        const bool first = ch * 16 < a.C1;
        const CUtensorMap* mx = first ? &map_x1 : &map_x2;
        const int c0 = first ? ch * 16 : ch * 16 - a.C1;
        mbar_expect_tx(full(st), (uint32_t)(P::kHaloTx + (RW ? 0 : P::kWBytes)));
        tma_load_5d(halo, mx, full(st), c0, w0 - 1, h0 - 1, d0 - 1, n);
        tma_load_5d(halo + P::kHalfBytes, mx, full(st), c0 + 8, w0 - 1, h0 - 1, d0 - 1, n);
        if (!RW) tma_load_4d(halo + 2u * P::kHalfBytes, &map_w, full(st), 0, 0, 2 * ch, 0);
      }
    }
    // copies still in flight (the last use of every stage), bounded
    const long long q0 = q - S < 0 ? 0 : q - S;
    for (long long p = q0; p < q; ++p) mbar_wait(full((int)(p % S)), (uint32_t)((p / S) & 1));
    if (RW) mbar_wait(wbar, 0);
  } else if (tid == 32) {
    // ---- MMA issue
    const uint32_t idesc = instr_desc(kMmaM, N);
    long long q = 0, done_q = -1;
    int lt = 0;
    bool ok = !RW || mbar_wait(wbar, 0);
    if (!ok) give_up();
    for (long long t = blockIdx.x; ok && t < tiles && !failed(); t += gridDim.x, ++lt) {
      const int b = lt & 1;
      if (lt >= 2 && !mbar_wait(acc_empty(b), (uint32_t)(((lt >> 1) - 1) & 1))) {
        give_up();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t acc = tmem + (uint32_t)(b * P::kAcc);
      for (int ch = 0; ch < nch; ++ch, ++q) {
        const int st = (int)(q % S);
        if (!mbar_wait(full(st), (uint32_t)((q / S) & 1))) {
          give_up();
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t halo = base + (uint32_t)(st * P::kStage);
        const uint32_t wsm = RW ? wreg + (uint32_t)(ch * P::kWBytes) : halo + 2u * P::kHalfBytes;
        conv_chunk_mmas<N, MT, P::kTile>(acc, halo, wsm, P::kHalfBytes, idesc, ch > 0);
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                empty(st))
            : "memory");
        done_q = q;
      }
      if (!ok) break;
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              acc_full(b))
          : "memory");
    }
    // MMAs still in flight (the last commit covers the earlier ones), bounded
    if (done_q >= 0) mbar_wait(empty((int)(done_q % S)), (uint32_t)((done_q / S) & 1));
  } else if (warp >= 2) {
    // ---- epilogue: TMEM lane quarter warp % 4, voxel m = lane of the tile
    const int m = (warp & 3) * 32 + lane;
    const bool leader = tid == 64;
    const int O2 = N - a.O1;
    unsigned char* stg_p = smem_raw + (stg - smem_u32(smem_raw));
    int lt = 0;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x, ++lt) {
      const int b = lt & 1;
      const bool got = mbar_wait(acc_full(b), (uint32_t)((lt >> 1) & 1));
      // the staging tile is free once the previous tile's stores have read it
      if (leader) asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
      // the four warps agree (barrier with an OR vote) on whether to go on
      uint32_t bad = (!got || failed()) ? 1u : 0u;
      asm volatile(
          "{\n.reg .pred pi, po;\nsetp.ne.u32 pi, %1, 0;\n"
          "bar.red.or.pred po, 1, 128, pi;\nselp.u32 %0, 1, 0, po;\n}\n"
          : "=r"(bad)
          : "r"(bad)
          : "memory");
      if (bad) {
        give_up();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll 1
      for (int s = 0; s < MT; ++s)
#pragma unroll 1
        for (int cb = 0; cb < N; cb += 16) {
          uint32_t r[16];
          const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) +
                                 (uint32_t)(b * P::kAcc + s * P::kTile + cb);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
              "%12,%13,%14,%15}, [%16];\n"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
          uint32_t pk[8];
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            const int co = cb + j;
            float v0 = __uint_as_float(r[j]), v1 = __uint_as_float(r[j + 1]);
            if (a.bias) {
              v0 += a.bias[co];
              v1 += a.bias[co + 1];
            }
            if (a.relu) {
              v0 = fmaxf(v0, 0.0f);
              v1 = fmaxf(v1, 0.0f);
            }
            const __nv_bfloat162 pr = __floats2bfloat162_rn(v0, v1);
            pk[j / 2] = *reinterpret_cast<const uint32_t*>(&pr);
          }
          uint4* d = cb < a.O1 ? reinterpret_cast<uint4*>(stg_p + ((s * kMmaM + m) * a.O1 + cb) * 2)
                               : reinterpret_cast<uint4*>(stg_p + MT * kMmaM * a.O1 * 2 +
                                                          ((s * kMmaM + m) * O2 + cb - a.O1) * 2);
          d[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
          d[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
      // the accumulator is free for the tile after next
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(acc_empty(b)) : "memory");
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      asm volatile("bar.sync 1, 128;\n" ::: "memory");
      if (leader) {
        int w0, h0, d0, n;
        tile_origin(t, w0, h0, d0, n);
        tma_store_5d(&map_y1, stg, a.Yo1, w0, h0, d0, n);
        if (O2 > 0) tma_store_5d(&map_y2, stg + (uint32_t)(MT * kMmaM * a.O1 * 2), a.Yo2, w0, h0, d0, n);
        asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
      }
    }
    if (leader) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
  }
  __syncwarp();
  __syncthreads();
  if (tid == 0 && fail_s) atomicExch(&g_conv_timeout, 1u);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(P::kAlloc)
                 : "memory");
}

// Weight gradient dW[co][t][ci] += sum_v dY[v][co] X[v + off(t)][ci] on the
// tensor cores.  GEMM rows are (tap, 16-channel input group) pairs, 8 such
// atoms (128 rows) per M-tile; N = Cout; K runs over voxels, 128 per stage
// (a box of 8 x 4 x 4 voxels).  Both operands are MN-major in shared memory
// with the 32-byte swizzle: the tiled tensor copy of one 16-channel box,
// written with that swizzle, is [voxel][16 channels] = one atom of the
// canonical layout (8-voxel K groups of 256 bytes one after another, so sbo =
// 256 B; atoms one box apart, lbo = 4 KB), and every copied piece is a whole
// 32-byte sector.  The input box of atom (t, c) is the output box shifted by
// tap t's offset; zero fill at the volume's edge is the convolution's
// padding, and voxels of a box beyond the volume carry a zero dY.  A CTA
// accumulates its range of boxes in TMEM and adds the result to dW with FP32
// atomics.  With db given, the last M-tile's first unused atom holds BF16
// ones, so its rows accumulate db[co] += sum_v dY[v][co].  Producer / MMA /
// epilogue roles and bounded waits as in k_conv3d.
constexpr int kWgBX = 8, kWgBY = 4, kWgBZ = 4;         // voxel box of one stage
constexpr int kWgKV = kWgBX * kWgBY * kWgBZ;           // K per stage (128)
constexpr int kWgAtoms = 8;                            // 16-row atoms per M-tile

template <int N>
struct WgPlan {
  static constexpr int kAtomBytes = kWgKV * 32;         // one 16-channel box (4 KB)
  static constexpr int kABytes = kWgAtoms * kAtomBytes;
  static constexpr int kStage = kABytes + N / 16 * kAtomBytes;
  static constexpr int smem(int stages) { return stages * kStage + 1024; }
  static constexpr int kAlloc = N <= 32 ? 32 : N <= 64 ? 64 : 128;
};

// Shared-memory descriptor of an MN-major operand with the 32-byte swizzle
// (layout type 6 in bits 61-63): lbo = distance between 16-element atoms,
// sbo = between 8-row groups along K.
__device__ __forceinline__ uint64_t smem_desc_sw32(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return smem_desc(addr, lbo, sbo) | (6ull << 61);
}

struct WgArgs {
  int C1, C2, N, D, H, W;
  float* dw;
  float* db;     // nullable
  int splits;    // CTAs sharing an M-tile (voxel ranges)
};

template <int N>
__global__ void __launch_bounds__(kConvThreads)
    k_wgrad_tc(WgArgs a, const __grid_constant__ CUtensorMap map_x1,
               const __grid_constant__ CUtensorMap map_x2,
               const __grid_constant__ CUtensorMap map_dy, int S) {
  using P = WgPlan<N>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[2 * kMaxStages + 1];
  __shared__ uint32_t tmem_slot;
  __shared__ int issued_s, committed_s, fail_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ci_total = a.C1 + a.C2, c16 = ci_total / 16;
  const int atoms = 27 * c16;
  const int g0 = blockIdx.y * kWgAtoms;
  const int ng = max(0, min(kWgAtoms, atoms - g0));
  const int bias_g = (a.db && ng < kWgAtoms) ? ng : -1;  // the atom of ones
  const int nbx = (a.W + kWgBX - 1) / kWgBX, nby = (a.H + kWgBY - 1) / kWgBY,
            nbz = (a.D + kWgBZ - 1) / kWgBZ;
  const long long nboxes = (long long)a.N * nbz * nby * nbx;
  const long long per = (nboxes + a.splits - 1) / a.splits;
  const long long b0 = blockIdx.x * per;
  const int nk = (int)max(0ll, min(nboxes, b0 + per) - b0);
  if (nk == 0) return;  // uniform over the CTA
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t bar0 = smem_u32(&bars[0]);
  auto full = [&](int st) { return bar0 + 8u * (uint32_t)st; };
  auto empty = [&](int st) { return bar0 + 8u * (uint32_t)(kMaxStages + st); };
  const uint32_t done_bar = bar0 + 8u * (uint32_t)(2 * kMaxStages);

  if (bias_g >= 0) {
    // the ones group of every stage (never written by the copies)
    unsigned char* sm = smem_raw + (base - smem_u32(smem_raw));
    const uint4 ones = make_uint4(0x3f803f80u, 0x3f803f80u, 0x3f803f80u, 0x3f803f80u);
    for (int q = tid; q < S * (P::kAtomBytes / 16); q += kConvThreads) {
      const int st = q / (P::kAtomBytes / 16), e = q % (P::kAtomBytes / 16);
      *reinterpret_cast<uint4*>(sm + st * P::kStage + bias_g * P::kAtomBytes + e * 16) = ones;
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < 2 * kMaxStages + 1; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0 + 8u * i) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    issued_s = 0;
    committed_s = 0;
    fail_s = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(P::kAlloc)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (tid == 0) {
    // producer
    for (int i = 0; i < nk; ++i) {
      const int st = i % S;
      if (i >= S && !mbar_wait(empty(st), (uint32_t)((i / S - 1) & 1))) {
        atomicExch(&fail_s, 1);
        break;
      }
      if (*(volatile int*)&fail_s) break;
      long long b = b0 + i;
      const int x0 = (int)(b % nbx) * kWgBX;
      b /= nbx;
      const int y0 = (int)(b % nby) * kWgBY;
      b /= nby;
      const int z0 = (int)(b % nbz) * kWgBZ;
      const int n = (int)(b / nbz);
      const uint32_t stage = base + (uint32_t)(st * P::kStage);
      mbar_expect_tx(full(st), (uint32_t)((ng + N / 16) * P::kAtomBytes));
      for (int g = 0; g < ng; ++g) {
        const int G = g0 + g, t = G / c16, ch = (G % c16) * 16;
        const int kw = t % 3, kh = (t / 3) % 3, kd = t / 9;
        const bool first = ch < a.C1;
        tma_load_5d(stage + (uint32_t)(g * P::kAtomBytes), first ? &map_x1 : &map_x2, full(st),
                    first ? ch : ch - a.C1, x0 + kw - 1, y0 + kh - 1, z0 + kd - 1, n);
      }
      for (int j = 0; j < N / 16; ++j)
        tma_load_5d(stage + (uint32_t)(P::kABytes + j * P::kAtomBytes), &map_dy, full(st),
                    16 * j, x0, y0, z0, n);
      issued_s = i + 1;
    }
  } else if (tid == 32) {
    // MMA issue: both operands MN-major (instruction descriptor bits 15, 16)
    const uint32_t idesc = instr_desc(kMmaM, N) | (1u << 15) | (1u << 16);
    for (int i = 0; i < nk; ++i) {
      const int st = i % S;
      if (!mbar_wait(full(st), (uint32_t)((i / S) & 1))) {
        atomicExch(&fail_s, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t stage = base + (uint32_t)(st * P::kStage);
      // 16 voxels (two 256-byte K groups = 32 descriptor units) per MMA
      const uint64_t a0 = smem_desc_sw32(stage, P::kAtomBytes, 256);
      const uint64_t b0 = smem_desc_sw32(stage + P::kABytes, P::kAtomBytes, 256);
#pragma unroll
      for (int kk = 0; kk < kWgKV / 16; ++kk)
        mma_f16(tmem, a0 + (uint64_t)(32 * kk), b0 + (uint64_t)(32 * kk), idesc,
                (i > 0 || kk > 0) ? 1u : 0u);
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              empty(st))
          : "memory");
      committed_s = i + 1;
    }
    if (!*(volatile int*)&fail_s)
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              done_bar)
          : "memory");
  }
  __syncwarp();
  bool ok = !*(volatile int*)&fail_s && mbar_wait(done_bar, 0);
  ok = __syncthreads_and(ok) && !fail_s;
  if (!ok && tid == 0) {
    atomicExch(&g_conv_timeout, 1u);
    for (int i = issued_s - S < 0 ? 0 : issued_s - S; i < issued_s; ++i)
      mbar_wait(full(i % S), (uint32_t)((i / S) & 1));
    if (committed_s > 0)
      mbar_wait(empty((committed_s - 1) % S), (uint32_t)(((committed_s - 1) / S) & 1));
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

  if (ok) {
    // epilogue: TMEM lane r = row (atom r / 16, channel r % 16 of the atom)
    const int r = warp * 32 + lane, g = r / 16;
    const int G = g0 + g, t = G / c16, ci = (G % c16) * 16 + r % 16;
    const bool wrow = g < ng, brow = g == bias_g && r % 16 == 0;
#pragma unroll 1
    for (int cb = 0; cb < N; cb += 16) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
          "%12,%13,%14,%15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
            "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
            "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (wrow)
#pragma unroll
        for (int j = 0; j < 16; ++j)
          atomicAdd(&a.dw[((long long)(cb + j) * 27 + t) * ci_total + ci], __uint_as_float(v[j]));
      if (brow)
#pragma unroll
        for (int j = 0; j < 16; ++j) atomicAdd(&a.db[cb + j], __uint_as_float(v[j]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(P::kAlloc)
                 : "memory");
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

bool conv_supported(int cin_total, int cout) {
  return cin_total % 16 == 0 && cin_total > 0 &&
         (cout == 16 || cout == 32 || cout == 48 || cout == 64 || cout == 96);
}

// cuTensorMapEncodeTiled, fetched from the driver once.
static PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// Halo map of a channels-last activation [n][d][h][w][c]: dims (c, w, h, d, n),
// box (8 channels, HW, HH, mt + 2, 1), zero fill outside.
static bool halo_map(CUtensorMap* m, const __nv_bfloat16* x, int c, const ConvArgs& a, int mt) {
  const cuuint64_t dim[5] = {(cuuint64_t)c, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.D,
                             (cuuint64_t)a.N};
  const cuuint64_t row = (cuuint64_t)c * 2;
  const cuuint64_t stride[4] = {row, row * a.W, row * a.W * a.H, row * a.W * a.H * a.D};
  const cuuint32_t box[5] = {8, HW, HH, (cuuint32_t)(mt + 2), 1};
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  return encode_tiled()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void*)x, dim, stride, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Output map of a channels-last tensor with ys channels per voxel, written
// o channels at a time: box (o, TW, TH, mt, 1).
static bool out_map(CUtensorMap* m, const __nv_bfloat16* y, int ys, int o, const ConvArgs& a,
                    int mt) {
  const cuuint64_t dim[5] = {(cuuint64_t)ys, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.D,
                             (cuuint64_t)a.N};
  const cuuint64_t row = (cuuint64_t)ys * 2;
  const cuuint64_t stride[4] = {row, row * a.W, row * a.W * a.H, row * a.W * a.H * a.D};
  const cuuint32_t box[5] = {(cuuint32_t)o, TW, TH, (cuuint32_t)mt, 1};
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  return encode_tiled()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void*)y, dim, stride, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Weight map of w[co][tap][ci] seen as (8 channels, co, ci / 8, tap) with
// strides (2 B, 27 Ct x 2 B, 16 B, Ct x 2 B): the box (8, cout, 2, 27) at
// (0, 0, 2 chunk, 0) lands in shared memory as [tap][half][co] x 16 B.
static bool weight_map(CUtensorMap* m, const __nv_bfloat16* w, int ct, int cout) {
  const cuuint64_t dim[4] = {8, (cuuint64_t)cout, (cuuint64_t)(ct / 8), 27};
  const cuuint64_t stride[3] = {(cuuint64_t)27 * ct * 2, 16, (cuuint64_t)ct * 2};
  const cuuint32_t box[4] = {8, (cuuint32_t)cout, 2, 27};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return encode_tiled()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)w, dim, stride, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The persistent kernel on one CTA per SM (the occupancy query allows more
// only where the shared memory does), with as many stages (2 .. 4) as fit.
template <int N, bool RW>
static cudaError_t launch_conv3d_p(const ConvArgs& a, const CUtensorMap& mx1,
                                   const CUtensorMap& mx2, const CUtensorMap& mw,
                                   const CUtensorMap& my1, const CUtensorMap& my2,
                                   long long tiles, cudaStream_t s) {
  using P = PPlan<N, RW>;
  constexpr int kDyn = 227 * 1024 - 2048;  // opt-in limit less the kernel's static shared memory
  const int nch = (a.C1 + a.C2) / 16;
  // as many stages as fit one CTA per SM (two CTAs per SM with fewer stages
  // each measured the same)
  int S = kPMaxStages;
  while (S > 2 && P::smem(S, nch) > kDyn) --S;
  if (P::smem(S, nch) > kDyn) return cudaErrorNotSupported;
  static bool attr_done = false;
  if (!attr_done) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_conv3d_p<N, RW>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDyn);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  int dev = 0, nsm = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_conv3d_p<N, RW>, kPThreads,
                                                      P::smem(S, nch));
  if (e != cudaSuccess) return e;
  if (nsm < 1) return cudaErrorInvalidDevice;
  occ = std::max(1, std::min(occ, 512 / P::kAlloc));  // TMEM columns of an SM
  const long long grid = std::min<long long>(tiles, (long long)nsm * occ);
  k_conv3d_p<N, RW><<<(unsigned)grid, kPThreads, P::smem(S, nch), s>>>(a, mx1, mx2, mw, my1, my2,
                                                                       S);
  add_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_conv3d(const ConvArgs& a, int cout, cudaStream_t s) {
  const int ct = a.C1 + a.C2;
  if (!conv_supported(ct, cout) || a.C1 % 16 || a.C2 % 16 || a.C1 <= 0 ||
      ((uintptr_t)a.x1 | (uintptr_t)a.x2 | (uintptr_t)a.w) % 16)
    return cudaErrorInvalidValue;
  if (!encode_tiled()) return cudaErrorNotSupported;
  // two M-tiles per CTA when that still gives two waves of CTAs on 152 SMs
  const long long plane = (long long)a.N * ((a.H + TH - 1) / TH) * ((a.W + TW - 1) / TW);
  const int mt = plane * ((a.D + 1) / 2) >= 2 * 152 ? 2 : 1;
  const long long tiles = plane * ((a.D + mt - 1) / mt);
  CUtensorMap mx1, mx2, mw;
  if (!halo_map(&mx1, a.x1, a.C1, a, mt) ||
      (a.C2 > 0 ? !halo_map(&mx2, a.x2, a.C2, a, mt) : false) || !weight_map(&mw, a.w, ct, cout))
    return cudaErrorInvalidValue;
  if (a.C2 == 0) mx2 = mx1;
  // output maps: channel slices [Yo, Yo + O) of tensors with Ys channels
  const int O2 = cout - a.O1;
  auto slice_ok = [](const void* p, int ys, int yo, int o) {
    return p && (uintptr_t)p % 16 == 0 && ys % 8 == 0 && yo % 8 == 0 && o % 16 == 0 && o > 0 &&
           yo + o <= ys;
  };
  int tma_out = slice_ok(a.y1, a.Ys1, a.Yo1, a.O1) && (O2 == 0 || slice_ok(a.y2, a.Ys2, a.Yo2, O2));
  CUtensorMap my1 = mx1, my2 = mx1;
  if (tma_out && (!out_map(&my1, a.y1, a.Ys1, a.O1, a, mt) ||
                  (O2 > 0 && !out_map(&my2, a.y2, a.Ys2, O2, a, mt))))
    tma_out = 0;
  // large grids: the persistent kernel (its configuration fits for Cout <= 64;
  // the wait self-check runs on the tile kernel)
  if (mt == 2 && tma_out && cout <= 64 && a.stall_bytes == 0) {
    const int nch = ct / 16;
    const bool rw = 27 * 2 * cout * 16 * nch <= 64 * 1024;
    cudaError_t e = cudaErrorInvalidValue;
    switch (cout * 2 + (rw ? 1 : 0)) {
      case 32: e = launch_conv3d_p<16, false>(a, mx1, mx2, mw, my1, my2, tiles, s); break;
      case 33: e = launch_conv3d_p<16, true>(a, mx1, mx2, mw, my1, my2, tiles, s); break;
      case 64: e = launch_conv3d_p<32, false>(a, mx1, mx2, mw, my1, my2, tiles, s); break;
      case 65: e = launch_conv3d_p<32, true>(a, mx1, mx2, mw, my1, my2, tiles, s); break;
      case 96: e = launch_conv3d_p<48, false>(a, mx1, mx2, mw, my1, my2, tiles, s); break;
      case 97: e = launch_conv3d_p<48, true>(a, mx1, mx2, mw, my1, my2, tiles, s); break;
      case 128: e = launch_conv3d_p<64, false>(a, mx1, mx2, mw, my1, my2, tiles, s); break;
      case 129: e = launch_conv3d_p<64, true>(a, mx1, mx2, mw, my1, my2, tiles, s); break;
    }
    if (e != cudaErrorNotSupported) return e;  // NotSupported: no stage count fits
  }
  // one stage once the CTAs fill the SMs twice, else two (when there are
  // two chunks)
  const int stages = tiles >= 2 * 152 || ct == 16 ? 1 : 2;
  static bool attr_done[2][5] = {};
  auto go = [&](auto kernel, auto plan, int slot) {
    using P = decltype(plan);
    static_assert(P::smem(kMaxStages) <= 227 * 1024 - 1024, "two stages fit");
    if (!attr_done[mt - 1][slot]) {
      if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               P::smem(kMaxStages)) != cudaSuccess)
        return;  // the launch below is skipped; cudaGetLastError reports the failure
      attr_done[mt - 1][slot] = true;
    }
    kernel<<<(unsigned)tiles, kConvThreads, P::smem(stages), s>>>(a, mx1, mx2, mw, my1, my2, stages,
                                                                  tma_out);
  };
#define CONV_CASE(C, SLOT)                                                   \
  case C:                                                                    \
    if (mt == 2)                                                             \
      go(k_conv3d<C, 2>, ConvPlan<C, 2>{}, SLOT);                            \
    else                                                                     \
      go(k_conv3d<C, 1>, ConvPlan<C, 1>{}, SLOT);                            \
    break;
  switch (cout) {
    CONV_CASE(16, 0)
    CONV_CASE(32, 1)
    CONV_CASE(48, 2)
    CONV_CASE(64, 3)
    CONV_CASE(96, 4)
    default: return cudaErrorInvalidValue;
  }
#undef CONV_CASE
  add_launches(1);
  return cudaGetLastError();
}

bool conv_timed_out() {
  unsigned v = 0;
  cudaMemcpyFromSymbol(&v, g_conv_timeout, sizeof(v));
  if (v) {
    const unsigned zero = 0;
    cudaMemcpyToSymbol(g_conv_timeout, &zero, sizeof(zero));
  }
  return v != 0;
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

// Map of a channels-last tensor [n][d][h][w][c] for the weight gradient:
// box (16 channels, 8, 4, 4 voxels, 1) written with the 32-byte swizzle,
// zero fill outside.
static bool wg_map(CUtensorMap* m, const __nv_bfloat16* x, int c, int N, int D, int H, int W) {
  const cuuint64_t dim[5] = {(cuuint64_t)c, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D,
                             (cuuint64_t)N};
  const cuuint64_t row = (cuuint64_t)c * 2;
  const cuuint64_t stride[4] = {row, row * W, row * W * H, row * W * H * D};
  const cuuint32_t box[5] = {16, kWgBX, kWgBY, kWgBZ, 1};
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  return encode_tiled()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void*)x, dim, stride, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_wgrad(const __nv_bfloat16* dy, int co, const __nv_bfloat16* x1, int c1,
                         const __nv_bfloat16* x2, int c2, int N, int D, int H, int W, float* dw,
                         float* db, cudaStream_t s) {
  const int ci = c1 + c2;
  if (!conv_supported(ci, co) || c1 % 16 || c2 % 16 || c1 <= 0 ||
      ((uintptr_t)dy | (uintptr_t)x1 | (uintptr_t)x2) % 16)
    return cudaErrorInvalidValue;
  if (!encode_tiled()) return cudaErrorNotSupported;
  CUtensorMap mx1, mx2, mdy;
  if (!wg_map(&mx1, x1, c1, N, D, H, W) || (c2 > 0 && !wg_map(&mx2, x2, c2, N, D, H, W)) ||
      !wg_map(&mdy, dy, co, N, D, H, W))
    return cudaErrorInvalidValue;
  if (c2 == 0) mx2 = mx1;
  // with db, one atom more: the ones (an extra M-tile when the last is full)
  const int mtiles = (27 * ci / 16 + (db ? 1 : 0) + kWgAtoms - 1) / kWgAtoms;
  const long long nboxes = (long long)N * ((D + kWgBZ - 1) / kWgBZ) *
                           ((H + kWgBY - 1) / kWgBY) * ((W + kWgBX - 1) / kWgBX);
  // about two CTAs per SM in one wave, each over a contiguous range of boxes
  WgArgs a{c1, c2, N, D, H, W, dw, db, 1};
  a.splits = (int)std::max<long long>(1, std::min<long long>(nboxes, (2 * 152 + mtiles - 1) / mtiles));
  const int stages = 2;
  static bool attr_done[5] = {};
  auto go = [&](auto kernel, auto plan, int slot) {
    using P = decltype(plan);
    static_assert(P::smem(kMaxStages) <= 227 * 1024 - 1024, "two stages fit");
    if (!attr_done[slot]) {
      if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               P::smem(kMaxStages)) != cudaSuccess)
        return;  // the launch below is skipped; cudaGetLastError reports the failure
      attr_done[slot] = true;
    }
    kernel<<<dim3((unsigned)a.splits, (unsigned)mtiles), kConvThreads, P::smem(stages), s>>>(
        a, mx1, mx2, mdy, stages);
  };
  switch (co) {
    case 16: go(k_wgrad_tc<16>, WgPlan<16>{}, 0); break;
    case 32: go(k_wgrad_tc<32>, WgPlan<32>{}, 1); break;
    case 48: go(k_wgrad_tc<48>, WgPlan<48>{}, 2); break;
    case 64: go(k_wgrad_tc<64>, WgPlan<64>{}, 3); break;
    case 96: go(k_wgrad_tc<96>, WgPlan<96>{}, 4); break;
    default: return cudaErrorInvalidValue;
  }
  add_launches(1);
  return cudaGetLastError();
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
