// Tensor-memory-accelerator plumbing shared by the staged kernels of the
// multigrid path (the half-sweep in mg_split32.cu, the refinement pass in
// mg_ir.cu): tiled 3D copies global -> shared that complete on an mbarrier,
// bounded waits on those barriers, and host-side encoding of FP32 3D tensor
// maps.  A tiled copy's innermost start coordinate times the element size
// must be a multiple of 16 bytes (callers round x down and index from the
// remainder); coordinates outside the tensor read zeros.
#ifndef MG_TMA_CUH
#define MG_TMA_CUH

#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

namespace mg {
namespace tma {

constexpr unsigned long long kWaitNs = 1000000000ull;  // a wait gives up after 1 s
constexpr long long kWaitIters = 1ll << 24;            // or after this many tries

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void bar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
}

// makes the barrier initialisations visible to the copy engine
__device__ __forceinline__ void bar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// the phase completes with this arrival alone (a slot that gets no copy)
__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

// the phase completes with this arrival once `bytes` have been copied
__device__ __forceinline__ void bar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar),
               "r"(bytes)
               : "memory");
}

// one test of the phase with this parity (true once it has completed)
__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// true once the phase with this parity has completed; false after kWaitIters
// tries or kWaitNs nanoseconds.  The first test needs no clock (the copies
// are usually in by then).
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  if (bar_try(bar, parity)) return true;
  const unsigned long long t0 = now_ns();
  for (long long it = 1; it < kWaitIters; ++it) {
    if (bar_try(bar, parity)) return true;
    if ((it & 63) == 0 && now_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

// box of the map at (x, y, z) into shared memory at dst, completing on bar
__device__ __forceinline__ void load3(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x,
                                      int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y), "r"(z)
      : "memory");
}

}  // namespace tma

// Host side (defined in mg_split32.cu).  An FP32 array of nx x ny x nz
// (x fastest, rows of nx floats) as a 3D tensor copied in boxes of bx x by x bz
// with zero fill; false if the driver entry point is missing or the encoding
// is refused (the caller then runs its register-fed kernel).
bool tma_map_f32(CUtensorMap* m, const void* p, long long nx, long long ny, long long nz, int bx,
                 int by, int bz = 1);

}  // namespace mg

#endif
