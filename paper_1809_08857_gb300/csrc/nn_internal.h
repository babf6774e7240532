// Internal declarations of the U-Net kernels (nn_kernels.cu).  Not ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "mg_internal.h"

namespace mg {
namespace nn {

// 3x3x3 convolution, zero padding 1, stride 1, on channels-last BF16
// tensors.  Input = concat(x1 [.., C1], x2 [.., C2]) along channels (x2 may be
// null with C2 = 0); weights [Cout][27][C1 + C2].  Output channels [0, O1)
// go to y1[v * Ys1 + Yo1 + co], the rest to y2[v * Ys2 + Yo2 + co - O1].
struct ConvArgs {
  const __nv_bfloat16* x1;
  int C1;
  const __nv_bfloat16* x2;
  int C2;
  const __nv_bfloat16* w;
  const float* bias;  // nullable
  int relu;
  int N, D, H, W;
  __nv_bfloat16* y1;
  int O1;
  int Ys1, Yo1;
  __nv_bfloat16* y2;
  int Ys2, Yo2;
  // self-check of the bounded waits (0 in normal use): bytes added to the
  // first chunk's expected copy size, which the copies never deliver, and
  // the wait limit in ns (0: the default)
  unsigned stall_bytes;
  unsigned long long wait_ns;
};

bool conv_supported(int cin_total, int cout);
cudaError_t launch_conv3d(const ConvArgs& a, int cout, cudaStream_t s);
// True once any conv CTA gave up waiting for its tensor-core MMAs (a bounded
// wait; its outputs were not written).  Synchronises.
// Whether a tensor-core kernel gave up waiting since the last call (the flag
// is cleared by reading it).
bool conv_timed_out();
void launch_flip_weights(const __nv_bfloat16* w, int co, int ci, __nv_bfloat16* wt,
                         cudaStream_t s);
void launch_relu_bwd(const __nv_bfloat16* y, __nv_bfloat16* dy, long long n, cudaStream_t s);
void launch_pool(const __nv_bfloat16* x, int N, int D, int H, int W, int C, __nv_bfloat16* y,
                 cudaStream_t s);
// dx (+)= pool backward of dy; accumulate into dx when acc != 0
void launch_pool_bwd(const __nv_bfloat16* dy, int N, int D, int H, int W, int C,
                     __nv_bfloat16* dx, int acc, cudaStream_t s);
void launch_up(const __nv_bfloat16* x, int N, int D, int H, int W, int C, __nv_bfloat16* y,
               cudaStream_t s);
void launch_up_bwd(const __nv_bfloat16* dy, int N, int D, int H, int W, int C, __nv_bfloat16* dx,
                   cudaStream_t s);
// dw += weight gradient; db += bias gradient when db is not null.
cudaError_t launch_wgrad(const __nv_bfloat16* dy, int co, const __nv_bfloat16* x1, int c1,
                         const __nv_bfloat16* x2, int c2, int N, int D, int H, int W, float* dw,
                         float* db, cudaStream_t s);
void launch_head(const __nv_bfloat16* x, int C, const float* w, const float* b, long long nvox,
                 float* out, cudaStream_t s);
void launch_head_bwd(const __nv_bfloat16* x, int C, const float* w, const float* g,
                     long long nvox, __nv_bfloat16* dx, float* dw, float* db, cudaStream_t s);
void launch_mse(const float* p, const float* t, long long n, float* g, float* loss,
                cudaStream_t s);
void launch_adam(float* w, float* m, float* v, const float* g, long long n, float lr, float b1,
                 float b2, float eps, int step, __nv_bfloat16* w16, cudaStream_t s);
void launch_f32_to_bf16(const float* x, long long n, __nv_bfloat16* y, cudaStream_t s);
void launch_pack_input(const double* a, double sa, const double* b, double sb, long long nvox,
                       __nv_bfloat16* x, cudaStream_t s);
void launch_apply_delta(const double* prev, const float* delta, double scale, long long n,
                        double* out, cudaStream_t s);
// target delta: t[v] = (phi[v] - prev[v]) * scale (FP32)
void launch_target(const double* phi, const double* prev, double scale, long long n, float* t,
                   cudaStream_t s);

}  // namespace nn
}  // namespace mg
