// The warm-start U-Net: 4 levels (16/32/48/64 channels), two 3x3x3 convs with
// ReLU per level, 2x average pooling down, nearest 2x upsampling followed by a
// 3x3x3 conv up, skip connections by channel concatenation, 1x1x1 head to one
// channel.  It predicts (phi_n - phi_{n-1}) * s_out from the packed input
// (rho_n * s_rho, phi_{n-1} * s_phi) (channels 2..15 of the input are zero).
//
// Forward, backward (input and weight gradients), MSE loss and Adam all run
// in this library's kernels (nn_kernels.cu); this file only sequences them.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "../../include/mg.h"
#include "nn_internal.h"

namespace {

using bf16 = __nv_bfloat16;
using namespace mg::nn;

constexpr int kChan[4] = {16, 32, 48, 64};
constexpr unsigned kMagic = 0x4d47554eu;  // file tag
constexpr unsigned kVersion = 1;

struct Conv {
  int cin1, cin2, cout;  // input = concat(cin1, cin2)
  float *w32 = nullptr, *b = nullptr, *dw = nullptr, *db = nullptr;
  float *mw = nullptr, *vw = nullptr, *mb = nullptr, *vb = nullptr;
  bf16 *w16 = nullptr, *wflip = nullptr;
  long long nw() const { return (long long)cout * 27 * (cin1 + cin2); }
};

// activations of one forward pass (for a given N, D, H, W)
struct Acts {
  int N = 0, D = 0, H = 0, W = 0;
  std::vector<void*> bufs;
  // level tensors (BF16, channels-last)
  bf16* x = nullptr;                 // input, 16 channels, level 0
  bf16 *a[4] = {}, *e[4] = {};       // first conv / second conv (skip) per level
  bf16 *p[3] = {};                   // pooled e[l] (level l+1 size, kChan[l] ch)
  bf16 *u[3] = {}, *uc[3] = {};      // upsampled (level l size, kChan[l+1] ch), up-conv out
  bf16 *da[3] = {}, *d[3] = {};      // decoder convs per level l = 0..2
  float *out = nullptr, *tgt = nullptr, *g = nullptr, *loss = nullptr;
  // gradients (same shapes)
  bf16 *gx = nullptr, *ga[4] = {}, *ge[4] = {}, *gp[3] = {}, *gu[3] = {}, *guc[3] = {},
       *gda[3] = {}, *gd[3] = {};
  long long vox(int l) const { return (long long)N * (D >> l) * (H >> l) * (W >> l); }
};

}  // namespace

struct mg_unet {
  // layers: enc[l][0..1], up[l] (l = 0..2 conv after upsampling to level l),
  // dec[l][0..1] (l = 0..2)
  Conv enc[4][2], up[3], dec[3][2];
  float *hw = nullptr, *hb = nullptr, *dhw = nullptr, *dhb = nullptr;  // 1x1x1 head
  float *mhw = nullptr, *vhw = nullptr, *mhb = nullptr, *vhb = nullptr;
  double s_rho = 1.0, s_phi = 1.0, s_out = 1.0;
  int step = 0;
  Acts act;
  std::vector<void*> allocs;
  std::string err;
};

namespace {

thread_local std::string g_nn_err;

mg_status nn_fail(mg_status st, const std::string& m) {
  g_nn_err = m;
  mg::set_last_error(m);
  return st;
}

#define NN_CUDA(call)                                                                 \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return nn_fail(e_ == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA,      \
                     std::string(#call) + ": " + cudaGetErrorString(e_));             \
  } while (0)

#define NN_TRY(x)                \
  do {                           \
    mg_status s_ = (x);          \
    if (s_ != MG_OK) return s_;  \
  } while (0)

template <class T>
mg_status dalloc(std::vector<void*>& list, T** p, size_t n, bool zero = true) {
  *p = nullptr;
  if (n == 0) return MG_OK;
  NN_CUDA(cudaMalloc((void**)p, n * sizeof(T)));
  list.push_back(*p);
  if (zero) NN_CUDA(cudaMemset(*p, 0, n * sizeof(T)));
  return MG_OK;
}

mg_status init_conv(mg_unet* u, Conv& c, int cin1, int cin2, int cout, std::mt19937_64& rng,
                    int fan_in_channels) {
  c.cin1 = cin1;
  c.cin2 = cin2;
  c.cout = cout;
  const long long n = c.nw();
  NN_TRY(dalloc(u->allocs, &c.w32, n));
  NN_TRY(dalloc(u->allocs, &c.dw, n));
  NN_TRY(dalloc(u->allocs, &c.mw, n));
  NN_TRY(dalloc(u->allocs, &c.vw, n));
  NN_TRY(dalloc(u->allocs, &c.w16, n));
  NN_TRY(dalloc(u->allocs, &c.wflip, n));
  NN_TRY(dalloc(u->allocs, &c.b, cout));
  NN_TRY(dalloc(u->allocs, &c.db, cout));
  NN_TRY(dalloc(u->allocs, &c.mb, cout));
  NN_TRY(dalloc(u->allocs, &c.vb, cout));
  // He-normal initialisation over the real input channels
  std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / (27.0 * fan_in_channels)));
  std::vector<float> h(n);
  const int ci = cin1 + cin2;
  for (long long q = 0; q < n; ++q) {
    const int c_in = (int)(q % ci);
    h[q] = c_in < fan_in_channels || cin1 != 16 || fan_in_channels == ci ? (float)nd(rng) : 0.0f;
  }
  NN_CUDA(cudaMemcpy(c.w32, h.data(), n * sizeof(float), cudaMemcpyHostToDevice));
  return MG_OK;
}

void refresh_bf16(Conv& c, cudaStream_t s) {
  launch_f32_to_bf16(c.w32, c.nw(), c.w16, s);
  launch_flip_weights(c.w16, c.cout, c.cin1 + c.cin2, c.wflip, s);
}

template <class F>
void for_each_conv(mg_unet* u, F f) {
  for (int l = 0; l < 4; ++l)
    for (int q = 0; q < 2; ++q) f(u->enc[l][q]);
  for (int l = 0; l < 3; ++l) {
    f(u->up[l]);
    f(u->dec[l][0]);
    f(u->dec[l][1]);
  }
}

mg_status ensure_acts(mg_unet* u, int N, int D, int H, int W) {
  Acts& A = u->act;
  if (A.N == N && A.D == D && A.H == H && A.W == W) return MG_OK;
  for (void* p : A.bufs) cudaFree(p);
  A = Acts();
  A.N = N;
  A.D = D;
  A.H = H;
  A.W = W;
  auto& L = A.bufs;
  NN_TRY(dalloc(L, &A.x, A.vox(0) * 16));
  NN_TRY(dalloc(L, &A.gx, A.vox(0) * 16));
  for (int l = 0; l < 4; ++l) {
    const long long n = A.vox(l) * kChan[l];
    NN_TRY(dalloc(L, &A.a[l], n));
    NN_TRY(dalloc(L, &A.e[l], n));
    NN_TRY(dalloc(L, &A.ga[l], n));
    NN_TRY(dalloc(L, &A.ge[l], n));
  }
  for (int l = 0; l < 3; ++l) {
    NN_TRY(dalloc(L, &A.p[l], A.vox(l + 1) * kChan[l]));
    NN_TRY(dalloc(L, &A.gp[l], A.vox(l + 1) * kChan[l]));
    NN_TRY(dalloc(L, &A.u[l], A.vox(l) * kChan[l + 1]));
    NN_TRY(dalloc(L, &A.gu[l], A.vox(l) * kChan[l + 1]));
    NN_TRY(dalloc(L, &A.uc[l], A.vox(l) * kChan[l]));
    NN_TRY(dalloc(L, &A.guc[l], A.vox(l) * kChan[l]));
    NN_TRY(dalloc(L, &A.da[l], A.vox(l) * kChan[l]));
    NN_TRY(dalloc(L, &A.gda[l], A.vox(l) * kChan[l]));
    NN_TRY(dalloc(L, &A.d[l], A.vox(l) * kChan[l]));
    NN_TRY(dalloc(L, &A.gd[l], A.vox(l) * kChan[l]));
  }
  NN_TRY(dalloc(L, &A.out, A.vox(0)));
  NN_TRY(dalloc(L, &A.tgt, A.vox(0)));
  NN_TRY(dalloc(L, &A.g, A.vox(0)));
  NN_TRY(dalloc(L, &A.loss, 1));
  return MG_OK;
}

// y = conv(concat(x1, x2)) with the layer's bias and ReLU
mg_status conv_fwd(const Conv& c, const bf16* x1, const bf16* x2, int N, int D, int H, int W,
                   bf16* y, cudaStream_t s) {
  ConvArgs a{};
  a.x1 = x1;
  a.C1 = c.cin1;
  a.x2 = x2;
  a.C2 = c.cin2;
  a.w = c.w16;
  a.bias = c.b;
  a.relu = 1;
  a.N = N;
  a.D = D;
  a.H = H;
  a.W = W;
  a.y1 = y;
  a.O1 = c.cout;
  a.Ys1 = c.cout;
  a.Yo1 = 0;
  NN_CUDA(launch_conv3d(a, c.cout, s));
  return MG_OK;
}

// Backward of y = relu(conv(concat(x1, x2))): gy is overwritten by the
// ReLU-masked gradient; weight and bias gradients accumulate; input
// gradients into g1 (cin1 channels) and g2 (cin2, may be null) unless both
// are null.
mg_status conv_bwd(Conv& c, const bf16* x1, const bf16* x2, const bf16* y, bf16* gy, bf16* g1,
                   bf16* g2, int N, int D, int H, int W, cudaStream_t s) {
  const long long nv = (long long)N * D * H * W;
  launch_relu_bwd(y, gy, nv * c.cout, s);
  NN_CUDA(launch_wgrad(gy, c.cout, x1, c.cin1, x2, c.cin2, N, D, H, W, c.dw, c.db, s));
  if (g1) {
    ConvArgs a{};
    a.x1 = gy;
    a.C1 = c.cout;
    a.x2 = nullptr;
    a.C2 = 0;
    a.w = c.wflip;
    a.bias = nullptr;
    a.relu = 0;
    a.N = N;
    a.D = D;
    a.H = H;
    a.W = W;
    a.y1 = g1;
    a.O1 = c.cin1;
    a.Ys1 = c.cin1;
    a.Yo1 = 0;
    a.y2 = g2;
    a.Ys2 = c.cin2;
    a.Yo2 = 0;
    NN_CUDA(launch_conv3d(a, c.cin1 + c.cin2, s));
  }
  return MG_OK;
}

mg_status forward(mg_unet* u, cudaStream_t s) {
  Acts& A = u->act;
  const int N = A.N;
  auto dims = [&](int l, int& d, int& h, int& w) {
    d = A.D >> l;
    h = A.H >> l;
    w = A.W >> l;
  };
  int d, h, w;
  const bf16* in = A.x;
  for (int l = 0; l < 4; ++l) {
    dims(l, d, h, w);
    NN_TRY(conv_fwd(u->enc[l][0], in, nullptr, N, d, h, w, A.a[l], s));
    NN_TRY(conv_fwd(u->enc[l][1], A.a[l], nullptr, N, d, h, w, A.e[l], s));
    if (l < 3) {
      launch_pool(A.e[l], N, d, h, w, kChan[l], A.p[l], s);
      in = A.p[l];
    }
  }
  const bf16* below = A.e[3];
  for (int l = 2; l >= 0; --l) {
    dims(l, d, h, w);
    launch_up(below, N, d, h, w, kChan[l + 1], A.u[l], s);
    NN_TRY(conv_fwd(u->up[l], A.u[l], nullptr, N, d, h, w, A.uc[l], s));
    NN_TRY(conv_fwd(u->dec[l][0], A.uc[l], A.e[l], N, d, h, w, A.da[l], s));
    NN_TRY(conv_fwd(u->dec[l][1], A.da[l], nullptr, N, d, h, w, A.d[l], s));
    below = A.d[l];
  }
  launch_head(A.d[0], kChan[0], u->hw, u->hb, A.vox(0), A.out, s);
  NN_CUDA(cudaGetLastError());
  return MG_OK;
}

mg_status backward(mg_unet* u, cudaStream_t s) {
  Acts& A = u->act;
  const int N = A.N;
  int d, h, w;
  auto dims = [&](int l) {
    d = A.D >> l;
    h = A.H >> l;
    w = A.W >> l;
  };
  launch_head_bwd(A.d[0], kChan[0], u->hw, A.g, A.vox(0), A.gd[0], u->dhw, u->dhb, s);
  // decoder, finest level first: level l+1's output gradient is complete once
  // level l has been processed (it comes from level l's upsampling)
  for (int l = 0; l < 3; ++l) {
    dims(l);
    NN_TRY(conv_bwd(u->dec[l][1], A.da[l], nullptr, A.d[l], A.gd[l], A.gda[l], nullptr, N, d, h,
                    w, s));
    // concat(uc, e): gradient of uc and the skip part of e's gradient
    NN_TRY(conv_bwd(u->dec[l][0], A.uc[l], A.e[l], A.da[l], A.gda[l], A.guc[l], A.ge[l], N, d, h,
                    w, s));
    NN_TRY(conv_bwd(u->up[l], A.u[l], nullptr, A.uc[l], A.guc[l], A.gu[l], nullptr, N, d, h, w,
                    s));
    // u[l] = upsample(d[l+1]) (e[3] for l = 2)
    launch_up_bwd(A.gu[l], N, d, h, w, kChan[l + 1], l < 2 ? A.gd[l + 1] : A.ge[3], s);
  }
  // encoder, coarsest level first
  for (int l = 3; l >= 0; --l) {
    dims(l);
    NN_TRY(conv_bwd(u->enc[l][1], A.a[l], nullptr, A.e[l], A.ge[l], A.ga[l], nullptr, N, d, h, w,
                    s));
    const bf16* in = l == 0 ? A.x : A.p[l - 1];
    NN_TRY(conv_bwd(u->enc[l][0], in, nullptr, A.a[l], A.ga[l], l == 0 ? nullptr : A.gp[l - 1],
                    nullptr, N, d, h, w, s));
    if (l > 0) {
      // p[l-1] = pool(e[l-1]): add to the skip gradient already in ge[l-1]
      launch_pool_bwd(A.gp[l - 1], N, A.D >> (l - 1), A.H >> (l - 1), A.W >> (l - 1),
                      kChan[l - 1], A.ge[l - 1], 1, s);
    }
  }
  NN_CUDA(cudaGetLastError());
  return MG_OK;
}

mg_status zero_grads(mg_unet* u, cudaStream_t s) {
  bool ok = true;
  for_each_conv(u, [&](Conv& c) {
    ok = ok && cudaMemsetAsync(c.dw, 0, c.nw() * sizeof(float), s) == cudaSuccess &&
         cudaMemsetAsync(c.db, 0, c.cout * sizeof(float), s) == cudaSuccess;
  });
  NN_CUDA(cudaMemsetAsync(u->dhw, 0, 16 * sizeof(float), s));
  NN_CUDA(cudaMemsetAsync(u->dhb, 0, sizeof(float), s));
  if (!ok) return nn_fail(MG_ERR_CUDA, "cudaMemsetAsync failed");
  return MG_OK;
}

mg_status check_dims(int n, int d, int h, int w) {
  if (n < 1 || d < 8 || h < 8 || w < 8 || d % 8 || h % 8 || w % 8)
    return nn_fail(MG_ERR_INVALID_ARG, "U-Net sizes must be multiples of 8 (three poolings)");
  return MG_OK;
}

// pack the input, run forward (and the loss against the target if phi != null)
mg_status run_forward(mg_unet* u, const double* rho, const double* prev, const double* phi,
                      int n, int d, int h, int w, cudaStream_t s) {
  NN_TRY(check_dims(n, d, h, w));
  NN_TRY(ensure_acts(u, n, d, h, w));
  Acts& A = u->act;
  const long long nv = A.vox(0);
  launch_pack_input(rho, u->s_rho, prev, u->s_phi, nv, A.x, s);
  NN_TRY(forward(u, s));
  if (phi) {
    launch_target(phi, prev, u->s_out, nv, A.tgt, s);
    NN_CUDA(cudaMemsetAsync(A.loss, 0, sizeof(float), s));
    launch_mse(A.out, A.tgt, nv, A.g, A.loss, s);
  }
  NN_CUDA(cudaGetLastError());
  return MG_OK;
}

mg_status create(unsigned long long seed, mg_unet** out) {
  mg_unet* u = new (std::nothrow) mg_unet;
  if (!u) return nn_fail(MG_ERR_OOM, "host allocation failed");
  *out = u;
  std::mt19937_64 rng(seed);
  for (int l = 0; l < 4; ++l) {
    const int cin = l == 0 ? 16 : kChan[l - 1];
    NN_TRY(init_conv(u, u->enc[l][0], cin, 0, kChan[l], rng, l == 0 ? 2 : cin));
    NN_TRY(init_conv(u, u->enc[l][1], kChan[l], 0, kChan[l], rng, kChan[l]));
  }
  for (int l = 0; l < 3; ++l) {
    NN_TRY(init_conv(u, u->up[l], kChan[l + 1], 0, kChan[l], rng, kChan[l + 1]));
    NN_TRY(init_conv(u, u->dec[l][0], kChan[l], kChan[l], kChan[l], rng, 2 * kChan[l]));
    NN_TRY(init_conv(u, u->dec[l][1], kChan[l], 0, kChan[l], rng, kChan[l]));
  }
  // the head starts at zero, so the untrained network predicts no change
  NN_TRY(dalloc(u->allocs, &u->hw, 16));
  NN_TRY(dalloc(u->allocs, &u->hb, 1));
  NN_TRY(dalloc(u->allocs, &u->dhw, 16));
  NN_TRY(dalloc(u->allocs, &u->dhb, 1));
  NN_TRY(dalloc(u->allocs, &u->mhw, 16));
  NN_TRY(dalloc(u->allocs, &u->vhw, 16));
  NN_TRY(dalloc(u->allocs, &u->mhb, 1));
  NN_TRY(dalloc(u->allocs, &u->vhb, 1));
  for_each_conv(u, [&](Conv& c) { refresh_bf16(c, nullptr); });
  NN_CUDA(cudaDeviceSynchronize());
  return MG_OK;
}

void destroy_unet(mg_unet* u) {
  if (!u) return;
  cudaDeviceSynchronize();
  for (void* p : u->act.bufs) cudaFree(p);
  for (void* p : u->allocs) cudaFree(p);
  delete u;
}

// parameters in a fixed order: every conv (w then b) in for_each_conv order,
// then the head (w[16], b)
template <class F>
void for_each_param(mg_unet* u, F f) {
  for_each_conv(u, [&](Conv& c) {
    f(c.w32, c.nw());
    f(c.b, (long long)c.cout);
  });
  f(u->hw, 16LL);
  f(u->hb, 1LL);
}

long long num_params(mg_unet* u) {
  long long n = 0;
  for_each_param(u, [&](float*, long long k) { n += k; });
  return n;
}

}  // namespace

extern "C" {

mg_status mg_unet_create(unsigned long long seed, mg_unet** out) {
  if (!out) return nn_fail(MG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  mg_unet* u = nullptr;
  const mg_status st = create(seed, &u);
  if (st != MG_OK) {
    destroy_unet(u);
    return st;
  }
  *out = u;
  return MG_OK;
}

void mg_unet_destroy(mg_unet* u) { destroy_unet(u); }

mg_status mg_unet_set_scales(mg_unet* u, double s_rho, double s_phi, double s_out) {
  if (!u || !(s_rho > 0) || !(s_phi > 0) || !(s_out > 0))
    return nn_fail(MG_ERR_INVALID_ARG, "scales must be > 0");
  u->s_rho = s_rho;
  u->s_phi = s_phi;
  u->s_out = s_out;
  return MG_OK;
}

mg_status mg_unet_get_scales(const mg_unet* u, double scales[3]) {
  if (!u || !scales) return nn_fail(MG_ERR_INVALID_ARG, "NULL argument");
  scales[0] = u->s_rho;
  scales[1] = u->s_phi;
  scales[2] = u->s_out;
  return MG_OK;
}

mg_status mg_unet_num_params(const mg_unet* u, long long* n) {
  if (!u || !n) return nn_fail(MG_ERR_INVALID_ARG, "NULL argument");
  *n = num_params(const_cast<mg_unet*>(u));
  return MG_OK;
}

mg_status mg_unet_get_params(const mg_unet* u, float* host) {
  if (!u || !host) return nn_fail(MG_ERR_INVALID_ARG, "NULL argument");
  NN_CUDA(cudaDeviceSynchronize());
  long long off = 0;
  cudaError_t e = cudaSuccess;
  for_each_param(const_cast<mg_unet*>(u), [&](float* p, long long k) {
    if (e == cudaSuccess) e = cudaMemcpy(host + off, p, k * sizeof(float), cudaMemcpyDeviceToHost);
    off += k;
  });
  NN_CUDA(e);
  return MG_OK;
}

mg_status mg_unet_set_params(mg_unet* u, const float* host) {
  if (!u || !host) return nn_fail(MG_ERR_INVALID_ARG, "NULL argument");
  long long off = 0;
  cudaError_t e = cudaSuccess;
  for_each_param(u, [&](float* p, long long k) {
    if (e == cudaSuccess) e = cudaMemcpy(p, host + off, k * sizeof(float), cudaMemcpyHostToDevice);
    off += k;
  });
  NN_CUDA(e);
  for_each_conv(u, [&](Conv& c) { refresh_bf16(c, nullptr); });
  NN_CUDA(cudaDeviceSynchronize());
  return MG_OK;
}

mg_status mg_unet_grads(mg_unet* u, const double* rho, const double* prev, const double* phi,
                        int n, int d, int h, int w, float* host_grads, float* loss) {
  if (!u || !rho || !prev || !phi || !host_grads)
    return nn_fail(MG_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = nullptr;
  NN_TRY(zero_grads(u, s));
  NN_TRY(run_forward(u, rho, prev, phi, n, d, h, w, s));
  NN_TRY(backward(u, s));
  NN_CUDA(cudaStreamSynchronize(s));
  if (conv_timed_out()) return nn_fail(MG_ERR_CUDA, "conv3d: a tensor-core completion wait gave up");
  long long off = 0;
  cudaError_t e = cudaSuccess;
  for_each_conv(u, [&](Conv& c) {
    if (e == cudaSuccess)
      e = cudaMemcpy(host_grads + off, c.dw, c.nw() * sizeof(float), cudaMemcpyDeviceToHost);
    off += c.nw();
    if (e == cudaSuccess)
      e = cudaMemcpy(host_grads + off, c.db, c.cout * sizeof(float), cudaMemcpyDeviceToHost);
    off += c.cout;
  });
  if (e == cudaSuccess)
    e = cudaMemcpy(host_grads + off, u->dhw, 16 * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(host_grads + off + 16, u->dhb, sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && loss)
    e = cudaMemcpy(loss, u->act.loss, sizeof(float), cudaMemcpyDeviceToHost);
  NN_CUDA(e);
  return MG_OK;
}

mg_status mg_unet_train_step(mg_unet* u, const double* rho, const double* prev, const double* phi,
                             int n, int d, int h, int w, float lr, float* loss,
                             void* cuda_stream) {
  if (!u || !rho || !prev || !phi || !(lr > 0)) return nn_fail(MG_ERR_INVALID_ARG, "bad argument");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  NN_TRY(zero_grads(u, s));
  NN_TRY(run_forward(u, rho, prev, phi, n, d, h, w, s));
  NN_TRY(backward(u, s));
  ++u->step;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for_each_conv(u, [&](Conv& c) {
    launch_adam(c.w32, c.mw, c.vw, c.dw, c.nw(), lr, b1, b2, eps, u->step, c.w16, s);
    launch_adam(c.b, c.mb, c.vb, c.db, c.cout, lr, b1, b2, eps, u->step, nullptr, s);
    launch_flip_weights(c.w16, c.cout, c.cin1 + c.cin2, c.wflip, s);
  });
  launch_adam(u->hw, u->mhw, u->vhw, u->dhw, 16, lr, b1, b2, eps, u->step, nullptr, s);
  launch_adam(u->hb, u->mhb, u->vhb, u->dhb, 1, lr, b1, b2, eps, u->step, nullptr, s);
  NN_CUDA(cudaGetLastError());
  if (loss) {
    NN_CUDA(cudaMemcpyAsync(loss, u->act.loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    NN_CUDA(cudaStreamSynchronize(s));
    if (conv_timed_out())
      return nn_fail(MG_ERR_CUDA, "conv3d: a tensor-core completion wait gave up");
  }
  return MG_OK;
}

mg_status mg_unet_predict(mg_unet* u, const double* rho, const double* prev, double* guess, int n,
                          int d, int h, int w, void* cuda_stream) {
  if (!u || !rho || !prev || !guess) return nn_fail(MG_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  NN_TRY(run_forward(u, rho, prev, nullptr, n, d, h, w, s));
  launch_apply_delta(prev, u->act.out, 1.0 / u->s_out, (long long)n * d * h * w, guess, s);
  NN_CUDA(cudaGetLastError());
  return MG_OK;
}

mg_status mg_unet_save(const mg_unet* u, const char* path) {
  if (!u || !path) return nn_fail(MG_ERR_INVALID_ARG, "NULL argument");
  mg_unet* m = const_cast<mg_unet*>(u);
  const long long np = num_params(m);
  std::vector<float> buf(np);
  NN_TRY(mg_unet_get_params(u, buf.data()));
  FILE* f = std::fopen(path, "wb");
  if (!f) return nn_fail(MG_ERR_INVALID_ARG, std::string("cannot write ") + path);
  const unsigned hdr[2] = {kMagic, kVersion};
  const double sc[3] = {u->s_rho, u->s_phi, u->s_out};
  bool ok = std::fwrite(hdr, sizeof hdr, 1, f) == 1 && std::fwrite(&np, sizeof np, 1, f) == 1 &&
            std::fwrite(sc, sizeof sc, 1, f) == 1 &&
            std::fwrite(buf.data(), sizeof(float), np, f) == (size_t)np;
  ok = std::fclose(f) == 0 && ok;
  if (!ok) return nn_fail(MG_ERR_INVALID_ARG, std::string("write failed: ") + path);
  return MG_OK;
}

mg_status mg_unet_load(mg_unet* u, const char* path) {
  if (!u || !path) return nn_fail(MG_ERR_INVALID_ARG, "NULL argument");
  FILE* f = std::fopen(path, "rb");
  if (!f) return nn_fail(MG_ERR_INVALID_ARG, std::string("cannot read ") + path);
  unsigned hdr[2] = {0, 0};
  long long np = 0;
  double sc[3] = {1, 1, 1};
  const long long want = num_params(u);
  bool ok = std::fread(hdr, sizeof hdr, 1, f) == 1 && hdr[0] == kMagic && hdr[1] == kVersion &&
            std::fread(&np, sizeof np, 1, f) == 1 && np == want &&
            std::fread(sc, sizeof sc, 1, f) == 1;
  std::vector<float> buf(ok ? np : 0);
  ok = ok && std::fread(buf.data(), sizeof(float), np, f) == (size_t)np;
  std::fclose(f);
  if (!ok) return nn_fail(MG_ERR_INVALID_ARG, std::string("not a U-Net weight file: ") + path);
  NN_TRY(mg_unet_set_params(u, buf.data()));
  u->s_rho = sc[0];
  u->s_phi = sc[1];
  u->s_out = sc[2];
  return MG_OK;
}

}  // extern "C"

// Argument checks and launch of one network convolution; stalled: the wait
// self-check (see mg_nn_conv3d_stalled).
static mg_status conv3d_entry(const void* x1, int c1, const void* x2, int c2, const void* w,
                              const float* bias, int relu, int cout, int n, int d, int h, int w_,
                              void* y, void* cuda_stream, bool stalled) {
  if (!x1 || !w || !y || (c2 > 0 && !x2)) return nn_fail(MG_ERR_INVALID_ARG, "NULL argument");
  if (!conv_supported(c1 + c2, cout) || c1 < 16 || c1 % 16 || c2 % 16 || n < 1 || d < 1 ||
      h < 1 || w_ < 1)
    return nn_fail(MG_ERR_UNSUPPORTED,
                   "conv3d: channels must be multiples of 16, cout in {16,32,48,64,96}");
  if (((uintptr_t)x1 | (uintptr_t)x2 | (uintptr_t)w) % 16)
    return nn_fail(MG_ERR_INVALID_ARG, "conv3d: x1, x2 and w must be 16-byte aligned");
  ConvArgs a{};
  a.x1 = (const bf16*)x1;
  a.C1 = c1;
  a.x2 = (const bf16*)x2;
  a.C2 = c2;
  a.w = (const bf16*)w;
  a.bias = bias;
  a.relu = relu;
  a.N = n;
  a.D = d;
  a.H = h;
  a.W = w_;
  a.y1 = (bf16*)y;
  a.O1 = cout;
  a.Ys1 = cout;
  if (stalled) {
    a.stall_bytes = 16;         // never delivered: the first chunk's wait must run out
    a.wait_ns = 50000000ull;    // after 50 ms
  }
  const cudaStream_t s = (cudaStream_t)cuda_stream;
  NN_CUDA(launch_conv3d(a, cout, s));
  if (stalled) {
    NN_CUDA(cudaStreamSynchronize(s));
    if (conv_timed_out())
      return nn_fail(MG_ERR_CUDA, "conv3d: a tensor-core completion wait gave up");
  }
  return MG_OK;
}

extern "C" {

mg_status mg_nn_conv3d(const void* x1, int c1, const void* x2, int c2, const void* w,
                       const float* bias, int relu, int cout, int n, int d, int h, int w_,
                       void* y, void* cuda_stream) {
  return conv3d_entry(x1, c1, x2, c2, w, bias, relu, cout, n, d, h, w_, y, cuda_stream, false);
}

mg_status mg_nn_conv3d_stalled(const void* x1, int c1, const void* x2, int c2, const void* w,
                               const float* bias, int relu, int cout, int n, int d, int h,
                               int w_, void* y, void* cuda_stream) {
  return conv3d_entry(x1, c1, x2, c2, w, bias, relu, cout, n, d, h, w_, y, cuda_stream, true);
}

mg_status mg_nn_conv3d_wgrad(const void* dy, int cout, const void* x1, int c1, const void* x2,
                             int c2, int n, int d, int h, int w, float* dw, float* db,
                             void* cuda_stream) {
  if (!dy || !x1 || !dw || (c2 > 0 && !x2)) return nn_fail(MG_ERR_INVALID_ARG, "NULL argument");
  if (!conv_supported(c1 + c2, cout) || c1 < 16 || c1 % 16 || c2 % 16 || n < 1 || d < 1 ||
      h < 1 || w < 1)
    return nn_fail(MG_ERR_UNSUPPORTED,
                   "conv3d_wgrad: channels must be multiples of 16, cout in {16,32,48,64,96}");
  if (((uintptr_t)dy | (uintptr_t)x1 | (uintptr_t)x2) % 16)
    return nn_fail(MG_ERR_INVALID_ARG, "conv3d_wgrad: dy, x1 and x2 must be 16-byte aligned");
  NN_CUDA(cudaMemsetAsync(dw, 0, (size_t)cout * 27 * (c1 + c2) * sizeof(float),
                          (cudaStream_t)cuda_stream));
  if (db) NN_CUDA(cudaMemsetAsync(db, 0, (size_t)cout * sizeof(float), (cudaStream_t)cuda_stream));
  NN_CUDA(launch_wgrad((const bf16*)dy, cout, (const bf16*)x1, c1, (const bf16*)x2, c2, n, d, h, w,
                       dw, db, (cudaStream_t)cuda_stream));
  return MG_OK;
}

}  // extern "C"
