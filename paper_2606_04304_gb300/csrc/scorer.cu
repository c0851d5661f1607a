// a13: learned candidate scorer (not in the paper; Section 2.4 keeps or drops
// triggers by threshold alone).  A multilayer perceptron 1600 -> 128 -> 32 -> 1
// with GELU hidden units scores 64-channel x 5 x 5-pixel cutouts of the
// high-passed standardised cube around a trigger.  Weights are served in BF16
// and every product is accumulated in FP32; training keeps FP32 master weights
// and Adam moments.  All kernels are plain SIMT: the contractions are small
// (a few hundred MFLOP per step) and memory/latency-bound at these sizes.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace ovro {
namespace {

constexpr int kIn = 1600, kH1 = 128, kH2 = 32;
constexpr int kCutCh = 64, kCutPix = 5;
constexpr int kNParams = kH1 * kIn + kH1 + kH2 * kH1 + kH2 + kH2 + 1;
// parameter offsets, layer by layer (W row-major [out][in], then b)
constexpr int kW1 = 0, kB1 = kW1 + kH1 * kIn, kW2 = kB1 + kH1, kB2 = kW2 + kH2 * kH1, kW3 = kB2 + kH2,
              kB3 = kW3 + kH2;

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

template <bool BF16>
__device__ __forceinline__ float ldw(const void* w, long long i) {
  if (BF16) return __bfloat162float(static_cast<const __nv_bfloat16*>(w)[i]);
  return static_cast<const float*>(w)[i];
}

// ---------------------------------------------------------------- cutouts
// x[t][i][dr][dc] = zp[k - 32 + i][r - 2 + dr][c - 2 + dc], 0 outside the
// trigger's coarse channel or the image.
__global__ void k_cutouts(const float* __restrict__ zp, int n_chan, int n, const int* __restrict__ chan0,
                          int n_coarse, const int* __restrict__ trig, int n_trig, float* __restrict__ x) {
  const long long total = static_cast<long long>(n_trig) * kIn;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int t = static_cast<int>(e / kIn);
    const int j = static_cast<int>(e - static_cast<long long>(t) * kIn);
    const int i = j / (kCutPix * kCutPix), rc = j - i * kCutPix * kCutPix;
    const int dr = rc / kCutPix, dc = rc - dr * kCutPix;
    const int k = trig[3 * t], r = trig[3 * t + 1], c = trig[3 * t + 2];
    int lo = 0, hi = n_chan;
    for (int q = 0; q < n_coarse; ++q)
      if (k >= chan0[q] && k < chan0[q + 1]) { lo = chan0[q]; hi = chan0[q + 1]; }
    const int kk = k - kCutCh / 2 + i, rr = r - kCutPix / 2 + dr, cc = c - kCutPix / 2 + dc;
    float v = 0.f;
    if (kk >= lo && kk < hi && rr >= 0 && rr < n && cc >= 0 && cc < n)
      v = zp[(static_cast<long long>(kk) * n + rr) * n + cc];
    x[e] = v;
  }
}

// ------------------------------------------------------------ dense layers
constexpr int kT = 32;

// y[b][o] = act(sum_i x[b][i] w[o][i] + bias[o]); z (optional) keeps the pre-activation
template <bool BF16>
__global__ void __launch_bounds__(256)
k_dense_fwd(const float* __restrict__ x, const void* __restrict__ w, int w_off, int b_off, int B, int in, int out,
            bool act, float* __restrict__ z, float* __restrict__ y) {
  __shared__ float xs[kT][kT + 1];
  __shared__ float ws[kT][kT + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;       // 32 x 8
  const int b0 = blockIdx.y * kT, o0 = blockIdx.x * kT;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < in; k0 += kT) {
    for (int r = ty; r < kT; r += 8) {
      const int b = b0 + r, k = k0 + tx;
      xs[r][tx] = (b < B && k < in) ? x[static_cast<long long>(b) * in + k] : 0.f;
      const int o = o0 + r;
      ws[r][tx] = (o < out && k < in) ? ldw<BF16>(w, w_off + static_cast<long long>(o) * in + k) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kT; ++k) {
      const float wv = ws[tx][k];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(xs[ty + 8 * q][k], wv, acc[q]);
    }
    __syncthreads();
  }
  const int o = o0 + tx;
  if (o >= out) return;
  const float bias = ldw<BF16>(w, b_off + o);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int b = b0 + ty + 8 * q;
    if (b >= B) continue;
    const float v = acc[q] + bias;
    if (z) z[static_cast<long long>(b) * out + o] = v;
    y[static_cast<long long>(b) * out + o] = act ? gelu(v) : v;
  }
}

// dx[b][i] = (sum_o dz[b][o] w[o][i]) * gelu'(zprev[b][i])
template <bool BF16>
__global__ void __launch_bounds__(256)
k_dense_bwd_x(const float* __restrict__ dz, const void* __restrict__ w, int w_off, int B, int in, int out,
              const float* __restrict__ zprev, float* __restrict__ dx) {
  __shared__ float ds[kT][kT + 1];
  __shared__ float ws[kT][kT + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int b0 = blockIdx.y * kT, i0 = blockIdx.x * kT;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int o0 = 0; o0 < out; o0 += kT) {
    for (int r = ty; r < kT; r += 8) {
      const int b = b0 + r, o = o0 + tx;
      ds[r][tx] = (b < B && o < out) ? dz[static_cast<long long>(b) * out + o] : 0.f;
      const int oo = o0 + r, i = i0 + tx;
      ws[r][tx] = (oo < out && i < in) ? ldw<BF16>(w, w_off + static_cast<long long>(oo) * in + i) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int o = 0; o < kT; ++o) {
      const float wv = ws[o][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(ds[ty + 8 * q][o], wv, acc[q]);
    }
    __syncthreads();
  }
  const int i = i0 + tx;
  if (i >= in) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int b = b0 + ty + 8 * q;
    if (b >= B) continue;
    const long long e = static_cast<long long>(b) * in + i;
    dx[e] = acc[q] * gelu_grad(zprev[e]);
  }
}

// dw[o][i] = sum_b dz[b][o] x[b][i]
__global__ void __launch_bounds__(256)
k_dense_bwd_w(const float* __restrict__ dz, const float* __restrict__ x, int B, int in, int out,
              float* __restrict__ dw) {
  __shared__ float ds[kT][kT + 1];
  __shared__ float xs[kT][kT + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int o0 = blockIdx.y * kT, i0 = blockIdx.x * kT;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int b0 = 0; b0 < B; b0 += kT) {
    for (int r = ty; r < kT; r += 8) {
      const int b = b0 + r;
      ds[r][tx] = (b < B && o0 + tx < out) ? dz[static_cast<long long>(b) * out + o0 + tx] : 0.f;
      xs[r][tx] = (b < B && i0 + tx < in) ? x[static_cast<long long>(b) * in + i0 + tx] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int b = 0; b < kT; ++b) {
      const float xv = xs[b][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(ds[b][ty + 8 * q], xv, acc[q]);
    }
    __syncthreads();
  }
  const int i = i0 + tx;
  if (i >= in) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int o = o0 + ty + 8 * q;
    if (o < out) dw[static_cast<long long>(o) * in + i] = acc[q];
  }
}

// db[o] = sum_b dz[b][o]  (one warp per output)
__global__ void k_bias_grad(const float* __restrict__ dz, int B, int out, float* __restrict__ db) {
  const int o = blockIdx.x;
  float s = 0.f;
  for (int b = threadIdx.x; b < B; b += blockDim.x) s += dz[static_cast<long long>(b) * out + o];
  for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
  __shared__ float part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.f;
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
    if (threadIdx.x == 0) db[o] = s;
  }
}

// mean BCE loss and dL/dlogit = (sigma(z) - y) / B; one block
__global__ void k_bce(const float* __restrict__ z, const float* __restrict__ y, int B, float* __restrict__ dz,
                      float* __restrict__ loss) {
  float s = 0.f;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const float v = z[b], t = y[b];
    s += fmaxf(v, 0.f) - t * v + log1pf(expf(-fabsf(v)));
    dz[b] = (1.0f / (1.0f + expf(-v)) - t) / static_cast<float>(B);
  }
  for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
  __shared__ float part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.f;
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
    if (threadIdx.x == 0 && loss) *loss = s / static_cast<float>(B);
  }
}

// 1 - b is passed on its own (1 - 0.999f in FP32 is 1.3e-5 off) and the bias
// corrections c = 1 - b^t come from the host in FP64.
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, int n, float lr, float b1, float omb1, float b2, float omb2,
                       float eps, float c1, float c2, __nv_bfloat16* __restrict__ wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + omb1 * gi;
  const float vi = b2 * v[i] + omb2 * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  if (wb) wb[i] = __float2bfloat16_rn(wi);
}

__global__ void k_to_bf16(const float* __restrict__ w, int n, __nv_bfloat16* __restrict__ wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) wb[i] = __float2bfloat16_rn(w[i]);
}

struct ScorerWs {
  float *z1, *h1, *z2, *h2, *z3, *d3, *d2, *d1, *loss;
  int* chan0;
};

ScorerWs carve_scorer(void* ws, size_t bytes, int B, int n_coarse, size_t* need) {
  Carver c(ws, bytes);
  ScorerWs w;
  w.z1 = c.take<float>(static_cast<size_t>(B) * kH1);
  w.h1 = c.take<float>(static_cast<size_t>(B) * kH1);
  w.z2 = c.take<float>(static_cast<size_t>(B) * kH2);
  w.h2 = c.take<float>(static_cast<size_t>(B) * kH2);
  w.z3 = c.take<float>(B);
  w.d3 = c.take<float>(B);
  w.d2 = c.take<float>(static_cast<size_t>(B) * kH2);
  w.d1 = c.take<float>(static_cast<size_t>(B) * kH1);
  w.loss = c.take<float>(1);
  w.chan0 = c.take<int>(n_coarse + 1);
  *need = c.used;
  return w;
}

dim3 tiles(int cols, int rows) { return dim3((cols + kT - 1) / kT, (rows + kT - 1) / kT); }

template <bool BF16>
int forward_impl(const void* w, const float* x, int B, const ScorerWs& s, float* logit, cudaStream_t st) {
  k_dense_fwd<BF16><<<tiles(kH1, B), 256, 0, st>>>(x, w, kW1, kB1, B, kIn, kH1, true, s.z1, s.h1);
  OVRO_LAUNCH_CHECK();
  k_dense_fwd<BF16><<<tiles(kH2, B), 256, 0, st>>>(s.h1, w, kW2, kB2, B, kH1, kH2, true, s.z2, s.h2);
  OVRO_LAUNCH_CHECK();
  k_dense_fwd<BF16><<<tiles(1, B), 256, 0, st>>>(s.h2, w, kW3, kB3, B, kH2, 1, false, nullptr, logit);
  OVRO_LAUNCH_CHECK();
  return OVRO_OK;
}

template <bool BF16>
int grad_impl(const void* w, const float* x, const float* y, int B, const ScorerWs& s, float* grad,
              float* loss_out, cudaStream_t st) {
  if (int e = forward_impl<BF16>(w, x, B, s, s.z3, st)) return e;
  k_bce<<<1, 1024, 0, st>>>(s.z3, y, B, s.d3, s.loss);
  OVRO_LAUNCH_CHECK();
  // layer 3
  k_dense_bwd_w<<<tiles(kH2, 1), 256, 0, st>>>(s.d3, s.h2, B, kH2, 1, grad + kW3);
  OVRO_LAUNCH_CHECK();
  k_bias_grad<<<1, 256, 0, st>>>(s.d3, B, 1, grad + kB3);
  OVRO_LAUNCH_CHECK();
  k_dense_bwd_x<BF16><<<tiles(kH2, B), 256, 0, st>>>(s.d3, w, kW3, B, kH2, 1, s.z2, s.d2);
  OVRO_LAUNCH_CHECK();
  // layer 2
  k_dense_bwd_w<<<tiles(kH1, kH2), 256, 0, st>>>(s.d2, s.h1, B, kH1, kH2, grad + kW2);
  OVRO_LAUNCH_CHECK();
  k_bias_grad<<<kH2, 256, 0, st>>>(s.d2, B, kH2, grad + kB2);
  OVRO_LAUNCH_CHECK();
  k_dense_bwd_x<BF16><<<tiles(kH1, B), 256, 0, st>>>(s.d2, w, kW2, B, kH1, kH2, s.z1, s.d1);
  OVRO_LAUNCH_CHECK();
  // layer 1
  k_dense_bwd_w<<<tiles(kIn, kH1), 256, 0, st>>>(s.d1, x, B, kIn, kH1, grad + kW1);
  OVRO_LAUNCH_CHECK();
  k_bias_grad<<<kH1, 256, 0, st>>>(s.d1, B, kH1, grad + kB1);
  OVRO_LAUNCH_CHECK();
  if (loss_out) OVRO_CUDA_TRY(cudaMemcpyAsync(loss_out, s.loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
  return OVRO_OK;
}

}  // namespace
}  // namespace ovro

extern "C" {

int ovro_scorer_n_params(void) { return ovro::kNParams; }

size_t ovro_scorer_workspace_size(int batch, int n_coarse) {
  if (batch <= 0) return 0;
  size_t need = 0;
  ovro::carve_scorer(nullptr, 0, batch, n_coarse > 0 ? n_coarse : 1, &need);
  return need;
}

int ovro_scorer_cutouts(const float* d_zp, int n_chan, int image_size, int n_coarse, const int32_t* h_nfft,
                        const int32_t* d_trig, int n_trig, float* d_x, void* d_ws, size_t ws_bytes,
                        void* stream) {
  using namespace ovro;
  if (!d_zp || !h_nfft || !d_x || n_chan <= 0 || image_size <= 0 || n_coarse <= 0 || n_trig < 0)
    return OVRO_ERR_INVALID_ARG;
  if (n_trig == 0) return OVRO_OK;
  if (!d_trig) return OVRO_ERR_INVALID_ARG;
  size_t need = 0;
  ScorerWs s = carve_scorer(d_ws, ws_bytes, 1, n_coarse, &need);
  if (int e = check_workspace(d_ws, ws_bytes, need)) return e;
  std::vector<int> c0(n_coarse + 1, 0);
  for (int c = 0; c < n_coarse; ++c) {
    if (h_nfft[c] <= 0) return OVRO_ERR_INVALID_ARG;
    c0[c + 1] = c0[c] + h_nfft[c];
  }
  if (c0[n_coarse] != n_chan) return OVRO_ERR_INVALID_ARG;
  cudaStream_t st = as_stream(stream);
  OVRO_CUDA_TRY(cudaMemcpyAsync(s.chan0, c0.data(), c0.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  const long long total = static_cast<long long>(n_trig) * kIn;
  const int blocks = static_cast<int>(std::min<long long>((total + 255) / 256, 8LL * num_sms()));
  k_cutouts<<<blocks, 256, 0, st>>>(d_zp, n_chan, image_size, s.chan0, n_coarse, d_trig, n_trig, d_x);
  OVRO_LAUNCH_CHECK();
  return OVRO_OK;
}

int ovro_scorer_forward(const void* d_w_bf16, const float* d_x, int batch, float* d_logit, void* d_ws,
                        size_t ws_bytes, void* stream) {
  using namespace ovro;
  if (!d_w_bf16 || !d_x || !d_logit || batch <= 0) return OVRO_ERR_INVALID_ARG;
  size_t need = 0;
  ScorerWs s = carve_scorer(d_ws, ws_bytes, batch, 1, &need);
  if (int e = check_workspace(d_ws, ws_bytes, need)) return e;
  OVRO_PROF("k_scorer_fwd", as_stream(stream));
  return forward_impl<true>(d_w_bf16, d_x, batch, s, d_logit, as_stream(stream));
}

int ovro_scorer_grad(const void* d_w, int w_is_bf16, const float* d_x, const float* d_y, int batch,
                     float* d_grad, float* d_loss_or_null, void* d_ws, size_t ws_bytes, void* stream) {
  using namespace ovro;
  if (!d_w || !d_x || !d_y || !d_grad || batch <= 0) return OVRO_ERR_INVALID_ARG;
  size_t need = 0;
  ScorerWs s = carve_scorer(d_ws, ws_bytes, batch, 1, &need);
  if (int e = check_workspace(d_ws, ws_bytes, need)) return e;
  cudaStream_t st = as_stream(stream);
  return w_is_bf16 ? grad_impl<true>(d_w, d_x, d_y, batch, s, d_grad, d_loss_or_null, st)
                   : grad_impl<false>(d_w, d_x, d_y, batch, s, d_grad, d_loss_or_null, st);
}

int ovro_scorer_adam(float* d_master, float* d_m, float* d_v, const float* d_grad, int step, float lr,
                     void* d_w_bf16_or_null, void* stream) {
  using namespace ovro;
  if (!d_master || !d_m || !d_v || !d_grad || step <= 0 || !(lr > 0.f)) return OVRO_ERR_INVALID_ARG;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = static_cast<float>(1.0 - std::pow(b1, step));
  const float c2 = static_cast<float>(1.0 - std::pow(b2, step));
  k_adam<<<(kNParams + 255) / 256, 256, 0, as_stream(stream)>>>(
      d_master, d_m, d_v, d_grad, kNParams, lr, static_cast<float>(b1), static_cast<float>(1.0 - b1),
      static_cast<float>(b2), static_cast<float>(1.0 - b2), 1e-8f, c1, c2,
      static_cast<__nv_bfloat16*>(d_w_bf16_or_null));
  OVRO_LAUNCH_CHECK();
  return OVRO_OK;
}

int ovro_scorer_to_bf16(const float* d_master, void* d_w_bf16, void* stream) {
  using namespace ovro;
  if (!d_master || !d_w_bf16) return OVRO_ERR_INVALID_ARG;
  k_to_bf16<<<(kNParams + 255) / 256, 256, 0, as_stream(stream)>>>(d_master, kNParams,
                                                                   static_cast<__nv_bfloat16*>(d_w_bf16));
  OVRO_LAUNCH_CHECK();
  return OVRO_OK;
}

}  // extern "C"
