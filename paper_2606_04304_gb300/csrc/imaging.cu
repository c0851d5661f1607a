// a5-a7: uvw, prolate-spheroidal gridding and dirty imaging per fine channel.
//
// Section 2.2 of the paper images every fine channel over the visible
// hemisphere; the dirty images are the search product.  Per channel:
//
//  a5  u = (x_a - x_b) s_nu in grid cells with s_nu = nu / (c du): one
//      correctly rounded FP64 multiply per coordinate, then rounded to 1/Q
//      cell.  GB300's FP64 pipe is narrow, so k_bin evaluates the product as a
//      float-float product and only falls back to a real FP64 multiply when
//      the float-float bound cannot decide rint(u Q) (|frac - 1/2| within the
//      error bound) -- the integer result equals the FP64 definition exactly.
//  a6  Stokes I = (XX + YY)/2 of each kept cross baseline is gridded once (the
//      mirror conj(V) at (-u, -v) is accounted for by taking 2 Re of the
//      transform, which is exact because the mirror's footprint is the point
//      reflection), with a separable 7 x 7 prolate-spheroidal kernel.  k_bin
//      sorts visibilities into row bands of the grid; k_grid accumulates one
//      band per CTA in shared memory with shared-memory atomics.
//  a7  The uv grid is padded by 2 (G = 2N cells a side, du = 1 / (G cell)) and
//      the image is the central N x N of its transform, as padded imagers do:
//      the horizon then sits where the kernel's transform is still > 0.25, so
//      the grid correction does not amplify FP32 round-off.  The grid is
//      transformed by row FFTs (k_fft_rows) and column FFTs of the N central
//      columns (k_fft_cols); the centring shifts become a (-1)^(ku+kv) sign at
//      gridding time and (-1)^(r+c) at output, the exp(+) transform becomes a
//      forward transform of the conjugated grid, and the column pass applies
//      normalisation, the grid correction and the horizon mask while writing
//      the image.  Channel batches keep the intermediate grids L2-sized.
#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "pswf.h"

namespace ovro {
namespace {

constexpr double kCLight = 299792458.0;
constexpr int kQ = kOversample;
constexpr int kHalfTab = kSupport * kOversample / 2;
constexpr int kTabLen = 2 * kHalfTab + 1;
constexpr int kHalfSup = kSupport / 2;
constexpr int kPad = 2;              // uv grid cells per image pixel, per axis

struct Baseline {
  double dx, dy;
  float dxh, dxl, dyh, dyl;
  long long bl;
};

struct ChanScale {
  double s;          // s_nu * Q
  float sh, sl;      // float-float split of s
};

__host__ __device__ __forceinline__ long long bl_index(int a, int b, int n) {
  return static_cast<long long>(a) * n - static_cast<long long>(a) * (a - 1) / 2 + (b - a);
}

__global__ void k_baselines(const double* __restrict__ ant, int n_ant, Baseline* __restrict__ out) {
  const int a = blockIdx.y;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_ant || b <= a) return;
  const long long bl = bl_index(a, b, n_ant);
  Baseline B;
  B.dx = ant[3 * a] - ant[3 * b];
  B.dy = ant[3 * a + 1] - ant[3 * b + 1];
  B.dxh = static_cast<float>(B.dx);
  B.dxl = static_cast<float>(B.dx - static_cast<double>(B.dxh));
  B.dyh = static_cast<float>(B.dy);
  B.dyl = static_cast<float>(B.dy - static_cast<double>(B.dyh));
  B.bl = bl;
  out[bl - a - 1] = B;            // cross baselines in (a, b), a < b, row-major order
}

__global__ void k_chan_scale(const double* __restrict__ freq, int n_chan, int n, double cell,
                             ChanScale* __restrict__ out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_chan) return;
  const double du = 1.0 / (static_cast<double>(n) * cell);
  const double s = freq[f] / (kCLight * du);
  ChanScale c;
  c.s = s * static_cast<double>(kQ);          // exact: Q is a power of two
  c.sh = static_cast<float>(c.s);
  c.sl = static_cast<float>(c.s - static_cast<double>(c.sh));
  out[f] = c;
}

// rint(fl64(x * s)) for the FP64 product, decided in FP32 whenever possible.
__device__ __forceinline__ long long exact_rint_prod(double x, float xh, float xl, const ChanScale& s) {
  const float hi = __fmul_rn(xh, s.sh);
  if (!(fabsf(hi) < 2097152.0f))                       // |P| >= 2^21: take the FP64 path
    return __double2ll_rn(__dmul_rn(x, s.s));
  const float e = __fmaf_rn(xh, s.sh, -hi);           // exact error of hi
  const float t = __fmaf_rn(xh, s.sl, __fmaf_rn(xl, s.sh, e));
  const float n = rintf(hi);
  const float f = __fadd_rn(hi - n, t);              // P - n, |error| < 1.2e-7
  const float margin = 2.5e-7f;
  long long p = static_cast<long long>(n);
  if (fabsf(fabsf(f) - 0.5f) <= margin) return __double2ll_rn(__dmul_rn(x, s.s));
  if (f > 0.5f) p += 1;
  else if (f < -0.5f) p -= 1;
  return p;
}

__device__ __forceinline__ void centre_cell(long long p, int& c0, int& off) {
  const long long ap = p < 0 ? -p : p;
  long long c = (ap + kQ / 2) / kQ;
  if (p < 0) c = -c;
  c0 = static_cast<int>(c);
  off = static_cast<int>(p - c * kQ);
}

// a5 on its own: rounded positions p_u, p_v (1/Q cells) of every cross baseline.
__global__ void k_uvw(const Baseline* __restrict__ base, int n_cross, const ChanScale* __restrict__ cs,
                      int32_t* __restrict__ pu, int32_t* __restrict__ pv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int f = blockIdx.y;
  if (i >= n_cross) return;
  const Baseline B = base[i];
  const ChanScale s = cs[f];
  const long long u = exact_rint_prod(B.dx, B.dxh, B.dxl, s);
  const long long v = exact_rint_prod(B.dy, B.dyh, B.dyl, s);
  const long long lim = 1LL << 30;
  const long long o = static_cast<long long>(f) * n_cross + i;
  pu[o] = static_cast<int32_t>(u > lim ? lim : (u < -lim ? -lim : u));
  pv[o] = static_cast<int32_t>(v > lim ? lim : (v < -lim ? -lim : v));
}

// Keep test + band binning of every (channel, cross baseline) in the batch.
__global__ void k_bin(const Baseline* __restrict__ base, int n_cross, const ChanScale* __restrict__ cs,
                      int ch0, int n, int band_h, int n_bands, long long cap,
                      int4* __restrict__ lists, int* __restrict__ list_cnt, int* __restrict__ kept) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int cb = blockIdx.y;
  bool keep = false;
  int c0u = 0, offu = 0, c0v = 0, offv = 0;
  long long pu = 0, pv = 0;
  if (i < n_cross) {
    const Baseline B = base[i];
    const ChanScale s = cs[ch0 + cb];
    pu = exact_rint_prod(B.dx, B.dxh, B.dxl, s);
    pv = exact_rint_prod(B.dy, B.dyh, B.dyl, s);
    const long long lim = static_cast<long long>(n / 2 - kHalfSup - 1) * kQ + kQ;  // loose pre-check
    if (pu > -lim && pu < lim && pv > -lim && pv < lim) {
      centre_cell(pu, c0u, offu);
      centre_cell(pv, c0v, offv);
      const int cmax = n / 2 - kHalfSup - 1;
      keep = (c0u <= cmax && c0u >= -cmax && c0v <= cmax && c0v >= -cmax);
    }
  }
  const unsigned m = __ballot_sync(0xffffffffu, keep);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(kept + ch0 + cb, __popc(m));
  if (!keep) return;
  const int kv_lo = n / 2 + c0v - kHalfSup;
  const int b0 = kv_lo / band_h, b1 = (kv_lo + kSupport - 1) / band_h;
  for (int b = b0; b <= b1; ++b) {
    const int slot = cb * n_bands + b;
    const int pos = atomicAdd(list_cnt + slot, 1);
    lists[static_cast<long long>(slot) * cap + pos] =
        make_int4(i, static_cast<int>(pu), static_cast<int>(pv), 0);
  }
}

// One row band of one channel's grid, accumulated in shared memory.
__global__ void __launch_bounds__(512)
k_grid(const int4* __restrict__ lists, const int* __restrict__ list_cnt, int n_bands, long long cap,
       const int32_t* __restrict__ vis, long long n_bl, const Baseline* __restrict__ base,
       const float* __restrict__ tab, int ch0, int n, int band_h, float2* __restrict__ grids) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* band = reinterpret_cast<float2*>(smem);
  float* stab = reinterpret_cast<float*>(smem + static_cast<size_t>(band_h) * n * sizeof(float2));
  const int b = blockIdx.x, cb = blockIdx.y;
  const int ncell = band_h * n;
  for (int i = threadIdx.x; i < ncell; i += blockDim.x) band[i] = make_float2(0.f, 0.f);
  for (int i = threadIdx.x; i < kTabLen; i += blockDim.x) stab[i] = tab[i];
  __syncthreads();
  const int slot = cb * n_bands + b;
  const int cnt = list_cnt[slot];
  const int4* L = lists + static_cast<long long>(slot) * cap;
  const int row0 = b * band_h;
  const long long chan = ch0 + cb;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int4 en = L[e];
    const long long bl = base[en.x].bl;
    const int4* v = reinterpret_cast<const int4*>(vis + (chan * n_bl + bl) * 8);
    const int4 xx_xy = __ldg(v);
    const int4 yx_yy = __ldg(v + 1);
    // conj of Stokes I: the exp(+) image transform is done as a forward FFT of conj(G)
    const float vr = 0.5f * static_cast<float>(xx_xy.x + yx_yy.z);
    const float vi = -0.5f * static_cast<float>(xx_xy.y + yx_yy.w);
    int c0u, offu, c0v, offv;
    centre_cell(en.y, c0u, offu);
    centre_cell(en.z, c0v, offv);
    float wu[kSupport];
#pragma unroll
    for (int t = 0; t < kSupport; ++t) {
      const int ku = n / 2 + c0u + t - kHalfSup;
      const float w = stab[kHalfTab + (t - kHalfSup) * kQ - offu];
      wu[t] = (ku & 1) ? -w : w;
    }
    const int ku0 = n / 2 + c0u - kHalfSup;
#pragma unroll
    for (int tv = 0; tv < kSupport; ++tv) {
      const int kv = n / 2 + c0v + tv - kHalfSup;
      const int row = kv - row0;
      if (row < 0 || row >= band_h) continue;
      float wv = stab[kHalfTab + (tv - kHalfSup) * kQ - offv];
      if (kv & 1) wv = -wv;
      float2* dst = band + row * n + ku0;
#pragma unroll
      for (int tu = 0; tu < kSupport; ++tu) {
        const float w = wv * wu[tu];
        atomicAdd(&dst[tu].x, w * vr);
        atomicAdd(&dst[tu].y, w * vi);
      }
    }
  }
  __syncthreads();
  float4* g = reinterpret_cast<float4*>(grids + (static_cast<long long>(cb) * n + row0) * n);
  const float4* s4 = reinterpret_cast<const float4*>(band);
  for (int i = threadIdx.x; i < ncell / 2; i += blockDim.x) g[i] = s4[i];
}

template <int LOG2N>
__global__ void __launch_bounds__(512)
k_fft_rows(float2* __restrict__ grids, int rows_per_cta, const float2* __restrict__ tw) {
  constexpr int N = 1 << LOG2N;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* A = reinterpret_cast<float2*>(smem);
  float2* B = A + rows_per_cta * N;
  const int cb = blockIdx.y;
  float2* g = grids + (static_cast<long long>(cb) * N + blockIdx.x * rows_per_cta) * N;
  const int n4 = rows_per_cta * N / 2;
  for (int i = threadIdx.x; i < n4; i += blockDim.x)
    reinterpret_cast<float4*>(A)[i] = reinterpret_cast<const float4*>(g)[i];
  __syncthreads();
  const float2* res = fft_rows_pingpong<LOG2N>(A, B, rows_per_cta, N, tw, 1);
  for (int i = threadIdx.x; i < n4; i += blockDim.x)
    reinterpret_cast<float4*>(g)[i] = reinterpret_cast<const float4*>(res)[i];
}

template <int LOG2G>
__global__ void __launch_bounds__(512)
k_fft_cols(const float2* __restrict__ grids, int n_img, int cols_per_cta, int ch0,
           const float2* __restrict__ tw, const float* __restrict__ inv_corr,
           const uint8_t* __restrict__ mask, const int* __restrict__ kept, float* __restrict__ img) {
  constexpr int G = 1 << LOG2G;
  constexpr int LD = G + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* A = reinterpret_cast<float2*>(smem);
  float2* B = A + cols_per_cta * LD;
  const int C = cols_per_cta;
  const int cb = blockIdx.y;
  const int off = G / 2 - n_img / 2;                  // first central grid row/column
  const int c0 = blockIdx.x * C;                      // image column of this strip
  const float2* g = grids + static_cast<long long>(cb) * G * G;
  for (int i = threadIdx.x; i < G * C; i += blockDim.x) {
    const int r = i / C, c = i - r * C;
    A[c * LD + r] = g[static_cast<long long>(r) * G + off + c0 + c];
  }
  __syncthreads();
  const float2* res = fft_rows_pingpong<LOG2G>(A, B, C, LD, tw, 1);
  const long long chan = ch0 + cb;
  const int k = kept[chan];
  const float norm = k > 0 ? 1.0f / static_cast<float>(k) : 0.0f;
  float* out = img + chan * n_img * n_img;
  for (int i = threadIdx.x; i < n_img * C; i += blockDim.x) {
    const int r = i / C, c = i - r * C;
    const int col = c0 + c;
    float v = 0.0f;
    if (mask[r * n_img + col]) {
      v = res[c * LD + off + r].x * norm * inv_corr[r] * inv_corr[col];
      if ((r + col) & 1) v = -v;
    }
    out[static_cast<long long>(r) * n_img + col] = v;
  }
}

__global__ void k_mask(int n, double cell, uint8_t* __restrict__ mask) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * n) return;
  const int r = i / n, c = i - r * n;
  const double l = static_cast<double>(c - n / 2) * cell;
  const double m = static_cast<double>(r - n / 2) * cell;
  mask[i] = (l * l + m * m) < 1.0 ? 1 : 0;
}

__global__ void k_twiddle_img(float2* tw, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double s, c;
  sincospi(-2.0 * static_cast<double>(k) / static_cast<double>(n), &s, &c);
  tw[k] = make_float2(static_cast<float>(c), static_cast<float>(s));
}

__global__ void k_counts_out(const int* __restrict__ kept, int n_chan, int32_t* __restrict__ out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < n_chan) out[f] = 2 * kept[f];
}

// ---------------------------------------------------------------- planning
struct ImgPlan {
  int n, g, log2g, band_h, n_bands, batch, rows_per_cta, cols_per_cta;
  long long n_cross, cap;
};

ImgPlan make_plan(int n_ant, int n_chan, int n) {
  ImgPlan p;
  p.n = n;
  p.g = kPad * n;
  p.log2g = ilog2(p.g);
  p.band_h = 16384 / p.g < p.g ? 16384 / p.g : p.g;   // band of <= 128 KB FP32 complex
  p.n_bands = p.g / p.band_h;
  p.n_cross = static_cast<long long>(n_ant) * (n_ant - 1) / 2;
  p.cap = p.n_cross > 0 ? p.n_cross : 1;
  const long long grid_bytes = 8LL * p.g * p.g;
  const long long list_bytes = 16LL * p.n_bands * p.cap;
  long long b = (64LL << 20) / grid_bytes;
  const long long bl = (512LL << 20) / list_bytes;
  if (bl < b) b = bl;
  if (b < 1) b = 1;
  if (b > 64) b = 64;
  if (b > n_chan) b = n_chan;
  p.batch = static_cast<int>(b);
  p.rows_per_cta = 8192 / p.g < p.g ? 8192 / p.g : p.g;
  int c = 8192 / p.g;
  if (c > n) c = n;
  if (c > 32) c = 32;
  p.cols_per_cta = c;
  return p;
}

struct ImgWs {
  float* tab;
  float* inv_corr;
  float2* tw;
  uint8_t* mask;
  double* ant;
  double* freq;
  Baseline* base;
  ChanScale* cs;
  int* kept;
  int* list_cnt;
  int4* lists;
  float2* grids;
};

ImgWs carve_img(void* ws, size_t bytes, const ImgPlan& p, int n_ant, int n_chan, size_t* need) {
  Carver c(ws, bytes);
  ImgWs w;
  w.tab = c.take<float>(kTabLen);
  w.inv_corr = c.take<float>(p.n);
  w.tw = c.take<float2>(p.g);
  w.mask = c.take<uint8_t>(static_cast<size_t>(p.n) * p.n);
  w.ant = c.take<double>(static_cast<size_t>(n_ant) * 3);
  w.freq = c.take<double>(n_chan);
  w.base = c.take<Baseline>(p.n_cross > 0 ? p.n_cross : 1);
  w.cs = c.take<ChanScale>(n_chan);
  w.kept = c.take<int>(n_chan);
  w.list_cnt = c.take<int>(static_cast<size_t>(p.batch) * p.n_bands);
  w.lists = c.take<int4>(static_cast<size_t>(p.batch) * p.n_bands * p.cap);
  w.grids = c.take<float2>(static_cast<size_t>(p.batch) * p.g * p.g);
  *need = c.used;
  return w;
}

template <int L>
int launch_ffts(const ImgPlan& p, const ImgWs& w, int ch0, int nb, float* img, cudaStream_t st) {
  constexpr int G = 1 << L;
  {
    const size_t sm = 2ull * p.rows_per_cta * G * sizeof(float2);
    OVRO_CUDA_TRY(cudaFuncSetAttribute(k_fft_rows<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sm)));
    dim3 grid(G / p.rows_per_cta, nb);
    k_fft_rows<L><<<grid, 512, sm, st>>>(w.grids, p.rows_per_cta, w.tw);
    OVRO_LAUNCH_CHECK();
  }
  {
    const size_t sm = 2ull * p.cols_per_cta * (G + 1) * sizeof(float2);
    OVRO_CUDA_TRY(cudaFuncSetAttribute(k_fft_cols<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sm)));
    dim3 grid(p.n / p.cols_per_cta, nb);
    k_fft_cols<L><<<grid, 512, sm, st>>>(w.grids, p.n, p.cols_per_cta, ch0, w.tw, w.inv_corr, w.mask,
                                         w.kept, img);
    OVRO_LAUNCH_CHECK();
  }
  return OVRO_OK;
}

int run_ffts(const ImgPlan& p, const ImgWs& w, int ch0, int nb, float* img, cudaStream_t st) {
  switch (p.log2g) {
    case 5: return launch_ffts<5>(p, w, ch0, nb, img, st);
    case 6: return launch_ffts<6>(p, w, ch0, nb, img, st);
    case 7: return launch_ffts<7>(p, w, ch0, nb, img, st);
    case 8: return launch_ffts<8>(p, w, ch0, nb, img, st);
    case 9: return launch_ffts<9>(p, w, ch0, nb, img, st);
    case 10: return launch_ffts<10>(p, w, ch0, nb, img, st);
    case 11: return launch_ffts<11>(p, w, ch0, nb, img, st);
    default: return OVRO_ERR_UNSUPPORTED;
  }
}

int upload_common(const ImgPlan& p, const ImgWs& w, int n_ant, const double* h_ant,
                  const double* h_freq, int n_chan, double cell, cudaStream_t st) {
  const KernelTables& kt = kernel_tables();
  std::vector<double> corr;
  grid_correction(p.n, p.g, corr);
  std::vector<float> inv(p.n);
  for (int i = 0; i < p.n; ++i) inv[i] = static_cast<float>(1.0 / corr[i]);
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.tab, kt.table32.data(), kTabLen * sizeof(float),
                                cudaMemcpyHostToDevice, st));
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.inv_corr, inv.data(), p.n * sizeof(float), cudaMemcpyHostToDevice, st));
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.ant, h_ant, static_cast<size_t>(n_ant) * 3 * sizeof(double),
                                cudaMemcpyHostToDevice, st));
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.freq, h_freq, static_cast<size_t>(n_chan) * sizeof(double),
                                cudaMemcpyHostToDevice, st));
  // host->device copies from pageable memory are staged before cudaMemcpyAsync
  // returns, so the temporaries above may go out of scope
  k_twiddle_img<<<(p.g + 255) / 256, 256, 0, st>>>(w.tw, p.g);
  OVRO_LAUNCH_CHECK();
  k_mask<<<(p.n * p.n + 255) / 256, 256, 0, st>>>(p.n, cell, w.mask);
  OVRO_LAUNCH_CHECK();
  if (p.n_cross > 0) {
    dim3 g((n_ant + 127) / 128, n_ant);
    k_baselines<<<g, 128, 0, st>>>(w.ant, n_ant, w.base);
    OVRO_LAUNCH_CHECK();
  }
  k_chan_scale<<<(n_chan + 255) / 256, 256, 0, st>>>(w.freq, n_chan, p.g, cell, w.cs);
  OVRO_LAUNCH_CHECK();
  return OVRO_OK;
}

int validate(int n_ant, const double* h_ant, const double* h_freq, int n_chan, int n, double cell) {
  if (!h_ant || !h_freq || n_ant <= 0 || n_chan <= 0) return OVRO_ERR_INVALID_ARG;
  if (!(cell > 0.0)) return OVRO_ERR_INVALID_ARG;
  if (!is_pow2(n) || n < 16 || n > 1024) return OVRO_ERR_UNSUPPORTED;
  if (n_ant > 4096) return OVRO_ERR_UNSUPPORTED;
  return OVRO_OK;
}

}  // namespace
}  // namespace ovro

extern "C" {

size_t ovro_grid_image_workspace_size(int n_ant, int n_chan, int image_size, int storage) {
  using namespace ovro;
  if (n_ant <= 0 || n_chan <= 0 || !is_pow2(image_size) || image_size < 16 || image_size > 1024)
    return 0;
  (void)storage;
  const ImgPlan p = make_plan(n_ant, n_chan, image_size);
  size_t need = 0;
  carve_img(nullptr, 0, p, n_ant, n_chan, &need);
  return need;
}

int ovro_grid_image(const int32_t* d_vis, int n_ant, const double* h_ant_enu_m,
                    const double* h_chan_freq_hz, int n_chan, int image_size, double cell_dircos,
                    int storage, float* d_img, int32_t* d_n_gridded_or_null, void* d_ws,
                    size_t ws_bytes, void* stream) {
  using namespace ovro;
  if (!d_vis || !d_img) return OVRO_ERR_INVALID_ARG;
  if (int e = validate(n_ant, h_ant_enu_m, h_chan_freq_hz, n_chan, image_size, cell_dircos)) return e;
  if (storage != OVRO_STORE_FP32 && storage != OVRO_STORE_BF16 && storage != OVRO_STORE_FP16)
    return OVRO_ERR_INVALID_ARG;
  if (storage != OVRO_STORE_FP32) return OVRO_ERR_UNSUPPORTED;
  if (reinterpret_cast<uintptr_t>(d_vis) % 16 != 0) return OVRO_ERR_INVALID_ARG;
  const ImgPlan p = make_plan(n_ant, n_chan, image_size);
  size_t need = 0;
  ImgWs w = carve_img(d_ws, ws_bytes, p, n_ant, n_chan, &need);
  if (int e = check_workspace(d_ws, ws_bytes, need)) return e;
  cudaStream_t st = as_stream(stream);
  if (int e = upload_common(p, w, n_ant, h_ant_enu_m, h_chan_freq_hz, n_chan, cell_dircos, st)) return e;
  OVRO_CUDA_TRY(cudaMemsetAsync(w.kept, 0, n_chan * sizeof(int), st));
  const long long n_bl = static_cast<long long>(n_ant) * (n_ant + 1) / 2;
  const size_t grid_smem = static_cast<size_t>(p.band_h) * p.g * sizeof(float2) + kTabLen * sizeof(float);
  OVRO_CUDA_TRY(cudaFuncSetAttribute(k_grid, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(grid_smem)));
  for (int ch0 = 0; ch0 < n_chan; ch0 += p.batch) {
    const int nb = n_chan - ch0 < p.batch ? n_chan - ch0 : p.batch;
    OVRO_CUDA_TRY(cudaMemsetAsync(w.list_cnt, 0, static_cast<size_t>(p.batch) * p.n_bands * sizeof(int), st));
    if (p.n_cross > 0) {
      dim3 gb(static_cast<unsigned>((p.n_cross + 255) / 256), nb);
      k_bin<<<gb, 256, 0, st>>>(w.base, static_cast<int>(p.n_cross), w.cs, ch0, p.g, p.band_h,
                                p.n_bands, p.cap, w.lists, w.list_cnt, w.kept);
      OVRO_LAUNCH_CHECK();
    }
    dim3 gg(p.n_bands, nb);
    k_grid<<<gg, 512, grid_smem, st>>>(w.lists, w.list_cnt, p.n_bands, p.cap, d_vis, n_bl, w.base,
                                       w.tab, ch0, p.g, p.band_h, w.grids);
    OVRO_LAUNCH_CHECK();
    if (int e = run_ffts(p, w, ch0, nb, d_img, st)) return e;
  }
  if (d_n_gridded_or_null) {
    k_counts_out<<<(n_chan + 255) / 256, 256, 0, st>>>(w.kept, n_chan, d_n_gridded_or_null);
    OVRO_LAUNCH_CHECK();
  }
  return OVRO_OK;
}

// a5 alone: rounded uv positions p = rint(u Q), Q = 1024, of every cross
// baseline (a < b, row-major) in every channel: int32 [n_chan][n_cross]
// (saturated at +-2^30).  Workspace as for ovro_grid_image.
int ovro_uvw(const double* h_ant_enu_m, int n_ant, const double* h_chan_freq_hz, int n_chan,
             int image_size, double cell_dircos, int32_t* d_pu, int32_t* d_pv, void* d_ws,
             size_t ws_bytes, void* stream) {
  using namespace ovro;
  if (!d_pu || !d_pv) return OVRO_ERR_INVALID_ARG;
  if (int e = validate(n_ant, h_ant_enu_m, h_chan_freq_hz, n_chan, image_size, cell_dircos)) return e;
  const ImgPlan p = make_plan(n_ant, n_chan, image_size);
  size_t need = 0;
  ImgWs w = carve_img(d_ws, ws_bytes, p, n_ant, n_chan, &need);
  if (int e = check_workspace(d_ws, ws_bytes, need)) return e;
  cudaStream_t st = as_stream(stream);
  if (int e = upload_common(p, w, n_ant, h_ant_enu_m, h_chan_freq_hz, n_chan, cell_dircos, st)) return e;
  if (p.n_cross == 0) return OVRO_OK;
  dim3 g(static_cast<unsigned>((p.n_cross + 255) / 256), n_chan);
  k_uvw<<<g, 256, 0, st>>>(w.base, static_cast<int>(p.n_cross), w.cs, d_pu, d_pv);
  OVRO_LAUNCH_CHECK();
  return OVRO_OK;
}

}  // extern "C"
