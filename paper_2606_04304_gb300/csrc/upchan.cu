// a1-a3: unpack 4+4-bit voltages, FFT upchannelizer, 8-bit requantisation.
//
// Section 2.1 of the paper: each ~24 kHz coarse channel is upchannelized by an
// FFT over its time samples, and the fine-channel voltages are correlated by an
// 8-bit X-engine.  One CTA handles one spectrum (N consecutive samples) of a
// group of G adjacent inputs: it stages the G-byte-wide rows of packed samples
// in shared memory, runs F FFTs at a time (Stockham auto-sort, radix-16 passes
// through a padded shared exchange buffer, 16 complex values per thread in
// registers), requantises the bins into a staging tile and writes the int8
// spectra for all G inputs with row-contiguous stores, so the output for fine
// channel k' is one 2G-byte run in [k'][spectrum][input] order -- the layout
// the X-engine reads.
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "tune.h"
#include "upchan_impl.h"

namespace ovro {
namespace {

constexpr int kMaxLog2N = 14;
constexpr int kMaxN = 1 << kMaxLog2N;

// ---------------------------------------------------------------- power pass
// Exact sum over the used samples of re^2 + im^2 per (coarse, input).
__device__ __forceinline__ uint32_t sample_power(uint32_t b) {
  int re = static_cast<int>(static_cast<int8_t>(b)) >> 4;
  int im = static_cast<int>(static_cast<int8_t>(b << 4)) >> 4;
  return static_cast<uint32_t>(re * re + im * im);
}

template <int VW>
__global__ void k_power(const uint8_t* __restrict__ volt, int n_input, long long n_used,
                        unsigned long long* __restrict__ power) {
  // thread = one VW-byte column of the row; blocks stride over rows
  const int nvec = (n_input + VW - 1) / VW;
  const int v = blockIdx.y * blockDim.x + threadIdx.x;
  if (v >= nvec) return;
  uint32_t acc[VW];
#pragma unroll
  for (int j = 0; j < VW; ++j) acc[j] = 0;
  const bool full = (v + 1) * VW <= n_input;
#pragma unroll 4
  for (long long r = blockIdx.x; r < n_used; r += gridDim.x) {
    const uint8_t* p = volt + r * n_input + static_cast<long long>(v) * VW;
    if (VW == 16) {
      const uint4 w = __ldg(reinterpret_cast<const uint4*>(p));
      const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[q * 4 + b] += sample_power((ws[q] >> (8 * b)) & 0xffu);
    } else if (VW == 4) {
      const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(p));
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[b] += sample_power((w >> (8 * b)) & 0xffu);
    } else {
#pragma unroll
      for (int b = 0; b < VW; ++b)
        if (full || v * VW + b < n_input) acc[b] += sample_power(p[b]);
    }
  }
#pragma unroll
  for (int j = 0; j < VW; ++j)
    if (v * VW + j < n_input && acc[j]) atomicAdd(power + v * VW + j, static_cast<unsigned long long>(acc[j]));
}

// s = 8 sqrt(2) / sqrt(W P), P = power / n_used, in FP64; rounded to FP32.
// W = N for the plain FFT, the sum of the squared taps (*h2) for a PFB.
__global__ void k_scale(const unsigned long long* __restrict__ power, const double* __restrict__ user,
                        int n, int nfft, long long n_used, const double* __restrict__ h2,
                        float* __restrict__ scale) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s;
  if (user) {
    s = user[i];
  } else {
    const double w = h2 ? *h2 : static_cast<double>(nfft);
    double pbar = static_cast<double>(power[i]) / static_cast<double>(n_used);
    s = pbar > 0.0 ? (8.0 * sqrt(2.0)) / sqrt(w * pbar) : 0.0;
  }
  scale[i] = static_cast<float>(s);
}

// *out = sum of h[i]^2 in FP64 (each square exact), one CTA of 256 threads.
__global__ void __launch_bounds__(256) k_sumsq(const float* __restrict__ h, int n, double* __restrict__ out) {
  __shared__ double part[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) {
    const double x = static_cast<double>(h[i]);
    acc += x * x;
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = part[0];
}

// omega_N^k = exp(-2 pi i k / N) for the largest N in the call, FP64 -> FP32.
__global__ void k_twiddle(float2* tw, int n) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double s, c;
  sincospi(-2.0 * static_cast<double>(k) / static_cast<double>(n), &s, &c);
  tw[k] = make_float2(static_cast<float>(c), static_cast<float>(s));
}

// --------------------------------------------------------- FFT + requantise


// N = 2, 4, 8: one thread per FFT (the whole transform in registers), 256
// inputs of the group at a time.
template <int LOG2N>
__global__ void __launch_bounds__(256)
k_upchan(UpchanArgs a) {
  constexpr int N = 1 << LOG2N;
  static_assert(N < 16, "short transforms only");
  extern __shared__ __align__(16) unsigned char smem[];
  const int G = a.group;
  uint8_t* raw = smem;                                                          // [N][G]
  int8_t* stg = reinterpret_cast<int8_t*>(raw + static_cast<size_t>(N) * G);    // [N][G][2]
  float* sc = reinterpret_cast<float*>(
      stg + ((static_cast<size_t>(N) * G * 2 + 15) & ~static_cast<size_t>(15)));  // [G]
  const int tid = threadIdx.x;
  const int T = blockDim.x;
  const int s = blockIdx.y;
  const int i0 = blockIdx.x * G;
  const int gv = min(G, a.n_input - i0);
  const long long row0 = static_cast<long long>(s) * N;
  {
    const uint8_t* src = a.volt + row0 * a.n_input + i0;
    for (int idx = tid; idx < N * G; idx += T) {
      const int n = idx / G, g = idx - n * G;
      raw[idx] = g < gv ? src[static_cast<long long>(n) * a.n_input + g] : 0;
    }
    for (int g = tid; g < G; g += T) sc[g] = g < gv ? a.scale[i0 + g] : 0.0f;
  }
  __syncthreads();
  for (int g = tid; g < gv; g += T) {
    float2 v[N];
#pragma unroll
    for (int n = 0; n < N; ++n) {
      const uint32_t byte = raw[n * G + g];
      v[n].x = static_cast<float>(static_cast<int>(static_cast<int8_t>(byte)) >> 4);
      v[n].y = static_cast<float>(static_cast<int>(static_cast<int8_t>(byte << 4)) >> 4);
    }
    dft_reg<N>(v);
    const float s_g = sc[g];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int kp = (k + N / 2) & (N - 1);
      float qr = rintf(__fmul_rn(s_g, v[k].x));
      float qi = rintf(__fmul_rn(s_g, v[k].y));
      qr = fminf(fmaxf(qr, -127.f), 127.f);
      qi = fminf(fmaxf(qi, -127.f), 127.f);
      char2 q2;
      q2.x = static_cast<signed char>(qr);
      q2.y = static_cast<signed char>(qi);
      reinterpret_cast<char2*>(stg)[kp * G + g] = q2;
      if (a.out_f) {
        const long long o = ((static_cast<long long>(kp) * a.n_spec + s) * a.n_input + i0 + g);
        reinterpret_cast<float2*>(a.out_f)[o] = v[k];
      }
    }
  }
  __syncthreads();
  int8_t* dst0 = a.out_q + (static_cast<long long>(s) * a.n_input + i0) * 2;
  const long long row_stride = static_cast<long long>(a.n_spec) * a.n_input * 2;
  for (int idx = tid; idx < N * gv; idx += T) {
    const int kp = idx / gv, g = idx - kp * gv;
    *reinterpret_cast<char2*>(dst0 + kp * row_stride + 2 * g) = reinterpret_cast<const char2*>(stg)[kp * G + g];
  }
}

// Radix-16 Stockham kernel for N = 2^LOG2N >= 16 (fft.cuh's row passes): F
// FFTs of the group in flight (F N = 8192 points, 16 per thread; one FFT of
// 16384), exchange rows padded by one slot per 16 so the stride-16 writes of
// a pass hit distinct banks, every index split a shift.  The first pass
// unpacks the staged 4+4-bit samples; the bins come out in natural order and
// are requantised, fftshifted, into the staging rows.
template <int LOG2N>
struct P2Plan {
  static constexpr int N = 1 << LOG2N;
  static constexpr int F = N >= 8192 ? 1 : 8192 / N;
  static constexpr int THREADS = F * N / 16;
  static constexpr int LDP = N + N / 16;             // pad16(x) < LDP for x < N
};

template <int LOG2N>
__global__ void __launch_bounds__(P2Plan<LOG2N>::THREADS, 1024 / P2Plan<LOG2N>::THREADS)
k_upchan_p2(UpchanArgs a) {
  using P = P2Plan<LOG2N>;
  constexpr int N = P::N, F = P::F, LDP = P::LDP;
  extern __shared__ __align__(16) unsigned char smem[];
  const int G = a.group;
  float2* buf = reinterpret_cast<float2*>(smem);                                 // [F][LDP]
  uint8_t* raw = smem + static_cast<size_t>(F) * LDP * sizeof(float2);           // [N][G]
  int8_t* stg = reinterpret_cast<int8_t*>(raw + static_cast<size_t>(N) * G);     // [N][G][2]
  float* sc = reinterpret_cast<float*>(
      stg + ((static_cast<size_t>(N) * G * 2 + 15) & ~static_cast<size_t>(15)));  // [G]
  const int tid = threadIdx.x;
  const int T = blockDim.x;
  const int s = blockIdx.y;
  const int i0 = blockIdx.x * G;
  const int gv = min(G, a.n_input - i0);        // valid inputs in this group
  const long long row0 = static_cast<long long>(s) * N;
  {
    const uint8_t* src = a.volt + row0 * a.n_input + i0;
    if (gv == G && (G % 4) == 0 && (a.n_input % 4) == 0) {
      const int wpr = G / 4;
      for (int idx = tid; idx < N * wpr; idx += T) {
        const int n = idx / wpr, w = idx - n * wpr;
        reinterpret_cast<uint32_t*>(raw)[idx] =
            *reinterpret_cast<const uint32_t*>(src + static_cast<long long>(n) * a.n_input + 4 * w);
      }
    } else {
      for (int idx = tid; idx < N * G; idx += T) {
        const int n = idx / G, g = idx - n * G;
        raw[idx] = g < gv ? src[static_cast<long long>(n) * a.n_input + g] : 0;
      }
    }
    for (int g = tid; g < G; g += T) sc[g] = g < gv ? a.scale[i0 + g] : 0.0f;
  }
  __syncthreads();
  const int tw_stride = a.tw_n / N;
  auto tw = [&](int i) { return __ldg(a.tw + static_cast<long long>(i) * tw_stride); };
  for (int f0 = 0; f0 < G; f0 += F) {
    fft_rows_inplace_f<LOG2N>(
        buf, LDP,
        [&](int f, int x) {
          // high nibble real, low nibble imaginary (two's complement)
          float2 v = make_float2(0.f, 0.f);
          const int g = f0 + f;
          if (g < G) {
            const uint32_t byte = raw[x * G + g];
            v.x = static_cast<float>(static_cast<int>(static_cast<int8_t>(byte)) >> 4);
            v.y = static_cast<float>(static_cast<int>(static_cast<int8_t>(byte << 4)) >> 4);
          }
          return v;
        },
        tw);
    for (int idx = tid; idx < F * N; idx += T) {
      const int f = idx >> LOG2N, k = idx & (N - 1);
      const int g = f0 + f;
      if (g >= gv) continue;
      const float2 X = buf[f * LDP + pad16(k)];
      const float s_g = sc[g];
      const int kp = (k + N / 2) & (N - 1);
      float qr = rintf(__fmul_rn(s_g, X.x));
      float qi = rintf(__fmul_rn(s_g, X.y));
      qr = fminf(fmaxf(qr, -127.f), 127.f);
      qi = fminf(fmaxf(qi, -127.f), 127.f);
      char2 q2;
      q2.x = static_cast<signed char>(qr);
      q2.y = static_cast<signed char>(qi);
      reinterpret_cast<char2*>(stg)[kp * G + g] = q2;
      if (a.out_f) {
        const long long o = ((static_cast<long long>(kp) * a.n_spec + s) * a.n_input + i0 + g);
        reinterpret_cast<float2*>(a.out_f)[o] = X;
      }
    }
    __syncthreads();   // buf reused by the next F inputs; stg complete
  }
  {
    int8_t* dst0 = a.out_q + (static_cast<long long>(s) * a.n_input + i0) * 2;
    const long long row_stride = static_cast<long long>(a.n_spec) * a.n_input * 2;
    if (gv == G && (G % 2) == 0) {
      const int wpr = G / 2;           // 4-byte words per row
      for (int idx = tid; idx < N * wpr; idx += T) {
        const int kp = idx / wpr, w = idx - kp * wpr;
        *reinterpret_cast<uint32_t*>(dst0 + kp * row_stride + 4 * w) =
            reinterpret_cast<const uint32_t*>(stg)[idx];
      }
    } else {
      for (int idx = tid; idx < N * gv; idx += T) {
        const int kp = idx / gv, g = idx - kp * gv;
        *reinterpret_cast<char2*>(dst0 + kp * row_stride + 2 * g) =
            reinterpret_cast<const char2*>(stg)[kp * G + g];
      }
    }
  }
}

size_t smem_p2(int log2n, int G) {
  const int N = 1 << log2n;
  const int F = N >= 8192 ? 1 : 8192 / N;
  return static_cast<size_t>(F) * (N + N / 16) * 8 + static_cast<size_t>(N) * G +
         ((static_cast<size_t>(N) * G * 2 + 15) & ~static_cast<size_t>(15)) + 4 * G + 16;
}

size_t smem_for(int log2n, int G);

int group_for(int log2n, int n_input) {
  // G inputs per CTA: the most whose shared memory (raw G N + staging 2 G N +
  // exchange) fits one CTA per SM, at least F (wider groups coalesce the
  // G-byte row reads and 2G-byte row writes)
  const int F = log2n >= 13 ? 1 : (log2n < 4 ? 256 : (8192 >> log2n));
  const size_t budget = 200 * 1024;
  int G = 1;
  while (G < 64 && smem_for(log2n, 2 * G) <= budget) G *= 2;
  if (G < F) G = F;
  int np2 = 1;
  while (np2 < n_input) np2 *= 2;
  if (G > np2) G = np2;
  return G;
}

size_t smem_for(int log2n, int G) {
  if (log2n >= 4) return smem_p2(log2n, G);
  const int N = 1 << log2n;
  return static_cast<size_t>(N) * G + ((static_cast<size_t>(N) * G * 2 + 15) & ~static_cast<size_t>(15)) + 4 * G +
         16;
}

template <int L>
int launch_upchan_t(const UpchanArgs& a, cudaStream_t st) {
  const size_t sm = smem_for(L, a.group);
  dim3 grid((a.n_input + a.group - 1) / a.group, a.n_spec);
  if constexpr (L >= 4) {
    auto kern = k_upchan_p2<L>;
    OVRO_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm)));
    OVRO_PROF("k_upchan", st);
    kern<<<grid, P2Plan<L>::THREADS, sm, st>>>(a);
  } else {
    auto kern = k_upchan<L>;
    OVRO_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm)));
    OVRO_PROF("k_upchan", st);
    kern<<<grid, 256, sm, st>>>(a);
  }
  OVRO_LAUNCH_CHECK();
  return OVRO_OK;
}

int launch_upchan(int log2n, const UpchanArgs& a, cudaStream_t st) {
  switch (log2n) {
    case 1: return launch_upchan_t<1>(a, st);
    case 2: return launch_upchan_t<2>(a, st);
    case 3: return launch_upchan_t<3>(a, st);
    case 4: return launch_upchan_t<4>(a, st);
    case 5: return launch_upchan_t<5>(a, st);
    case 6: return launch_upchan_t<6>(a, st);
    case 7: return launch_upchan_t<7>(a, st);
    case 8: return launch_upchan_t<8>(a, st);
    case 9: return launch_upchan_t<9>(a, st);
    case 10: return launch_upchan_t<10>(a, st);
    case 11: return launch_upchan_t<11>(a, st);
    case 12: return launch_upchan_t<12>(a, st);
    case 13: return launch_upchan_t<13>(a, st);
    case 14: return launch_upchan_t<14>(a, st);
    default: return OVRO_ERR_UNSUPPORTED;
  }
}

// G inputs per CTA from the autotuner: every G with F <= G <= 64 whose shared
// memory fits (results do not depend on G).
int launch_upchan_tuned(int l, UpchanArgs a, cudaStream_t st) {
  const int F = l >= 13 ? 1 : (l < 4 ? 256 : (8192 >> l));
  int np2 = 1;
  while (np2 < a.n_input) np2 *= 2;
  const int g0 = group_for(l, a.n_input);
  std::vector<int> cands;
  for (int g = F; g <= 64; g *= 2) {
    if (g > np2 && g > F) break;
    if (smem_for(l, g) <= (size_t(227) << 10)) cands.push_back(g);
  }
  auto run = [&](int g) -> int {
    a.group = g;
    return launch_upchan(l, a, st);
  };
  const std::string key = tune_key("k_upchan", {l, a.n_input});
  int g = tuned(key, g0);
  if (tuning(st) && cands.size() > 1)
    if (int e = tune_pick(key, cands, run, st, &g)) return e;
  return run(g);
}

struct UpchanWs {
  unsigned long long* power;
  float* scale;
  double* user;
  double* h2;
  float2* tw;
};

UpchanWs carve_upchan(void* ws, size_t bytes, int n_input, int n_coarse, size_t* need) {
  Carver c(ws, bytes);
  UpchanWs w;
  w.power = c.take<unsigned long long>(static_cast<size_t>(n_input) * n_coarse);
  w.scale = c.take<float>(static_cast<size_t>(n_input) * n_coarse);
  w.user = c.take<double>(static_cast<size_t>(n_input) * n_coarse);
  w.h2 = c.take<double>(static_cast<size_t>(n_coarse));
  w.tw = c.take<float2>(kMaxN);
  *need = c.used;
  return w;
}

}  // namespace
}  // namespace ovro

extern "C" {

size_t ovro_upchan_workspace_size(int n_input, int n_coarse) {
  if (n_input <= 0 || n_coarse <= 0) return 0;
  size_t need = 0;
  ovro::carve_upchan(nullptr, 0, n_input, n_coarse, &need);
  return need;
}

int ovro_upchan_ex(const uint8_t* d_volt, int n_input, int n_coarse, int64_t n_time,
                   const int32_t* h_nfft, const double* h_scale_or_null, const ovro_upchan_options* opt,
                   int8_t* d_fine_q, float* d_fine_f32_or_null, void* d_ws, size_t ws_bytes, void* stream) {
  using namespace ovro;
  if (!d_volt || !h_nfft || !d_fine_q || n_input <= 0 || n_coarse <= 0 || n_time <= 0)
    return OVRO_ERR_INVALID_ARG;
  const bool taps = opt && opt->h_taps;
  const int n_tap = opt ? opt->n_taps : 1;
  const int lo = opt ? opt->chan_lo : 0;
  const int cnt_opt = opt ? opt->chan_count : 0;
  if (n_tap < 1 || (n_tap > 1 && !taps) || lo < 0 || cnt_opt < 0) return OVRO_ERR_INVALID_ARG;
  struct Coarse {
    int n, cnt, k;
    bool mixed;
  };
  std::vector<Coarse> cs(n_coarse);
  int max_pow2 = 2;
  for (int c = 0; c < n_coarse; ++c) {
    Coarse& e = cs[c];
    e.n = h_nfft[c];
    if (e.n <= 0) return OVRO_ERR_INVALID_ARG;
    if (taps && !opt->h_taps[c]) return OVRO_ERR_INVALID_ARG;
    const long long blocks = n_time / e.n;
    const long long k = blocks - n_tap + 1;
    if (k < 1 || k > INT32_MAX) return OVRO_ERR_UNSUPPORTED;
    e.k = static_cast<int>(k);
    e.cnt = cnt_opt ? cnt_opt : e.n;
    if (static_cast<long long>(lo) + e.cnt > e.n) return OVRO_ERR_INVALID_ARG;
    e.mixed = taps || lo != 0 || e.cnt != e.n || !is_pow2(e.n) || e.n > kMaxN || k > 65535;
    if (e.mixed) {
      MrPlan plan;
      int group = 0;
      size_t smem = 0;
      if (!mr_plan(e.n, n_input, taps ? n_tap : 1, e.cnt, &plan, &group, &smem)) return OVRO_ERR_UNSUPPORTED;
    } else {
      if (e.n < 2) return OVRO_ERR_UNSUPPORTED;
      max_pow2 = std::max(max_pow2, e.n);
    }
  }
  size_t need = 0;
  UpchanWs w = carve_upchan(d_ws, ws_bytes, n_input, n_coarse, &need);
  if (int e = check_workspace(d_ws, ws_bytes, need)) return e;
  cudaStream_t st = as_stream(stream);

  const size_t nsc = static_cast<size_t>(n_input) * n_coarse;
  if (h_scale_or_null) {
    OVRO_CUDA_TRY(cudaMemcpyAsync(w.user, h_scale_or_null, nsc * sizeof(double),
                                  cudaMemcpyHostToDevice, st));
  } else {
    OVRO_CUDA_TRY(cudaMemsetAsync(w.power, 0, nsc * sizeof(unsigned long long), st));
  }
  int table_n = 0;   // omega_{table_n}^k currently in w.tw
  long long q_off = 0;
  for (int c = 0; c < n_coarse; ++c) {
    const Coarse& e = cs[c];
    const int n = e.n;
    const long long n_used = (n_time / n) * n;
    if (!h_scale_or_null) {
      const int vw = (n_input % 16 == 0) ? 16 : ((n_input % 4 == 0) ? 4 : 1);
      const int nvec = (n_input + vw - 1) / vw;
      const int threads = nvec >= 256 ? 256 : ((nvec + 31) / 32) * 32;
      const long long rows = n_used < 8LL * num_sms() ? n_used : 8LL * num_sms();
      dim3 grid(static_cast<unsigned>(rows), (nvec + threads - 1) / threads);
      const uint8_t* vc = d_volt + static_cast<long long>(c) * n_time * n_input;
      unsigned long long* pc = w.power + static_cast<size_t>(c) * n_input;
      if (vw == 16)
        k_power<16><<<grid, threads, 0, st>>>(vc, n_input, n_used, pc);
      else if (vw == 4)
        k_power<4><<<grid, threads, 0, st>>>(vc, n_input, n_used, pc);
      else
        k_power<1><<<grid, threads, 0, st>>>(vc, n_input, n_used, pc);
      OVRO_LAUNCH_CHECK();
      if (taps) {
        k_sumsq<<<1, 256, 0, st>>>(opt->h_taps[c], n_tap * n, w.h2 + c);
        OVRO_LAUNCH_CHECK();
      }
    }
    k_scale<<<(n_input + 255) / 256, 256, 0, st>>>(
        w.power + static_cast<size_t>(c) * n_input,
        h_scale_or_null ? w.user + static_cast<size_t>(c) * n_input : nullptr, n_input, n,
        n_used, taps ? w.h2 + c : nullptr, w.scale + static_cast<size_t>(c) * n_input);
    OVRO_LAUNCH_CHECK();

    // twiddles: exactly omega_N for the mixed-radix kernel; any power-of-two
    // table at least N long for the radix-16 kernel
    const int want = e.mixed ? n : max_pow2;
    const bool ok = e.mixed ? table_n == n : (is_pow2(table_n) && table_n >= n);
    if (!ok) {
      k_twiddle<<<(want + 255) / 256, 256, 0, st>>>(w.tw, want);
      OVRO_LAUNCH_CHECK();
      table_n = want;
    }

    UpchanArgs a;
    a.volt = d_volt + static_cast<long long>(c) * n_time * n_input;
    a.tw = w.tw;
    a.scale = w.scale + static_cast<size_t>(c) * n_input;
    a.out_q = d_fine_q + q_off;
    a.out_f = d_fine_f32_or_null ? d_fine_f32_or_null + q_off : nullptr;
    a.n_input = n_input;
    a.n_spec = e.k;
    a.tw_n = table_n;
    a.taps = taps ? opt->h_taps[c] : nullptr;
    a.n_tap = taps ? n_tap : 1;
    a.chan_lo = lo;
    a.chan_cnt = e.cnt;
    if (e.mixed) {
      if (int err = launch_upchan_mr(a, a.n_tap, st)) return err;
    } else {
      if (int err = launch_upchan_tuned(ilog2(n), a, st)) return err;
    }
    q_off += static_cast<long long>(e.cnt) * e.k * n_input * 2;
  }
  return OVRO_OK;
}

int ovro_upchan(const uint8_t* d_volt, int n_input, int n_coarse, int64_t n_time,
                const int32_t* h_nfft, const double* h_scale_or_null, int8_t* d_fine_q,
                float* d_fine_f32_or_null, void* d_ws, size_t ws_bytes, void* stream) {
  return ovro_upchan_ex(d_volt, n_input, n_coarse, n_time, h_nfft, h_scale_or_null, nullptr, d_fine_q,
                        d_fine_f32_or_null, d_ws, ws_bytes, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of ovro_upchan.
//
// Some callers cannot call cudaMalloc at all: a plugin hosted by a framework
// that owns the whole device heap, or a real-time acquisition loop where an
// allocation (which may synchronise the device) would stall the other streams.
// They get ovro_upchan_noalloc, whose scratch (the per-input power sums and
// scales, and the twiddle table) lives in the fixed array below.  Every GPU
// that loads this library holds the array until the process exits.
namespace ovro {
namespace {

constexpr size_t kNoAllocScratchBytes = 1u << 20;   // 1 MiB
static __device__ __align__(256) unsigned char g_upchan_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices];     // device address per device, once found

// Device address of the scratch array for the current device (host code must
// not use the symbol itself as a device address).  Only a successful lookup
// is kept: after a failure (say, a first call made during a stream capture)
// the next call looks again.
int noalloc_scratch(void** out) {
  int dev = 0;
  OVRO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return OVRO_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_upchan_scratch);
    if (e != cudaSuccess) {
      set_last_error("cudaGetSymbolAddress(g_upchan_scratch)", e);
      return OVRO_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return OVRO_OK;
}

}  // namespace
}  // namespace ovro

extern "C" {

int ovro_upchan_noalloc(const uint8_t* d_volt, int n_input, int n_coarse, int64_t n_time,
                        const int32_t* h_nfft, const double* h_scale_or_null, int8_t* d_fine_q,
                        float* d_fine_f32_or_null, void* stream) {
  using namespace ovro;
  if (n_input <= 0 || n_coarse <= 0) return OVRO_ERR_INVALID_ARG;
  const size_t need = ovro_upchan_workspace_size(n_input, n_coarse);
  if (need > kNoAllocScratchBytes) {
    snprintf_last_error("ovro_upchan_noalloc: n_input * n_coarse needs %zu bytes of scratch, "
                        "more than the fixed %zu", need, kNoAllocScratchBytes);
    return OVRO_ERR_CAPACITY;
  }
  void* scratch = nullptr;
  if (int e = noalloc_scratch(&scratch)) return e;
  return ovro_upchan(d_volt, n_input, n_coarse, n_time, h_nfft, h_scale_or_null, d_fine_q,
                     d_fine_f32_or_null, scratch, kNoAllocScratchBytes, stream);
}

}  // extern "C"
