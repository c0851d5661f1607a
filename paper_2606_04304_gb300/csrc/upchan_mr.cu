// a1-a3 for N = 2^a 3^b 5^c: the mixed-radix upchannelizer kernel, with the
// polyphase-filter-bank and fine-channel-window options (Section 2.1).
#include <algorithm>

#include "common.cuh"
#include "mixed_radix.cuh"
#include "tune.h"
#include "upchan_impl.h"

namespace ovro {
namespace {

// N = 2^a 3^b 5^c (even), N <= 8192, such as the paper's 2400 = 16 x 15 x 10.
// One CTA handles one spectrum of G adjacent inputs, F of them at a time.  The
// packed rows of the P N samples the spectrum needs are staged in shared
// memory; pass 0 forms the polyphase sums y_n = sum_p h[p N + n] x[(s+p) N + n]
// (the bare samples when P = 1 and there are no taps) and runs its radix-R0
// DFTs; every further pass is a Stockham auto-sort step through a padded
// exchange buffer (twiddles from an omega_N table); the last pass requantises
// the fine channels inside [chan_lo, chan_lo + chan_cnt) of the fftshifted
// axis into a staging tile, written out as rows of 2G bytes.  Each thread owns
// up to 16 complex values per pass: 16 / R butterflies of radix R.
constexpr int kMrVals = 16;
constexpr int kMrThreads = 512;

// exchange-buffer index with one pad slot per 16: strided radix-16 stores hit
// 16 different bank pairs
__device__ __forceinline__ int mr_pad(int i) { return i + (i >> 4); }

// Per-pass constants of the plan, kept in shared memory (hdr).
constexpr int kMrHdrInts = 32;                 // [0] threads, [1 + p] radix, [9 + p] N / radix
constexpr int kMrHdrBytes = kMrHdrInts * 4;

struct MrSmem {
  const int* hdr;
  float2* buf;              // [F N] padded
  const uint8_t* raw;       // [P N][G] packed samples
  char2* stg;               // [chan_cnt][G]
  const float* sc;          // [G]
};

template <int R>
__device__ __forceinline__ void mr_pass(const UpchanArgs& a, const MrSmem& m, int N, int F, int f0, int gv,
                                        int s, int Ns, int p_idx, bool first, bool last) {
  constexpr int C = kMrVals / R;            // butterflies per thread
  const int T = m.hdr[0];
  const int tid = threadIdx.x;
  const int G = a.group;
  const int nbf = m.hdr[9 + p_idx];         // N / R butterflies per FFT
  const int total = F * nbf;
  float2 v[C][R];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int gb = tid + c * T;
    if (gb >= total) continue;
    const int f = gb / nbf, j = gb - f * nbf;
    if (first) {
      const int g = f0 + f;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int n = j + r * nbf;
        float2 x = make_float2(0.f, 0.f);
        if (g < G) {
          if (a.taps) {
            for (int p = 0; p < a.n_tap; ++p) {
              const uint32_t byte = m.raw[(p * N + n) * G + g];
              const float h = __ldg(a.taps + p * N + n);
              x.x = fmaf(h, static_cast<float>(static_cast<int>(static_cast<int8_t>(byte)) >> 4), x.x);
              x.y = fmaf(h, static_cast<float>(static_cast<int>(static_cast<int8_t>(byte << 4)) >> 4), x.y);
            }
          } else {
            const uint32_t byte = m.raw[n * G + g];
            x.x = static_cast<float>(static_cast<int>(static_cast<int8_t>(byte)) >> 4);
            x.y = static_cast<float>(static_cast<int>(static_cast<int8_t>(byte << 4)) >> 4);
          }
        }
        v[c][r] = x;
      }
    } else {
      const int base = f * N + j;
#pragma unroll
      for (int r = 0; r < R; ++r) v[c][r] = m.buf[mr_pad(base + r * nbf)];
      const int k = j % Ns;
      const int step = k * (N / (Ns * R));  // omega_{Ns R}^{r k} = omega_N^{r step}
#pragma unroll
      for (int r = 1; r < R; ++r) v[c][r] = mr::mul(v[c][r], __ldg(a.tw + r * step));
    }
    mr::dft<R>(v[c]);
  }
  if (!first) __syncthreads();              // every read of this pass done before the writes
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int gb = tid + c * T;
    if (gb >= total) continue;
    const int f = gb / nbf, j = gb - f * nbf;
    const int k = j % Ns;
    const int q0 = (j - k) * R + k;         // (j / Ns) Ns R + k
    if (!last) {
#pragma unroll
      for (int r = 0; r < R; ++r) m.buf[mr_pad(f * N + q0 + r * Ns)] = v[c][r];
    } else {
      const int g = f0 + f;
      if (g >= gv) continue;
      const float s_g = m.sc[g];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        int kp = q0 + r * Ns + (N >> 1);    // fftshift
        if (kp >= N) kp -= N;
        const int idx = kp - a.chan_lo;
        if (idx < 0 || idx >= a.chan_cnt) continue;
        const float2 X = v[c][r];
        float qr = rintf(__fmul_rn(s_g, X.x));
        float qi = rintf(__fmul_rn(s_g, X.y));
        qr = fminf(fmaxf(qr, -127.f), 127.f);
        qi = fminf(fmaxf(qi, -127.f), 127.f);
        char2 q2;
        q2.x = static_cast<signed char>(qr);
        q2.y = static_cast<signed char>(qi);
        m.stg[idx * G + g] = q2;
        if (a.out_f) {
          const long long o = (static_cast<long long>(idx) * a.n_spec + s) * a.n_input + (blockIdx.x * G + g);
          reinterpret_cast<float2*>(a.out_f)[o] = X;
        }
      }
    }
  }
  __syncthreads();
}

__host__ __device__ constexpr unsigned radix_bit(int r) { return 1u << r; }
constexpr unsigned kMrAll = radix_bit(2) | radix_bit(3) | radix_bit(4) | radix_bit(5) | radix_bit(6) |
                            radix_bit(8) | radix_bit(10) | radix_bit(12) | radix_bit(15) | radix_bit(16);

// SET: the radices this instantiation handles (a bit per radix).  Every radix
// compiled in keeps some registers busy, so the common schedules get kernels
// with just their own radices; kMrAll serves every other length.  MINB: CTAs
// per SM the register allocation leaves room for (the autotuner picks 1 or 2).
template <unsigned SET, int MINB>
__global__ void __launch_bounds__(kMrThreads, MINB) k_upchan_mr(UpchanArgs a, MrPlan pl) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = pl.n;
  const int F = pl.f;
  const int G = a.group;
  const int P = a.taps ? a.n_tap : 1;
  const int tid = threadIdx.x;
  const int T = blockDim.x;
  const int i0 = blockIdx.x * G;
  const int gv = min(G, a.n_input - i0);
  MrSmem m;
  int* hdr = reinterpret_cast<int*>(smem);
  m.hdr = hdr;
  m.buf = reinterpret_cast<float2*>(smem + kMrHdrBytes);
  const size_t buf_bytes = (static_cast<size_t>(mr_pad(F * N - 1) + 1) * sizeof(float2) + 15) & ~size_t(15);
  uint8_t* raw = smem + kMrHdrBytes + buf_bytes;
  const size_t raw_bytes = (static_cast<size_t>(P) * N * G + 15) & ~size_t(15);
  char2* stg = reinterpret_cast<char2*>(raw + raw_bytes);
  const size_t stg_bytes = (static_cast<size_t>(a.chan_cnt) * G * 2 + 15) & ~size_t(15);
  float* sc = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(stg) + stg_bytes);
  m.raw = raw;
  m.stg = stg;
  m.sc = sc;
  for (int g = tid; g < G; g += T) sc[g] = g < gv ? a.scale[i0 + g] : 0.0f;
  if (tid == 0) hdr[0] = T;
  if (tid < kMrMaxPass) {
    const int r = tid < pl.n_pass ? pl.radix[tid] : 1;
    hdr[1 + tid] = r;
    hdr[9 + tid] = N / r;
  }

  for (int s = blockIdx.y; s < a.n_spec; s += gridDim.y) {
    // stage the P N packed rows of this spectrum (G bytes each)
    const uint8_t* src = a.volt + static_cast<long long>(s) * N * a.n_input + i0;
    const int rows = P * N;
    if (gv == G && (G % 4) == 0 && (a.n_input % 4) == 0) {
      const int wpr = G / 4;
      for (int idx = tid; idx < rows * wpr; idx += T) {
        const int n = idx / wpr, w = idx - n * wpr;
        reinterpret_cast<uint32_t*>(raw)[idx] =
            __ldg(reinterpret_cast<const uint32_t*>(src + static_cast<long long>(n) * a.n_input + 4 * w));
      }
    } else if (gv == G && G == 2 && (a.n_input % 2) == 0) {
      for (int n = tid; n < rows; n += T)
        reinterpret_cast<uint16_t*>(raw)[n] =
            __ldg(reinterpret_cast<const unsigned short*>(src + static_cast<long long>(n) * a.n_input));
    } else {
      for (int idx = tid; idx < rows * G; idx += T) {
        const int n = idx / G, g = idx - n * G;
        raw[idx] = g < gv ? src[static_cast<long long>(n) * a.n_input + g] : 0;
      }
    }
    __syncthreads();

    for (int f0 = 0; f0 < G; f0 += F) {
      int Ns = 1;
      for (int p = 0; p < pl.n_pass; ++p) {
        const bool first = p == 0, last = p == pl.n_pass - 1;
        const int r = hdr[1 + p];
        if constexpr ((SET & radix_bit(16)) != 0) if (r == 16) mr_pass<16>(a, m, N, F, f0, gv, s, Ns, p, first, last);
        if constexpr ((SET & radix_bit(15)) != 0) if (r == 15) mr_pass<15>(a, m, N, F, f0, gv, s, Ns, p, first, last);
        if constexpr ((SET & radix_bit(12)) != 0) if (r == 12) mr_pass<12>(a, m, N, F, f0, gv, s, Ns, p, first, last);
        if constexpr ((SET & radix_bit(10)) != 0) if (r == 10) mr_pass<10>(a, m, N, F, f0, gv, s, Ns, p, first, last);
        if constexpr ((SET & radix_bit(8)) != 0) if (r == 8) mr_pass<8>(a, m, N, F, f0, gv, s, Ns, p, first, last);
        if constexpr ((SET & radix_bit(6)) != 0) if (r == 6) mr_pass<6>(a, m, N, F, f0, gv, s, Ns, p, first, last);
        if constexpr ((SET & radix_bit(5)) != 0) if (r == 5) mr_pass<5>(a, m, N, F, f0, gv, s, Ns, p, first, last);
        if constexpr ((SET & radix_bit(4)) != 0) if (r == 4) mr_pass<4>(a, m, N, F, f0, gv, s, Ns, p, first, last);
        if constexpr ((SET & radix_bit(3)) != 0) if (r == 3) mr_pass<3>(a, m, N, F, f0, gv, s, Ns, p, first, last);
        if constexpr ((SET & radix_bit(2)) != 0) if (r == 2) mr_pass<2>(a, m, N, F, f0, gv, s, Ns, p, first, last);
        Ns *= r;
      }
    }

    // the staged int8 rows: fine channel idx is 2 gv contiguous bytes
    int8_t* dst0 = a.out_q + (static_cast<long long>(s) * a.n_input + i0) * 2;
    const long long row_stride = static_cast<long long>(a.n_spec) * a.n_input * 2;
    const int cnt = a.chan_cnt;
    if (gv == G && (G % 2) == 0 && (a.n_input % 2) == 0) {
      const int wpr = G / 2;
      for (int idx = tid; idx < cnt * wpr; idx += T) {
        const int kp = idx / wpr, w = idx - kp * wpr;
        *reinterpret_cast<uint32_t*>(dst0 + kp * row_stride + 4 * w) = reinterpret_cast<const uint32_t*>(stg)[idx];
      }
    } else {
      for (int idx = tid; idx < cnt * gv; idx += T) {
        const int kp = idx / gv, g = idx - kp * gv;
        *reinterpret_cast<char2*>(dst0 + kp * row_stride + 2 * g) = stg[kp * G + g];
      }
    }
    __syncthreads();                          // raw / stg reused by the next spectrum
  }
}

size_t mr_smem(int n, int f, int g, int p, int cnt) {
  const size_t buf = (static_cast<size_t>((f * n - 1) + ((f * n - 1) >> 4) + 1) * 8 + 15) & ~size_t(15);
  const size_t raw = (static_cast<size_t>(p) * n * g + 15) & ~size_t(15);
  const size_t stg = (static_cast<size_t>(cnt) * g * 2 + 15) & ~size_t(15);
  return kMrHdrBytes + buf + raw + stg + 4 * static_cast<size_t>(g);
}

// Radix schedule for even N = 2^a 3^b 5^c: 15 = 3 x 5 while both remain, then
// 10 = 2 x 5 or 5, 12 = 4 x 3 / 6 = 2 x 3 / 3, then 16s and one of 8, 4, 2.
// Returns false for other N.
bool mr_radices(int n, int* radix, int* n_pass) {
  if (n < 2 || (n & 1)) return false;
  int a = 0, b = 0, c = 0, x = n;
  while (x % 2 == 0) { x /= 2; ++a; }
  while (x % 3 == 0) { x /= 3; ++b; }
  while (x % 5 == 0) { x /= 5; ++c; }
  if (x != 1) return false;
  int np = 0;
  auto push = [&](int r) {
    if (np < kMrMaxPass) radix[np] = r;
    ++np;
  };
  // 16s first, keeping the twos that pair with leftover fives (10) and threes (12)
  const int e5 = c > b ? c - b : 0, e3 = b > c ? b - c : 0;
  const int keep = std::min(a, e5 + 2 * e3);
  while (a - 4 >= keep) {
    push(16);
    a -= 4;
  }
  while (b > 0 && c > 0) { push(15); --b; --c; }
  while (c > 0) {
    if (a >= 1) { push(10); --a; } else push(5);
    --c;
  }
  while (b > 0) {
    if (a >= 2) { push(12); a -= 2; } else if (a >= 1) { push(6); --a; } else push(3);
    --b;
  }
  while (a >= 4) { push(16); a -= 4; }
  if (a == 3) push(8);
  if (a == 2) push(4);
  if (a == 1) push(2);
  *n_pass = np;
  return np <= kMrMaxPass;
}

int mr_threads(int n, int f, const int* radix, int n_pass) {
  int t = 0;
  for (int p = 0; p < n_pass; ++p) {
    const int per = kMrVals / radix[p];
    const int need = (f * (n / radix[p]) + per - 1) / per;
    if (need > t) t = need;
  }
  return (t + 31) / 32 * 32;
}

// F FFTs in flight and G inputs per CTA: the largest F with at most
// kMrThreads threads, then the largest G (a multiple of F, at most 8) whose
// shared memory lets two CTAs share an SM, else one.
bool mr_plan_impl(int n, int n_input, int p, int cnt, MrPlan* pl, int* group, size_t* smem) {
  if (n > kMrMaxN || !mr_radices(n, pl->radix, &pl->n_pass)) return false;
  pl->n = n;
  pl->f = 0;
  for (int f = 4; f >= 1; f /= 2) {
    const int t = mr_threads(n, f, pl->radix, pl->n_pass);
    if (t <= kMrThreads) {
      pl->f = f;
      pl->threads = t;
      break;
    }
  }
  if (!pl->f) return false;
  int np2 = 1;
  while (np2 < n_input) np2 *= 2;
  for (const size_t budget : {size_t(110) << 10, size_t(220) << 10}) {
    for (int g = 8; g >= 1; g /= 2) {
      if (g > np2 && g > 1) continue;
      const int f = std::min(pl->f, g);
      const size_t sm = mr_smem(n, f, g, p, cnt);
      if (sm <= budget) {
        pl->f = f;
        pl->threads = mr_threads(n, f, pl->radix, pl->n_pass);
        *group = g;
        *smem = sm;
        return true;
      }
    }
  }
  return false;
}

template <unsigned SET, int MINB>
int launch_mr_set(const UpchanArgs& a, const MrPlan& pl, size_t smem, cudaStream_t st) {
  auto kern = k_upchan_mr<SET, MINB>;
  OVRO_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  dim3 grid((a.n_input + a.group - 1) / a.group, std::min(a.n_spec, 65535));
  OVRO_PROF("k_upchan_mr", st);
  kern<<<grid, pl.threads, smem, st>>>(a, pl);
  OVRO_LAUNCH_CHECK();
  return OVRO_OK;
}

constexpr unsigned k2400 = radix_bit(16) | radix_bit(15) | radix_bit(10);   // 2400 = 16 x 15 x 10
constexpr unsigned kPow2a = radix_bit(16) | radix_bit(2);
constexpr unsigned kPow2b = radix_bit(16) | radix_bit(4);
constexpr unsigned kPow2c = radix_bit(16) | radix_bit(8);

unsigned radix_set(const MrPlan& pl) {
  unsigned set = 0;
  for (int p = 0; p < pl.n_pass; ++p) set |= radix_bit(pl.radix[p]);
  return set;
}

bool has_minb2(unsigned set) { return set == k2400 || set == kPow2a; }

int launch_shape(const UpchanArgs& a, const MrPlan& pl, size_t smem, int minb, cudaStream_t st) {
  const unsigned set = radix_set(pl);
  if (minb == 2 && set == k2400) return launch_mr_set<k2400, 2>(a, pl, smem, st);
  if (minb == 2 && set == kPow2a) return launch_mr_set<kPow2a, 2>(a, pl, smem, st);
  switch (set) {
    case k2400: return launch_mr_set<k2400, 1>(a, pl, smem, st);
    case kPow2a: return launch_mr_set<kPow2a, 1>(a, pl, smem, st);
    case kPow2b: return launch_mr_set<kPow2b, 1>(a, pl, smem, st);
    case kPow2c: return launch_mr_set<kPow2c, 1>(a, pl, smem, st);
    case radix_bit(16): return launch_mr_set<radix_bit(16), 1>(a, pl, smem, st);
    default: return launch_mr_set<kMrAll, 1>(a, pl, smem, st);
  }
}

// The plan for G inputs per CTA (F = min(largest F within the thread limit, G)).
bool mr_shape(int n, int g, int p, int cnt, const MrPlan& base, int f_max, MrPlan* pl, size_t* smem) {
  *pl = base;
  pl->f = std::min(f_max, g);
  pl->threads = mr_threads(n, pl->f, pl->radix, pl->n_pass);
  *smem = mr_smem(n, pl->f, g, p, cnt);
  return pl->threads <= kMrThreads && *smem <= (size_t(220) << 10);
}

}  // namespace

bool mr_plan(int n, int n_input, int p, int cnt, MrPlan* pl, int* group, size_t* smem) {
  return mr_plan_impl(n, n_input, p, cnt, pl, group, smem);
}

// Shape: G inputs per CTA and the register budget (1 or 2 CTAs per SM), from
// the autotuner (every shape computes the same values in the same order).
int launch_upchan_mr(const UpchanArgs& a_in, int n_tap, cudaStream_t st) {
  const int n = a_in.tw_n;
  MrPlan base;
  int g0 = 1;
  size_t sm0 = 0;
  if (!mr_plan_impl(n, a_in.n_input, n_tap, a_in.chan_cnt, &base, &g0, &sm0)) return OVRO_ERR_UNSUPPORTED;
  int f_max = 0;
  for (int f = 4; f >= 1 && !f_max; f /= 2)
    if (mr_threads(n, f, base.radix, base.n_pass) <= kMrThreads) f_max = f;
  int np2 = 1;
  while (np2 < a_in.n_input) np2 *= 2;
  std::vector<int> cands;
  const bool two = has_minb2(radix_set(base));
  for (int g = 1; g <= 8; g *= 2) {
    if (g > np2 && g > 1) break;
    MrPlan pl;
    size_t sm = 0;
    if (!mr_shape(n, g, n_tap, a_in.chan_cnt, base, f_max, &pl, &sm)) continue;
    cands.push_back(g * 4 + 1);
    if (two) cands.push_back(g * 4 + 2);
  }
  auto run = [&](int c) -> int {
    UpchanArgs a = a_in;
    a.group = c / 4;
    MrPlan pl;
    size_t sm = 0;
    if (!mr_shape(n, a.group, n_tap, a.chan_cnt, base, f_max, &pl, &sm)) return OVRO_ERR_UNSUPPORTED;
    return launch_shape(a, pl, sm, c % 4, st);
  };
  const std::string key = tune_key("k_upchan_mr", {n, a_in.n_input, n_tap, a_in.chan_cnt});
  int choice = tuned(key, g0 * 4 + 1);
  if (tuning(st) && cands.size() > 1)
    if (int e = tune_pick(key, cands, run, st, &choice)) return e;
  return run(choice);
}

}  // namespace ovro
