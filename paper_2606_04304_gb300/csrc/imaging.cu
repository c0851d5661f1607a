// a5-a7: uvw, prolate-spheroidal gridding and dirty imaging per fine channel.
//
// Section 2.2 of the paper images every fine channel over the visible
// hemisphere; the dirty images are the search product.  Per channel:
//
//  a5  u = (x_a - x_b) s_nu in grid cells with s_nu = nu / (c du): one
//      correctly rounded FP64 multiply per coordinate, then rounded to 1/Q
//      cell.  GB300's FP64 pipe is narrow, so the kernels evaluate it as a
//      float-float product and only falls back to a real FP64 multiply when
//      the float-float bound cannot decide rint(u Q) (|frac - 1/2| within the
//      error bound) -- the integer result equals the FP64 definition exactly.
//  a6  Stokes I = (XX + YY)/2 of each kept cross baseline is gridded once (the
//      mirror conj(V) at (-u, -v) is accounted for by taking 2 Re of the
//      transform, which is exact because the mirror's footprint is the point
//      reflection), with a separable 7 x 7 prolate-spheroidal kernel.  The uv
//      position of a baseline moves by a fraction of a cell across a call's
//      channels, so the host lists, once per call, the baselines that can
//      touch each band of grid rows; k_grid_rows then works on one
//      (channel, band): exact uv, keep test, shared-memory atomics into the
//      band, and the band's row FFTs in place.
//  a7  The uv grid is padded by 2 (G = 2N cells a side, du = 1 / (G cell)) and
//      the image is the central N x N of its transform, as padded imagers do:
//      the horizon then sits where the kernel's transform is still > 0.25, so
//      the grid correction does not amplify FP32 round-off.  k_grid_rows keeps
//      only the N central columns of its row transforms; k_fft_cols
//      transforms those columns, keeps the N central rows, and applies the
//      (-1)^(r+c) centring sign, normalisation, grid correction and horizon
//      mask while writing the image.  The (-1)^(ku+kv) centring sign is
//      applied at gridding time, and the exp(+) transform is a forward
//      transform of the conjugated grid.  Channel batches keep the
//      intermediate half-transformed grids L2-sized.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "fft.cuh"
#include "pswf.h"
#include "stages.h"
#include "tune.h"

namespace ovro {
namespace {

constexpr double kCLight = 299792458.0;
constexpr int kQ = kOversample;
constexpr int kHalfTab = kSupport * kOversample / 2;
constexpr int kTabLen = 2 * kHalfTab + 1;
constexpr int kHalfSup = kSupport / 2;
constexpr int kPad = 2;              // uv grid cells per image pixel, per axis
// storage of the half-transformed grid between the row and column passes
constexpr int kStoreF32 = OVRO_STORE_FP32, kStoreBF16 = OVRO_STORE_BF16, kStoreF16 = OVRO_STORE_FP16;

struct Baseline {
  double dx, dy;
  float dxh, dxl, dyh, dyl;
  long long bl;
};

struct ChanScale {
  double s;          // s_nu * Q
  double nu_c;       // nu / c (wavelengths per metre)
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
  c.nu_c = freq[f] / kCLight;
  c.sh = static_cast<float>(c.s);
  c.sl = static_cast<float>(c.s - static_cast<double>(c.sh));
  out[f] = c;
}

// rint(fl64(x * s)) decided in FP32: a float-float product, exact unless the
// fractional part is within the error bound (1.2e-7) of 1/2 or |x s| >= 2^21;
// returns false in those (rare) cases, where the FP64 product must be taken.
__device__ __forceinline__ bool fast_rint_prod(float xh, float xl, const ChanScale& s, long long* p) {
  const float hi = __fmul_rn(xh, s.sh);
  if (!(fabsf(hi) < 2097152.0f)) return false;
  const float e = __fmaf_rn(xh, s.sh, -hi);           // exact error of hi
  const float t = __fmaf_rn(xh, s.sl, __fmaf_rn(xl, s.sh, e));
  const float n = rintf(hi);
  const float f = __fadd_rn(hi - n, t);              // x s - n, |error| < 1.2e-7
  if (fabsf(fabsf(f) - 0.5f) <= 2.5e-7f) return false;
  long long q = static_cast<long long>(n);
  if (f > 0.5f) ++q;
  else if (f < -0.5f) --q;
  *p = q;
  return true;
}

__device__ __forceinline__ long long exact_rint_prod(double x, float xh, float xl, const ChanScale& s) {
  long long p;
  if (fast_rint_prod(xh, xl, s, &p)) return p;
  return __double2ll_rn(__dmul_rn(x, s.s));
}

// The same decision in 32-bit integers (|x s| < 2^21 is required anyway).
__device__ __forceinline__ bool fast_rint_prod32(float xh, float xl, const ChanScale& s, int* p) {
  const float hi = __fmul_rn(xh, s.sh);
  if (!(fabsf(hi) < 2097152.0f)) return false;
  const float e = __fmaf_rn(xh, s.sh, -hi);
  const float t = __fmaf_rn(xh, s.sl, __fmaf_rn(xl, s.sh, e));
  const float n = rintf(hi);
  const float f = __fadd_rn(hi - n, t);
  if (fabsf(fabsf(f) - 0.5f) <= 2.5e-7f) return false;
  *p = __float2int_rn(n) + (f > 0.5f ? 1 : 0) - (f < -0.5f ? 1 : 0);   // n is integral, |n| < 2^21
  return true;
}

static_assert(kQ == 1024, "centre_cell32 divides by shifting");
__device__ __forceinline__ void centre_cell32(int p, int& c0, int& off) {
  const int c = (abs(p) + kQ / 2) >> 10;
  c0 = p < 0 ? -c : c;
  off = p - c0 * kQ;
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

struct GridEntry {
  int bl;            // baseline index in the visibility record
  int cross;         // cross-baseline index (FP64 fallback, baseline length)
  int a;             // antennas a < b
  int bf;            // b | kCheckUv when the uv range must be decided per channel
  float dxh, dxl, dyh, dyl;
};
constexpr int kCheckUv = 1 << 16;

// Calibration and baseline-selection options of one gridding call.
struct GridOpts {
  const float2* gains;      // [n_chan][n_input] corrections or nullptr
  int n_input;
  const double* blen;       // [n_cross] baseline lengths, metres (FP64)
  double uv_min, uv_max;    // wavelengths, [uv_min, uv_max)
};

// Row pitch of a shared-memory grid band: G + G/16 pad slots, rounded so the
// pitch is 7 (mod 16) float2 -- consecutive rows then start 14 banks apart and
// the 7 rows of one kernel footprint, or 16 consecutive transposed columns, hit
// distinct banks.
__host__ __device__ constexpr int band_pitch(int g) { return (g + g / 16) + ((7 - (g + g / 16) % 16) + 16) % 16; }

// Gridding records per chunk (one per prepared visibility).
constexpr int kRecMax = 512;
constexpr int kWuStride = 5;       // float2 per record: (w_t, w_{t+4}), t < 4; odd word stride
constexpr int kWvStride = 9;       // floats per record: w_t, t < 8 (w_7 = 0)

// Planar row pitch of a band during gridding: G + 4 floats, so that the 7 rows
// x 4 columns of one footprint quarter fall in 28 distinct banks.
__host__ __device__ constexpr int planar_pitch(int g) { return g + 4; }

// One band of grid rows of one channel: grid in shared memory, row FFTs in
// place, central N columns written to h ([batch][G][N]).  The band's candidate
// list is taken in chunks of blockDim/2 visibilities; a pair of threads
// prepares one (exact u on the even thread, exact v on the odd one, the keep
// test, the seven separable weights of each axis with the centring sign, and
// Stokes I), then every warp takes whole records: lane (tv, tu) = (lane / 4,
// lane % 4) adds taps (tv, tu) and (tv, tu + 4) of the 7 x 7 footprint.  The
// band is held as two real planes during gridding (every atomic of a warp hits
// its own bank) and in the interleaved, padded FFT layout afterwards; the
// first FFT pass converts.
template <int LOG2G, int S, bool CAL>
__global__ void __launch_bounds__(1024)
k_grid_rows(const GridEntry* __restrict__ entries, const int* __restrict__ band_off,
            const int32_t* __restrict__ vis, long long n_bl, const Baseline* __restrict__ base,
            const ChanScale* __restrict__ cs, const float* __restrict__ tab,
            const float2* __restrict__ tw_g, int ch0, int n_img, int band_h,
            int* __restrict__ kept, void* __restrict__ h, float* __restrict__ hs, GridOpts opt) {
  constexpr int G = 1 << LOG2G;
  constexpr int LDP = band_pitch(G);
  constexpr int P = planar_pitch(G);
  static_assert(P <= LDP, "planar band fits in the FFT layout");
  extern __shared__ __align__(16) unsigned char smem[];
  float2* band = reinterpret_cast<float2*>(smem);                     // [band_h][LDP] (FFT layout)
  float* pre = reinterpret_cast<float*>(smem);                        // [band_h][P]   (gridding)
  float* pim = pre + band_h * P;
  float2* tw = band + band_h * LDP;                                   // [G]
  float4* r_hdr = reinterpret_cast<float4*>(tw + G);                  // [kRecMax] (Vr, Vi, base, kv_rel)
  float2* r_wu = reinterpret_cast<float2*>(r_hdr + kRecMax);          // [kRecMax][kWuStride]
  float* r_wv = reinterpret_cast<float*>(r_wu + kRecMax * kWuStride); // [kRecMax][kWvStride]
  __shared__ int n_home, n_rec[2];
  const int b = blockIdx.x, cb = blockIdx.y;
  const long long chan = ch0 + cb;
  for (int i = threadIdx.x; i < (2 * band_h * P) / 4; i += blockDim.x)
    reinterpret_cast<float4*>(pre)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int i = threadIdx.x; i < G; i += blockDim.x) tw[i] = tw_g[i];
  if (threadIdx.x == 0) n_home = 0;
  const ChanScale s = cs[chan];
  const int row0 = b * band_h;
  const int cmax = G / 2 - kHalfSup - 1;
  const int lim = (cmax + 1) * kQ;                     // < 2^21
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
  const int axis = threadIdx.x & 1;                  // 0: u, 1: v
  const int chunk = blockDim.x >> 1;
  const unsigned full = 0xffffffffu;
  int my_home = 0;
  const int e0 = band_off[b], e1 = band_off[b + 1];
  const int pair = threadIdx.x >> 1;
  // the fields of a candidate entry one thread of a pair needs
  struct Ent {
    int bl, cross, a, bf;
    float h, l;                                      // this thread's axis, float-float
  };
  auto load_ent = [&](int e) {
    Ent x{};
    if (e < e1) {
      const int4 hd = __ldg(reinterpret_cast<const int4*>(entries + e));
      const float2 d = __ldg(reinterpret_cast<const float2*>(&entries[e].dxh) + axis);
      x.bl = hd.x; x.cross = hd.y; x.a = hd.z; x.bf = hd.w;
      x.h = d.x; x.l = d.y;
    }
    return x;
  };
  // a chunk's keep test and the loads its records need, taken one chunk ahead
  struct Keep {
    int cu, cv, off;
    bool use;
    int2 q;                                          // XX (even thread) or YY (odd thread)
    float2 ca, cb;                                   // calibration corrections
  };
  auto keep_test = [&](const Ent& en, bool valid) {
    Keep k{};
    int cc = 0, off = 0;
    bool in = false;
    if (valid) {
      int pc;
      if (!fast_rint_prod32(en.h, en.l, s, &pc)) {
        const Baseline B = base[en.cross];           // FP64 product of the definition
        const long long pl = __double2ll_rn(__dmul_rn(axis ? B.dy : B.dx, s.s));
        pc = static_cast<int>(pl > lim ? lim : (pl < -lim ? -lim : pl));
      }
      if (pc > -lim && pc < lim) {
        centre_cell32(pc, cc, off);
        in = cc <= cmax && cc >= -cmax;
      }
      // baselines straddling an edge of the uv range: decide in FP64, L * (nu / c)
      if (CAL && axis == 0 && (en.bf & kCheckUv)) {
        const double lam = __dmul_rn(opt.blen[en.cross], s.nu_c);
        in = in && lam >= opt.uv_min && lam < opt.uv_max;
      }
    }
    const int cc_o = __shfl_xor_sync(full, cc, 1);
    const int in_o = __shfl_xor_sync(full, in ? 1 : 0, 1);   // every lane takes part
    const bool kp = in && in_o;
    k.cu = axis ? cc_o : cc;
    k.cv = axis ? cc : cc_o;
    k.off = off;
    const int kv_home = G / 2 + k.cv;
    const int kv_rel = kv_home - kHalfSup - row0;
    if (kp && axis && kv_home >= row0 && kv_home < row0 + band_h) ++my_home;
    k.use = kp && kv_rel + kSupport > 0 && kv_rel < band_h;
    if (k.use) {
      k.q = __ldg(reinterpret_cast<const int2*>(vis) + (chan * n_bl + en.bl) * 4 + axis * 3);
      if (CAL && opt.gains != nullptr) {
        const float2* gc = opt.gains + chan * opt.n_input;
        k.ca = __ldg(gc + 2 * en.a + axis);
        k.cb = __ldg(gc + 2 * (en.bf & 0xffff) + axis);
      }
    }
    return k;
  };
  if (threadIdx.x == 0) n_rec[0] = 0;
  Keep kn = keep_test(load_ent(e0 + pair), e0 + pair < e1);
  Ent en = load_ent(e0 + chunk + pair);
  __syncthreads();
  int it = 0;
  for (int c0 = e0; c0 < e1; c0 += chunk, ++it) {
    // ---- records of this chunk: one visibility per thread pair
    // Stokes I = (XX + YY) / 2: XX on the even thread, YY on the odd one;
    // exact integer sums, or with the calibration corrections c_a conj(c_b)
    // applied per polarisation in FP32
    const Keep k = kn;
    float fr, fi;
    if (!CAL || opt.gains == nullptr) {
      const int sr = k.q.x + __shfl_xor_sync(full, k.q.x, 1);
      const int si = k.q.y + __shfl_xor_sync(full, k.q.y, 1);
      fr = static_cast<float>(sr);
      fi = static_cast<float>(si);
    } else {
      float pr = 0.f, pi = 0.f;
      if (k.use) {
        const float vr = static_cast<float>(k.q.x), vi = static_cast<float>(k.q.y);
        const float gr = k.ca.x * k.cb.x + k.ca.y * k.cb.y, gi = k.ca.y * k.cb.x - k.ca.x * k.cb.y;
        pr = gr * vr - gi * vi;
        pi = gr * vi + gi * vr;
      }
      fr = pr + __shfl_xor_sync(full, pr, 1);
      fi = pi + __shfl_xor_sync(full, pi, 1);
    }
    const unsigned m = __ballot_sync(full, k.use) & 0x55555555u;
    int base_slot = 0;
    if (lane == 0 && m) base_slot = atomicAdd(&n_rec[it & 1], __popc(m));
    base_slot = __shfl_sync(full, base_slot, 0);
    if (k.use) {
      const int slot = base_slot + __popc(m & ((1u << (lane & ~1)) - 1u));
      const int kv_rel = G / 2 + k.cv - kHalfSup - row0;
      const int ku0 = G / 2 + k.cu - kHalfSup;
      float w[8];
#pragma unroll
      for (int t = 0; t < kSupport; ++t) w[t] = __ldg(tab + kHalfTab + (t - kHalfSup) * kQ - k.off);
      w[7] = 0.0f;
      if (axis == 0) {
        // (-1)^ku centring sign; conj of Stokes I: the exp(+) transform is a
        // forward FFT of conj(G)
#pragma unroll
        for (int t = 0; t < kSupport; ++t)
          if ((ku0 + t) & 1) w[t] = -w[t];
        r_hdr[slot] = make_float4(0.5f * fr, -0.5f * fi, __int_as_float(kv_rel * P + ku0), __int_as_float(kv_rel));
#pragma unroll
        for (int t = 0; t < 4; ++t) r_wu[slot * kWuStride + t] = make_float2(w[t], w[t + 4]);
      } else {
        const int kv0 = row0 + kv_rel;               // (-1)^kv centring sign
#pragma unroll
        for (int t = 0; t < kSupport; ++t)
          if ((kv0 + t) & 1) w[t] = -w[t];
#pragma unroll
        for (int t = 0; t < 8; ++t) r_wv[slot * kWvStride + t] = w[t];
      }
    }
    __syncthreads();
    const int nr = n_rec[it & 1];
    if (threadIdx.x == 0) n_rec[(it + 1) & 1] = 0;   // last read before the previous barrier
    // ---- the next chunk's keep test, visibility loads and the entries after
    // it, in flight while this chunk is swept
    kn = keep_test(en, c0 + chunk + pair < e1);
    en = load_ent(c0 + 2 * chunk + pair);
    // ---- sweep: one record per warp, 49 taps in four atomic instructions
    const int tv = lane >> 2, tu = lane & 3;
    for (int rec = warp; rec < nr; rec += n_warps) {
      const float4 hd = r_hdr[rec];
      const float2 wp = r_wu[rec * kWuStride + tu];
      const float wv = r_wv[rec * kWvStride + tv];
      const int row = __float_as_int(hd.w) + tv;
      if (tv < kSupport && static_cast<unsigned>(row) < static_cast<unsigned>(band_h)) {
        const int a = __float_as_int(hd.z) + tv * P + tu;
        const float w0 = wv * wp.x;
        atomicAdd(pre + a, w0 * hd.x);
        atomicAdd(pim + a, w0 * hd.y);
        if (tu < kSupport - 4) {
          const float w1 = wv * wp.y;
          atomicAdd(pre + a + 4, w1 * hd.x);
          atomicAdd(pim + a + 4, w1 * hd.y);
        }
      }
    }
    __syncthreads();
  }
  if (my_home) atomicAdd(&n_home, my_home);
  __syncthreads();
  if (threadIdx.x == 0 && n_home) atomicAdd(kept + chan, n_home);
  fft_rows_inplace<LOG2G>(band, LDP, tw, pre, pim, P);
  // central N columns of each transformed row, in the storage format
  const int offc = G / 2 - n_img / 2;
  const long long hrow0 = static_cast<long long>(cb) * G + row0;
  if constexpr (S == kStoreF32) {
    float2* hb = static_cast<float2*>(h) + hrow0 * n_img;
    for (int i = threadIdx.x; i < band_h * n_img; i += blockDim.x) {
      const int r = i / n_img, c = i - r * n_img;
      hb[static_cast<long long>(r) * n_img + c] = band[r * LDP + pad16(offc + c)];
    }
  } else if constexpr (S == kStoreBF16) {
    __nv_bfloat162* hb = static_cast<__nv_bfloat162*>(h) + hrow0 * n_img;
    for (int i = threadIdx.x; i < band_h * n_img; i += blockDim.x) {
      const int r = i / n_img, c = i - r * n_img;
      hb[static_cast<long long>(r) * n_img + c] = __float22bfloat162_rn(band[r * LDP + pad16(offc + c)]);
    }
  } else {
    // FP16 with a power-of-two scale per row: the row's largest component
    // lands in [2^13, 2^14), far from FP16 overflow; scaling is exact
    __half2* hb = static_cast<__half2*>(h) + hrow0 * n_img;
    const int lane = threadIdx.x & 31, n_w = blockDim.x >> 5;
    for (int r = threadIdx.x >> 5; r < band_h; r += n_w) {
      float m = 0.f;
      for (int c = lane; c < n_img; c += 32) {
        const float2 v = band[r * LDP + pad16(offc + c)];
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      int e = 0;
      if (m > 0.f) frexpf(m, &e);
      const float sc = m > 0.f ? ldexpf(1.0f, 14 - e) : 1.0f;
      if (lane == 0) hs[hrow0 + r] = m > 0.f ? ldexpf(1.0f, e - 14) : 0.0f;
      for (int c = lane; c < n_img; c += 32) {
        const float2 v = band[r * LDP + pad16(offc + c)];
        hb[static_cast<long long>(r) * n_img + c] = __float22half2_rn(make_float2(v.x * sc, v.y * sc));
      }
    }
  }
}

// Two adjacent values (idx even) of the half-transformed grid in FP32.
template <int S>
__device__ __forceinline__ void load_h2(const void* h, const float* hs, long long row, long long idx, float2& v0,
                                        float2& v1) {
  if constexpr (S == kStoreF32) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(static_cast<const float2*>(h) + idx));
    v0 = make_float2(q.x, q.y);
    v1 = make_float2(q.z, q.w);
  } else {
    const uint2 raw = __ldg(reinterpret_cast<const uint2*>(static_cast<const unsigned*>(h) + idx));
    if constexpr (S == kStoreBF16) {
      __nv_bfloat162 b0, b1;
      memcpy(&b0, &raw.x, sizeof(b0));
      memcpy(&b1, &raw.y, sizeof(b1));
      v0 = __bfloat1622float2(b0);
      v1 = __bfloat1622float2(b1);
    } else {
      __half2 b0, b1;
      memcpy(&b0, &raw.x, sizeof(b0));
      memcpy(&b1, &raw.y, sizeof(b1));
      const float sc = __ldg(hs + row);
      v0 = __half22float2(b0);
      v1 = __half22float2(b1);
      v0 = make_float2(v0.x * sc, v0.y * sc);
      v1 = make_float2(v1.x * sc, v1.y * sc);
    }
  }
}

// Column transforms of the N central columns and the image itself.
//
// The image is the real part of the transform.  The real part of the DFT of a
// column c is the DFT of its Hermitian part (c(k) + conj c(-k)) / 2 (indices
// mod G), whose DFT is real; so two columns c1, c2 share one complex FFT of
// d = h1 + i h2, with DFT Re DFT(c1) + i Re DFT(c2).  d is formed, doubled,
// while the column pair is read (rows k and G - k together), and the output
// scale takes the factor 1/2 back.  C columns per CTA, C / 2 transforms.
template <int LOG2G, int S>
__global__ void __launch_bounds__(512, 2)
k_fft_cols(const void* __restrict__ h, const float* __restrict__ hs, int n_img, int cols_per_cta, int ch0,
           const float2* __restrict__ tw_g, const float* __restrict__ inv_corr,
           const uint8_t* __restrict__ mask, const int* __restrict__ kept, float* __restrict__ img) {
  constexpr int G = 1 << LOG2G;
  constexpr int LDP = band_pitch(G);
  extern __shared__ __align__(16) unsigned char smem[];
  const int C = cols_per_cta, CP = C / 2;
  float2* A = reinterpret_cast<float2*>(smem);        // [C / 2][LDP]: packed column pairs
  float2* tw = A + CP * LDP;
  const int cb = blockIdx.y;
  const int c0 = blockIdx.x * C;
  const long long hrow0 = static_cast<long long>(cb) * G;
  for (int i = threadIdx.x; i < G; i += blockDim.x) tw[i] = tw_g[i];
  // U items per thread in flight: the reads come from L2 and would otherwise
  // wait one round trip each
  constexpr int U = 4;
  const int n_items = (G / 2 + 1) * CP;
  for (int i0 = threadIdx.x; i0 < n_items; i0 += U * blockDim.x) {
    float2 a[U], e[U], b[U], f[U];                    // c1(k), c2(k), c1(-k), c2(-k)
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < n_items) {
        const int k = i / CP, p = i - k * CP;
        const int km = (G - k) & (G - 1);
        load_h2<S>(h, hs, hrow0 + k, (hrow0 + k) * n_img + c0 + 2 * p, a[u], e[u]);
        load_h2<S>(h, hs, hrow0 + km, (hrow0 + km) * n_img + c0 + 2 * p, b[u], f[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < n_items) {
        const int k = i / CP, p = i - k * CP;
        const int km = (G - k) & (G - 1);
        A[p * LDP + pad16(k)] =
            make_float2((a[u].x + b[u].x) - (e[u].y - f[u].y), (a[u].y - b[u].y) + (e[u].x + f[u].x));
        if (km != k)
          A[p * LDP + pad16(km)] =
              make_float2((b[u].x + a[u].x) - (f[u].y - e[u].y), (b[u].y - a[u].y) + (f[u].x + e[u].x));
      }
    }
  }
  __syncthreads();
  fft_rows_inplace<LOG2G>(A, LDP, tw);
  const long long chan = ch0 + cb;
  const int k = kept[chan];
  const float norm = k > 0 ? 0.5f / static_cast<float>(k) : 0.0f;
  const int off = G / 2 - n_img / 2;
  float* out = img + chan * n_img * n_img;
#pragma unroll 4
  for (int i = threadIdx.x; i < n_img * C; i += blockDim.x) {
    const int r = i / C, c = i - r * C;
    const int col = c0 + c;
    float v = 0.0f;
    if (mask[r * n_img + col]) {
      const float2 z = A[(c >> 1) * LDP + pad16(off + r)];
      v = (c & 1 ? z.y : z.x) * norm * inv_corr[r] * inv_corr[col];
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
  int n, g, log2g, band_h, n_bands, batch, cols_per_cta, storage;
  long long n_cross;
};

ImgPlan make_plan(int n_ant, int n_chan, int n, int storage) {
  ImgPlan p;
  p.n = n;
  p.storage = storage;
  p.g = kPad * n;
  p.log2g = ilog2(p.g);
  // 16384 complex values per band: one CTA of 1024 threads per SM, and each
  // 7-row footprint spills into a second band only (7 - 1) / band_h of the time
  p.band_h = 16384 / p.g < p.g ? 16384 / p.g : p.g;
  p.n_bands = p.g / p.band_h;
  p.n_cross = static_cast<long long>(n_ant) * (n_ant - 1) / 2;
  const long long h_bytes = 8LL * p.g * n;           // half-transformed grid of one channel
  long long b = (64LL << 20) / h_bytes;
  if (b < 1) b = 1;
  if (b > 64) b = 64;
  if (b > n_chan) b = n_chan;
  p.batch = static_cast<int>(b);
  // an even number of columns per CTA (the column pass pairs them)
  int c = 8192 / p.g;
  // 16-bit storage: at least 8 columns per CTA, so each row segment the
  // column pass reads is a whole 32-byte sector
  if (storage != kStoreF32 && c < 8 && 8 * p.g / 32 <= 512) c = 8;
  if (c > n) c = n;
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
  int* band_off;
  GridEntry* entries;
  double* blen;      // [n_cross] baseline lengths (metres)
  void* h;           // [batch][G][N] complex in the storage format
  float* hs;         // [batch][G] row scales (FP16 storage)
};

// Candidate entries: each cross baseline once per band it can touch (at most
// 2 for 7-row footprints in >= 4-row bands... bounded by n_bands in general).
long long entry_capacity(const ImgPlan& p) {
  const long long per = std::min<long long>(p.n_bands, kSupport + 2);
  return std::max<long long>(1, p.n_cross * per);
}

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
  w.band_off = c.take<int>(p.n_bands + 1);
  w.entries = c.take<GridEntry>(entry_capacity(p));
  w.blen = c.take<double>(p.n_cross > 0 ? p.n_cross : 1);
  w.h = c.take<float2>(static_cast<size_t>(p.batch) * p.g * p.n);
  w.hs = c.take<float>(static_cast<size_t>(p.batch) * p.g);
  *need = c.used;
  return w;
}

// Host: which baselines can touch which band of grid rows for any channel of
// the call (u, v scale linearly with frequency; one cell of margin).
// Baseline length in metres, sqrt(dx^2 + dy^2) in FP64 (host code is built
// without FMA contraction, so this rounds like the definition).
double baseline_length(const double* ant, int a, int b) {
  const double dx = ant[3 * a] - ant[3 * b], dy = ant[3 * a + 1] - ant[3 * b + 1];
  const double x2 = dx * dx, y2 = dy * dy;
  return std::sqrt(x2 + y2);
}

void build_entries(const ImgPlan& p, int n_ant, const double* ant, const double* freq, int n_chan,
                   double cell, double uv_min, double uv_max, std::vector<GridEntry>& out, std::vector<int>& off) {
  const double du = 1.0 / (static_cast<double>(p.g) * cell);
  double fmin = freq[0], fmax = freq[0];
  for (int f = 1; f < n_chan; ++f) {
    fmin = std::min(fmin, freq[f]);
    fmax = std::max(fmax, freq[f]);
  }
  const double s_lo = fmin / (kCLight * du), s_hi = fmax / (kCLight * du);   // cells per metre
  const bool uv_cut = uv_min > 0.0 || std::isfinite(uv_max);
  const double w_lo = fmin / kCLight, w_hi = fmax / kCLight;                  // wavelengths per metre
  const int cmax = p.g / 2 - kHalfSup - 1;
  std::vector<std::vector<GridEntry>> bands(p.n_bands);
  long long cross = 0;
  for (int a = 0; a < n_ant; ++a)
    for (int b = a + 1; b < n_ant; ++b, ++cross) {
      const double dx = ant[3 * a] - ant[3 * b], dy = ant[3 * a + 1] - ant[3 * b + 1];
      const double u0 = std::min(dx * s_lo, dx * s_hi), u1 = std::max(dx * s_lo, dx * s_hi);
      const double v0 = std::min(dy * s_lo, dy * s_hi), v1 = std::max(dy * s_lo, dy * s_hi);
      // can the centre cell ever satisfy |c0| <= cmax?
      if (u0 > cmax + 1.5 || u1 < -cmax - 1.5 || v0 > cmax + 1.5 || v1 < -cmax - 1.5) continue;
      // uv range: decided here when every channel of the call agrees (with a
      // relative margin), per channel on the device otherwise
      bool check = false;
      if (uv_cut) {
        const double L = baseline_length(ant, a, b);
        const double l0 = L * w_lo, l1 = L * w_hi, eps = 1e-9;
        if (l1 < uv_min * (1.0 - eps) || l0 >= uv_max * (1.0 + eps)) continue;      // always outside
        check = !(l0 >= uv_min * (1.0 + eps) && l1 < uv_max * (1.0 - eps));       // not always inside
      }
      int r_lo = p.g / 2 + static_cast<int>(std::floor(v0)) - 1 - kHalfSup;
      int r_hi = p.g / 2 + static_cast<int>(std::ceil(v1)) + 1 + kHalfSup;
      r_lo = std::max(r_lo, 0);
      r_hi = std::min(r_hi, p.g - 1);
      GridEntry e;
      e.bl = static_cast<int>(a * static_cast<long long>(n_ant) - static_cast<long long>(a) * (a - 1) / 2 + (b - a));
      e.cross = static_cast<int>(cross);
      e.a = a;
      e.bf = b | (check ? kCheckUv : 0);
      e.dxh = static_cast<float>(dx);
      e.dxl = static_cast<float>(dx - static_cast<double>(e.dxh));
      e.dyh = static_cast<float>(dy);
      e.dyl = static_cast<float>(dy - static_cast<double>(e.dyh));
      for (int bd = r_lo / p.band_h; bd <= r_hi / p.band_h; ++bd) bands[bd].push_back(e);
    }
  out.clear();
  off.assign(p.n_bands + 1, 0);
  for (int bd = 0; bd < p.n_bands; ++bd) {
    off[bd] = static_cast<int>(out.size());
    out.insert(out.end(), bands[bd].begin(), bands[bd].end());
  }
  off[p.n_bands] = static_cast<int>(out.size());
}

template <int L, int S>
int launch_bands(const ImgPlan& p, const ImgWs& w, const GridOpts& o, const int32_t* vis, long long n_bl, int ch0,
                 int nb, float* img, cudaStream_t st) {
  constexpr int G = 1 << L;
  constexpr int LDP = band_pitch(G);
  {
    const size_t sm = static_cast<size_t>(p.band_h) * LDP * sizeof(float2) + G * sizeof(float2) +
                      kRecMax * (sizeof(float4) + kWuStride * sizeof(float2) + kWvStride * sizeof(float));
    // calibration corrections or a uv range select the variant that applies them
    const bool cal = o.gains != nullptr || o.uv_min > 0.0 || std::isfinite(o.uv_max);
    auto kern = cal ? k_grid_rows<L, S, true> : k_grid_rows<L, S, false>;
    OVRO_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm)));
    const int threads = p.band_h * G / 16;
    dim3 grid(p.n_bands, nb);
    OVRO_PROF("k_grid_rows", st);
    kern<<<grid, threads, sm, st>>>(w.entries, w.band_off, vis, n_bl, w.base, w.cs, w.tab, w.tw, ch0, p.n, p.band_h,
                                    w.kept, w.h, w.hs, o);
    OVRO_LAUNCH_CHECK();
  }
  {
    const size_t sm = static_cast<size_t>(p.cols_per_cta / 2) * LDP * sizeof(float2) + G * sizeof(float2);
    OVRO_CUDA_TRY(cudaFuncSetAttribute(k_fft_cols<L, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sm)));
    const int threads = p.cols_per_cta * G / 32;
    dim3 grid(p.n / p.cols_per_cta, nb);
    OVRO_PROF("k_fft_cols", st);
    k_fft_cols<L, S><<<grid, threads, sm, st>>>(w.h, w.hs, p.n, p.cols_per_cta, ch0, w.tw, w.inv_corr, w.mask,
                                                w.kept, img);
    OVRO_LAUNCH_CHECK();
  }
  return OVRO_OK;
}

template <int L>
int launch_storage(const ImgPlan& p, const ImgWs& w, const GridOpts& o, const int32_t* vis, long long n_bl, int ch0,
                   int nb, float* img, cudaStream_t st) {
  switch (p.storage) {
    case kStoreF32: return launch_bands<L, kStoreF32>(p, w, o, vis, n_bl, ch0, nb, img, st);
    case kStoreBF16: return launch_bands<L, kStoreBF16>(p, w, o, vis, n_bl, ch0, nb, img, st);
    case kStoreF16: return launch_bands<L, kStoreF16>(p, w, o, vis, n_bl, ch0, nb, img, st);
    default: return OVRO_ERR_INVALID_ARG;
  }
}

int run_bands(const ImgPlan& p, const ImgWs& w, const GridOpts& o, const int32_t* vis, long long n_bl, int ch0,
              int nb, float* img, cudaStream_t st) {
  switch (p.log2g) {
    case 5: return launch_storage<5>(p, w, o, vis, n_bl, ch0, nb, img, st);
    case 6: return launch_storage<6>(p, w, o, vis, n_bl, ch0, nb, img, st);
    case 7: return launch_storage<7>(p, w, o, vis, n_bl, ch0, nb, img, st);
    case 8: return launch_storage<8>(p, w, o, vis, n_bl, ch0, nb, img, st);
    case 9: return launch_storage<9>(p, w, o, vis, n_bl, ch0, nb, img, st);
    case 10: return launch_storage<10>(p, w, o, vis, n_bl, ch0, nb, img, st);
    case 11: return launch_storage<11>(p, w, o, vis, n_bl, ch0, nb, img, st);
    default: return OVRO_ERR_UNSUPPORTED;
  }
}

int upload_common(const ImgPlan& p, const ImgWs& w, int n_ant, const double* h_ant,
                  const double* h_freq, int n_chan, double cell, cudaStream_t st,
                  double uv_min = 0.0, double uv_max = HUGE_VAL) {
  const KernelTables& kt = kernel_tables();
  std::vector<double> corr;
  grid_correction(p.n, p.g, corr);
  std::vector<float> inv(p.n);
  for (int i = 0; i < p.n; ++i) inv[i] = static_cast<float>(1.0 / corr[i]);
  std::vector<GridEntry> entries;
  std::vector<int> off;
  build_entries(p, n_ant, h_ant, h_freq, n_chan, cell, uv_min, uv_max, entries, off);
  if (static_cast<long long>(entries.size()) > entry_capacity(p)) return OVRO_ERR_CAPACITY;
  std::vector<double> blen(p.n_cross > 0 ? p.n_cross : 1, 0.0);
  {
    long long x = 0;
    for (int a = 0; a < n_ant; ++a)
      for (int b = a + 1; b < n_ant; ++b) blen[x++] = baseline_length(h_ant, a, b);
  }
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.blen, blen.data(), blen.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.tab, kt.table32.data(), kTabLen * sizeof(float),
                                cudaMemcpyHostToDevice, st));
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.inv_corr, inv.data(), p.n * sizeof(float), cudaMemcpyHostToDevice, st));
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.ant, h_ant, static_cast<size_t>(n_ant) * 3 * sizeof(double),
                                cudaMemcpyHostToDevice, st));
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.freq, h_freq, static_cast<size_t>(n_chan) * sizeof(double),
                                cudaMemcpyHostToDevice, st));
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.band_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  if (!entries.empty())
    OVRO_CUDA_TRY(cudaMemcpyAsync(w.entries, entries.data(), entries.size() * sizeof(GridEntry),
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

struct GridCtx {
  ImgPlan p;
  ImgWs w;
  int n_ant = 0, n_chan = 0;
  double cell = 0.0;
  const float2* gains = nullptr;      // calibration corrections [n_chan][2 n_ant]
  double uv_min = 0.0, uv_max = HUGE_VAL;
};

size_t grid_ctx_workspace(int n_ant, int n_chan, int image_size, int storage) {
  if (n_ant <= 0 || n_chan <= 0 || !is_pow2(image_size) || image_size < 16 || image_size > 1024) return 0;
  if (storage != OVRO_STORE_FP32 && storage != OVRO_STORE_BF16 && storage != OVRO_STORE_FP16) return 0;
  const ImgPlan p = make_plan(n_ant, n_chan, image_size, storage);
  size_t need = 0;
  carve_img(nullptr, 0, p, n_ant, n_chan, &need);
  return need;
}

int grid_ctx_init(GridCtx** out, int n_ant, int n_chan, int image_size, double cell, int storage, void* d_ws,
                  size_t ws_bytes, const void* d_gains, double uv_min, double uv_max) {
  if (!out) return OVRO_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_ant <= 0 || n_chan <= 0 || !(cell > 0.0)) return OVRO_ERR_INVALID_ARG;
  if (storage != OVRO_STORE_FP32 && storage != OVRO_STORE_BF16 && storage != OVRO_STORE_FP16)
    return OVRO_ERR_INVALID_ARG;
  if (!is_pow2(image_size) || image_size < 16 || image_size > 1024 || n_ant > 4096) return OVRO_ERR_UNSUPPORTED;
  GridCtx* g = new GridCtx;
  g->p = make_plan(n_ant, n_chan, image_size, storage);
  size_t need = 0;
  g->w = carve_img(d_ws, ws_bytes, g->p, n_ant, n_chan, &need);
  if (int e = check_workspace(d_ws, ws_bytes, need)) {
    delete g;
    return e;
  }
  g->n_ant = n_ant;
  g->n_chan = n_chan;
  g->cell = cell;
  g->gains = static_cast<const float2*>(d_gains);
  g->uv_min = uv_min;
  g->uv_max = uv_max;
  *out = g;
  return OVRO_OK;
}

int grid_ctx_upload(GridCtx* g, const double* h_ant_enu_m, const double* h_chan_freq_hz, cudaStream_t st) {
  if (!g) return OVRO_ERR_INVALID_ARG;
  if (int e = validate(g->n_ant, h_ant_enu_m, h_chan_freq_hz, g->n_chan, g->p.n, g->cell)) return e;
  return upload_common(g->p, g->w, g->n_ant, h_ant_enu_m, h_chan_freq_hz, g->n_chan, g->cell, st, g->uv_min,
                       g->uv_max);
}

int grid_ctx_enqueue(GridCtx* g, const int32_t* d_vis, float* d_img, int32_t* d_counts_or_null, cudaStream_t st) {
  if (!g || !d_vis || !d_img) return OVRO_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_vis) % 16 != 0) return OVRO_ERR_INVALID_ARG;
  const ImgPlan& p = g->p;
  const long long n_bl = static_cast<long long>(g->n_ant) * (g->n_ant + 1) / 2;
  GridOpts o;
  o.gains = g->gains;
  o.n_input = 2 * g->n_ant;
  o.blen = g->w.blen;
  o.uv_min = g->uv_min;
  o.uv_max = g->uv_max;
  // channels per launch pair (at most the workspace's batch): every choice
  // gives the same images and counts
  auto all = [&](int batch) -> int {
    OVRO_CUDA_TRY(cudaMemsetAsync(g->w.kept, 0, g->n_chan * sizeof(int), st));
    for (int ch0 = 0; ch0 < g->n_chan; ch0 += batch) {
      const int nb = g->n_chan - ch0 < batch ? g->n_chan - ch0 : batch;
      if (int e = run_bands(p, g->w, o, d_vis, n_bl, ch0, nb, d_img, st)) return e;
    }
    return OVRO_OK;
  };
  const std::string key = tune_key("grid_batch", {g->n_ant, g->n_chan, p.n, p.storage});
  int batch = std::min(p.batch, std::max(1, tuned(key, p.batch)));
  if (tuning(st)) {
    std::vector<int> cands;
    for (int b = p.batch; b >= 1 && cands.size() < 4; b /= 2) cands.push_back(b);
    if (int e = tune_pick(key, cands, all, st, &batch)) return e;
  }
  if (int e = all(batch)) return e;
  if (d_counts_or_null) {
    k_counts_out<<<(g->n_chan + 255) / 256, 256, 0, st>>>(g->w.kept, g->n_chan, d_counts_or_null);
    OVRO_LAUNCH_CHECK();
  }
  return OVRO_OK;
}

int grid_ctx_gridded(GridCtx* g, long long* total, cudaStream_t st) {
  if (!g || !total) return OVRO_ERR_INVALID_ARG;
  std::vector<int> k(g->n_chan);
  OVRO_CUDA_TRY(cudaMemcpyAsync(k.data(), g->w.kept, g->n_chan * sizeof(int), cudaMemcpyDeviceToHost, st));
  OVRO_CUDA_TRY(cudaStreamSynchronize(st));
  long long s = 0;
  for (int v : k) s += v;
  *total = s;
  return OVRO_OK;
}

void grid_ctx_free(GridCtx* g) { delete g; }

}  // namespace ovro

extern "C" {

size_t ovro_grid_image_workspace_size(int n_ant, int n_chan, int image_size, int storage) {
  return ovro::grid_ctx_workspace(n_ant, n_chan, image_size, storage);
}

int ovro_grid_image(const int32_t* d_vis, int n_ant, const double* h_ant_enu_m,
                    const double* h_chan_freq_hz, int n_chan, int image_size, double cell_dircos,
                    int storage, float* d_img, int32_t* d_n_gridded_or_null, void* d_ws,
                    size_t ws_bytes, void* stream) {
  ovro_grid_options o;
  o.storage = storage;
  o.d_gains_or_null = nullptr;
  o.uv_min_lambda = 0.0;
  o.uv_max_lambda = 0.0;
  return ovro_grid_image_ex(d_vis, n_ant, h_ant_enu_m, h_chan_freq_hz, n_chan, image_size, cell_dircos, &o, d_img,
                            d_n_gridded_or_null, d_ws, ws_bytes, stream);
}

int ovro_grid_image_ex(const int32_t* d_vis, int n_ant, const double* h_ant_enu_m, const double* h_chan_freq_hz,
                       int n_chan, int image_size, double cell_dircos, const ovro_grid_options* opt, float* d_img,
                       int32_t* d_n_gridded_or_null, void* d_ws, size_t ws_bytes, void* stream) {
  using namespace ovro;
  if (!d_vis || !d_img || !opt) return OVRO_ERR_INVALID_ARG;
  if (int e = validate(n_ant, h_ant_enu_m, h_chan_freq_hz, n_chan, image_size, cell_dircos)) return e;
  const int storage = opt->storage;
  if (storage != OVRO_STORE_FP32 && storage != OVRO_STORE_BF16 && storage != OVRO_STORE_FP16)
    return OVRO_ERR_INVALID_ARG;
  if (!(opt->uv_min_lambda >= 0.0) || std::isnan(opt->uv_max_lambda)) return OVRO_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_vis) % 16 != 0) return OVRO_ERR_INVALID_ARG;
  if (opt->d_gains_or_null && reinterpret_cast<uintptr_t>(opt->d_gains_or_null) % 8 != 0) return OVRO_ERR_INVALID_ARG;
  const double uv_max = opt->uv_max_lambda > 0.0 ? opt->uv_max_lambda : HUGE_VAL;
  GridCtx* g = nullptr;
  if (int e = grid_ctx_init(&g, n_ant, n_chan, image_size, cell_dircos, storage, d_ws, ws_bytes,
                            opt->d_gains_or_null, opt->uv_min_lambda, uv_max))
    return e;
  cudaStream_t st = as_stream(stream);
  int e = grid_ctx_upload(g, h_ant_enu_m, h_chan_freq_hz, st);
  if (!e) e = grid_ctx_enqueue(g, d_vis, d_img, d_n_gridded_or_null, st);
  grid_ctx_free(g);
  return e;
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
  const ImgPlan p = make_plan(n_ant, n_chan, image_size, OVRO_STORE_FP32);
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
