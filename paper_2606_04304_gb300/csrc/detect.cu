// a8-a12: Stage I candidate search over the image cube (Section 2.4).
//
//  a8  k_stats       per channel image: exact median and MAD of the in-horizon
//                    pixels (radix selection on order-preserving keys; the
//                    MAD's |x - med| ordering is decided on FP32 keys and the
//                    few elements inside the FP32 error window are resolved in
//                    FP64), giving FP64 statistics.
//      k_ztrans      standardises (z = (x - med) / (1.4826 MAD)) and turns the
//                    cube into per-pixel spectra [coarse][pixel][channel].
//  a9  k_rank        per pixel spectrum: stable LSD radix sort (4 x 8-bit
//                    digits, ballot multisplit for in-warp ranks) -> sorted values and
//                    the rank of every channel.
//      k_walk        one thread per pixel walks the channels keeping the
//                    window's ranks in a bitset (shared memory, interleaved per
//                    thread) and a cursor on the lower median, so every step of
//                    the exact running median costs O(1) amortised.
//  a10 k_mf          per 8 consecutive channels a thread holds the 107-value
//                    neighbourhood as register prefix sums and evaluates all 29
//                    boxcars as prefix differences; keeps max SNR and width and
//                    histograms the SNRs above the p = alpha floor.
//  a11 host + k_gather_bins  Benjamini-Hochberg: counts above every
//                    histogram bin edge are exact, so the step-up rule is
//                    decided bin by bin in FP64; only the bins whose outcome
//                    the edges leave open are gathered (one pass) and ranked
//                    value by value.
//  a12 k_nms_warp    greedy 1D non-maximum suppression per (pixel, coarse
//      k_nms_big     channel) on the device, one warp per pair (one CTA with a
//                    bitonic sort for pairs with many detections) in one
//                    pass over the SNR cube, each pair's detections written to
//                    a range reserved by an atomic; the host orders the pairs
//                    (counting sort) into (pixel, coarse, channel) order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "common.cuh"
#include "stages.h"
#include "tune.h"

namespace ovro {
namespace {

constexpr double kMadToSigma = 1.482602218505602;
constexpr int kNW = 29;
// default boxcar widths: 1..10, 13..49 step 3, 50..100 step 10 (29 widths)
__host__ __device__ constexpr int width_of(int i) {
  return i < 10 ? i + 1 : (i < 23 ? 13 + 3 * (i - 10) : 50 + 10 * (i - 23));
}
// 1 / sqrt(w) for the default widths, correctly rounded from FP64
__host__ __device__ constexpr float rsqrt_width(int i) {
  return i == 0 ? 1.f : i == 1 ? 0.70710678118654746f : i == 2 ? 0.57735026918962584f
       : i == 3 ? 0.5f : i == 4 ? 0.44721359549995793f : i == 5 ? 0.40824829046386307f
       : i == 6 ? 0.3779644730092272f : i == 7 ? 0.35355339059327373f
       : i == 8 ? 0.33333333333333331f : i == 9 ? 0.31622776601683794f
       : i == 10 ? 0.27735009811261457f : i == 11 ? 0.25f : i == 12 ? 0.22941573387056174f
       : i == 13 ? 0.21320071635561041f : i == 14 ? 0.20000000000000001f
       : i == 15 ? 0.1889822365046136f : i == 16 ? 0.17960530202677491f
       : i == 17 ? 0.17149858514250882f : i == 18 ? 0.16439898730535729f
       : i == 19 ? 0.15811388300841897f : i == 20 ? 0.15249857033260467f
       : i == 21 ? 0.14744195615489714f : i == 22 ? 0.14285714285714285f
       : i == 23 ? 0.1414213562373095f : i == 24 ? 0.12909944487358055f
       : i == 25 ? 0.11952286093343936f : i == 26 ? 0.11180339887498948f
       : i == 27 ? 0.10540925533894598f : 0.10000000000000001f;
}
constexpr int kMaxLo = 49, kMaxHi = 50;
constexpr int kVox = 8;                                  // voxels per thread in k_mf
constexpr int kWin = kVox + kMaxLo + kMaxHi;             // 107

// histogram of SNRs: bins of 2^-7 relative width from the floor up to 64, then overflow
constexpr int kHistShift = 16;

__device__ int g_detect_status;

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ float ulpf(float x) {
  x = fabsf(x);
  if (x == 0.f) return 1.4e-45f;
  const int e = (__float_as_int(x) >> 23) & 0xff;
  return e > 23 ? __int_as_float((e - 23) << 23) : 1.4e-45f;
}

// block-wide exclusive scan of `n` uint32 counters in shared memory (any blockDim multiple of 32)
__device__ void block_exclusive_scan(uint32_t* a, int n, uint32_t* warp_tot) {
  const int T = blockDim.x, tid = threadIdx.x;
  const int per = (n + T - 1) / T;
  const int lo = tid * per, hi = min(n, lo + per);
  uint32_t s = 0;
  for (int i = lo; i < hi; ++i) s += a[i];
  // inclusive warp scan of s
  const int lane = tid & 31, warp = tid >> 5;
  uint32_t v = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) warp_tot[warp] = v;
  __syncthreads();
  if (warp == 0) {
    const int nw = T >> 5;
    uint32_t w = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < nw) warp_tot[lane] = w;
  }
  __syncthreads();
  uint32_t run = v - s + (warp > 0 ? warp_tot[warp - 1] : 0);
  for (int i = lo; i < hi; ++i) {
    const uint32_t c = a[i];
    a[i] = run;
    run += c;
  }
  __syncthreads();
}

// ------------------------------------------------------------------ a8 stats
struct SelectState {
  uint32_t prefix;
  int k;
};

// k-th smallest (0-based) of the keys produced by key_of(i), i < n.
// hist: 2048 uint32 in shared memory; tot: 64 uint32 scratch; result broadcast.
template <class KeyOf>
__device__ uint32_t block_select(int n, int k, const KeyOf& key_of, uint32_t* hist, uint32_t* tot,
                                 int* sel) {
  const int tid = threadIdx.x, T = blockDim.x;
  uint32_t prefix = 0;
  int kk = k;
  const int shifts[3] = {21, 10, 0};
  const int widths[3] = {11, 11, 10};
  for (int pass = 0; pass < 3; ++pass) {
    const int sh = shifts[pass];
    const int nb = 1 << widths[pass];
    for (int i = tid; i < nb; i += T) hist[i] = 0;
    __syncthreads();
    for (int i = tid; i < n; i += T) {
      const uint32_t key = key_of(i);
      const bool match = pass == 0 ? true : ((key >> (sh + widths[pass])) == prefix);
      if (match) atomicAdd(&hist[(key >> sh) & (nb - 1)], 1u);
    }
    __syncthreads();
    block_exclusive_scan(hist, nb, tot);
    // find b with hist[b] <= kk < hist[b+1] (exclusive prefix)
    for (int b = tid; b < nb; b += T) {
      const uint32_t lo = hist[b];
      const uint32_t hi = (b + 1 < nb) ? hist[b + 1] : 0xffffffffu;
      if (lo <= static_cast<uint32_t>(kk) && static_cast<uint32_t>(kk) < hi) {
        sel[0] = b;
        sel[1] = kk - static_cast<int>(lo);
      }
    }
    __syncthreads();
    prefix = (prefix << widths[pass]) | static_cast<uint32_t>(sel[0]);
    kk = sel[1];
    __syncthreads();
  }
  return prefix;
}

__global__ void __launch_bounds__(1024)
k_stats(const float* __restrict__ img, const int* __restrict__ pix, int n_valid, long long npix,
        int in_smem, double* __restrict__ stats64, float* __restrict__ stats32) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* hist = reinterpret_cast<uint32_t*>(smem);            // 2048
  uint32_t* tot = hist + 2048;                                    // 64
  int* sel = reinterpret_cast<int*>(tot + 64);                    // 8
  double* wbuf = reinterpret_cast<double*>(sel + 8);              // 2048 window values
  float* vals = reinterpret_cast<float*>(wbuf + 2048);            // n_valid (if in_smem)
  __shared__ int wcount;
  __shared__ int lcount;
  const int ch = blockIdx.x;
  const float* im = img + static_cast<long long>(ch) * npix;
  if (in_smem)
    for (int i = threadIdx.x; i < n_valid; i += blockDim.x) vals[i] = im[pix[i]];
  __syncthreads();
  auto xval = [&](int i) -> float { return in_smem ? vals[i] : im[pix[i]]; };
  auto key_x = [&](int i) -> uint32_t { return f2key(xval(i)); };

  const int n = n_valid;
  const int k1 = (n - 1) / 2, k2 = n / 2;
  const uint32_t key1 = block_select(n, k1, key_x, hist, tot, sel);
  uint32_t key2 = key1;
  if (k2 != k1) key2 = block_select(n, k2, key_x, hist, tot, sel);
  const double x1 = static_cast<double>(key2f(key1)), x2 = static_cast<double>(key2f(key2));
  const double med = (k1 == k2) ? x1 : (x1 + x2) / 2.0;
  const float m32 = static_cast<float>(med);
  auto key_d = [&](int i) -> uint32_t { return f2key(fabsf(xval(i) - m32)); };
  const uint32_t d1k = block_select(n, k1, key_d, hist, tot, sel);
  uint32_t d2k = d1k;
  if (k2 != k1) d2k = block_select(n, k2, key_d, hist, tot, sel);
  const float v1 = key2f(d1k), v2 = key2f(d2k);
  const float margin = 4.0f * (ulpf(v2) + ulpf(m32)) + 4.0f * ulpf(fmaxf(v2, fabsf(m32)));
  const float vlo = v1 - margin, vhi = v2 + margin;
  if (threadIdx.x == 0) { wcount = 0; lcount = 0; }
  __syncthreads();
  int my_l = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float x = xval(i);
    const float d = fabsf(x - m32);
    if (d < vlo) {
      ++my_l;
    } else if (d <= vhi) {
      const int s = atomicAdd(&wcount, 1);
      if (s < 2048) wbuf[s] = fabs(static_cast<double>(x) - med);
    }
  }
  atomicAdd(&lcount, my_l);
  __syncthreads();
  const int nw = wcount, L = lcount;
  double mad = 0.0;
  bool ok = nw <= 2048 && k1 - L >= 0 && k2 - L < nw;
  // more than half the pixels equal an exactly representable median: MAD = 0
  const bool zero_mad = (v2 == 0.0f) && (static_cast<double>(m32) == med);
  if (zero_mad) ok = true;
  if (ok && !zero_mad) {
    // ranks inside the window by counting (ties broken by slot index)
    const int r1 = k1 - L, r2 = k2 - L;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) {
      const double v = wbuf[i];
      int r = 0;
      for (int j = 0; j < nw; ++j) {
        const double u = wbuf[j];
        r += (u < v || (u == v && j < i)) ? 1 : 0;
      }
      if (r == r1) reinterpret_cast<double*>(tot)[0] = v;
      if (r == r2) reinterpret_cast<double*>(tot)[1] = v;
    }
    __syncthreads();
    const double d1 = reinterpret_cast<double*>(tot)[0], d2 = reinterpret_cast<double*>(tot)[1];
    mad = (k1 == k2) ? d1 : (d1 + d2) / 2.0;
  }
  if (threadIdx.x == 0) {
    if (!ok) atomicExch(&g_detect_status, 2);
    stats64[2 * ch] = med;
    stats64[2 * ch + 1] = ok ? mad : nan("");
    stats32[2 * ch] = m32;
    stats32[2 * ch + 1] = (ok && mad > 0.0) ? static_cast<float>(1.0 / (kMadToSigma * mad)) : 0.0f;
  }
}

__global__ void k_stats32(const double* __restrict__ s64, int n_chan, float* __restrict__ s32) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_chan) return;
  const double med = s64[2 * f], mad = s64[2 * f + 1];
  s32[2 * f] = static_cast<float>(med);
  s32[2 * f + 1] = mad > 0.0 ? static_cast<float>(1.0 / (kMadToSigma * mad)) : 0.0f;
}

// ------------------------------------------------- standardise + transpose
// z[p][k] = (x[chan0 + k][pix[p]] - med) * inv, tiles of 32 pixels x kZtK
// channels (256 threads, kZtK / 8 reads in flight per thread).
constexpr int kZtK = 64;
__global__ void __launch_bounds__(256)
k_ztrans(const float* __restrict__ img, const int* __restrict__ pix, int n_valid, long long npix, int chan0,
         int nc, const float* __restrict__ stats32, float* __restrict__ z) {
  __shared__ float t[kZtK][33];
  const int p0 = blockIdx.x * 32, k0 = blockIdx.y * kZtK;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;    // 32 x 8
  const int p = p0 + tx;
  const long long px = p < n_valid ? pix[p] : 0;
#pragma unroll
  for (int jj = 0; jj < kZtK / 8; ++jj) {
    const int j = ty + 8 * jj, k = k0 + j;
    float v = 0.f;
    if (k < nc && p < n_valid) {
      const int ch = chan0 + k;
      const float x = __ldg(img + static_cast<long long>(ch) * npix + px);
      v = (x - __ldg(stats32 + 2 * ch)) * __ldg(stats32 + 2 * ch + 1);
    }
    t[j][tx] = v;
  }
  __syncthreads();
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) {
    const int pp = p0 + ty + 8 * jj;
#pragma unroll
    for (int u = 0; u < kZtK / 32; ++u) {
      const int k = k0 + 32 * u + tx;
      if (pp < n_valid && k < nc) z[static_cast<long long>(pp) * nc + k] = t[32 * u + tx][ty + 8 * jj];
    }
  }
}

// --------------------------------------------------------------- a9 sort
// words per pixel of the running-median step stream
__host__ __device__ __forceinline__ int walk_stride(int nc, int h) {
  return (nc + ((h + 3) & ~3) + 3) & ~3;
}

// Stream codes: a rank word of 0xffff is no element; in a band stream
// (band-relative ranks) 0xfffe is an element below the band and 0xfffd one
// above it.
constexpr uint32_t kRankNone = 0xffffu, kRankBelow = 0xfffeu, kRankAbove = 0xfffdu;

// Stable LSD radix sort of m keys with 16-bit payloads in shared memory by the
// whole CTA: four passes of 8 bits; each warp ranks a contiguous segment
// (in-warp ranks by an 8-ballot multisplit, per-warp digit histograms at a
// padded pitch, so an exclusive scan in digit-major order gives every
// (digit, warp) its stable output offset).  The sorted keys end in ks / is.
//   sw: the warps that rank segments (<= blockDim / 32).  All 32 for the band
//   too: with 8 (a scan over a quarter of the digit counters) the idle warps
//   waited at the barriers and the sort took longer.
__device__ void lsd_sort(uint32_t* ks, uint16_t* is, uint32_t* kd, uint16_t* id, int m, uint32_t* hist,
                         uint32_t* tot, int sw) {
  const int W = sw;
  const int HP = W + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int seg = warp < W ? ((m + W - 1) / W + 31) / 32 * 32 : 0;   // idle warps rank nothing
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int pass = 0; pass < 4; ++pass) {
    const int sh = 8 * pass;
    for (int i = threadIdx.x; i < 256 * HP; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int i = lane; i < seg; i += 32) {
      const int k = warp * seg + i;
      if (k < m) atomicAdd(&hist[((ks[k] >> sh) & 255u) * HP + warp], 1u);
    }
    __syncthreads();
    block_exclusive_scan(hist, 256 * HP, tot);
    for (int b = 0; b < seg; b += 32) {
      const int k = warp * seg + b + lane;
      const bool valid = k < m;
      const uint32_t key = valid ? ks[k] : 0u;
      const uint32_t d = (key >> sh) & 255u;
      // lanes holding the same digit: one ballot per digit bit
      unsigned peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
      for (int bit = 0; bit < 8; ++bit) {
        const bool x = (d >> bit) & 1u;
        const unsigned bb = __ballot_sync(0xffffffffu, x);
        peers &= x ? bb : ~bb;
      }
      if (valid) {
        const uint32_t pos = hist[d * HP + warp] + __popc(peers & lt_mask);
        kd[pos] = key;
        id[pos] = is[k];
      }
      __syncwarp();
      if (valid && lane == __ffs(peers) - 1) hist[d * HP + warp] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    uint32_t* t1 = ks; ks = kd; kd = t1;
    uint16_t* t2 = is; is = id; id = t2;
  }
}

// The step stream from per-channel ranks rk (shared memory): step k inserts
// channel k + h and removes channel k - h - 1, stored at index k + H (H = h
// rounded up to 4) as (insert rank, remove rank); indices below H hold the
// insert-only steps that build the first window.  16-byte coalesced stores.
__device__ void write_stream(const uint16_t* rk, int nc, int h, uint32_t* sp) {
  const int H = (h + 3) & ~3;
  const int S = walk_stride(nc, h);
  for (int q = threadIdx.x; q < S / 4; q += blockDim.x) {
    uint32_t wv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = 4 * q + u;
      const int cin = i - H + h, cout = i - H - h - 1;
      const uint32_t rin = (cin >= 0 && cin < nc) ? rk[cin] : kRankNone;
      const uint32_t rout = (cout >= 0 && i - H < nc) ? rk[cout] : kRankNone;
      wv[u] = rin | (rout << 16);
    }
    reinterpret_cast<uint4*>(sp)[q] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
  }
}

// Full ranks of one pixel spectrum per CTA iteration: the sorted values
// (sv [pixel][nc]) and the step stream of absolute ranks.  With a pixel list
// (the band walk's failures) iteration i ranks list[i], i < *n_list.
__global__ void __launch_bounds__(1024)
k_rank(const float* __restrict__ z, int n_valid, int nc, int h, float* __restrict__ sv,
       uint32_t* __restrict__ steps, const int* __restrict__ list, const int* __restrict__ n_list) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int W = blockDim.x >> 5;
  uint32_t* hist = reinterpret_cast<uint32_t*>(smem);           // 256 * (W + 1)
  uint32_t* tot = hist + 256 * (W + 1);                          // 32
  uint32_t* ka = tot + 32;
  uint32_t* kb = ka + nc;
  uint16_t* ia = reinterpret_cast<uint16_t*>(kb + nc);
  uint16_t* ib = ia + nc;
  const int n_items = list ? min(*n_list, n_valid) : n_valid;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int p = list ? list[it] : it;
    const float* zp = z + static_cast<long long>(p) * nc;
#pragma unroll 4
    for (int k = threadIdx.x; k < nc; k += blockDim.x) {
      ka[k] = f2key(__ldg(zp + k));
      ia[k] = static_cast<uint16_t>(k);
    }
    __syncthreads();
    lsd_sort(ka, ia, kb, ib, nc, hist, tot, W);
    float* svp = sv + static_cast<long long>(p) * nc;
    for (int r = threadIdx.x; r < nc; r += blockDim.x) {
      svp[r] = key2f(ka[r]);
      ib[ia[r]] = static_cast<uint16_t>(r);                     // channel -> rank
    }
    __syncthreads();
    write_stream(ib, nc, h, steps + static_cast<long long>(p) * walk_stride(nc, h));
    __syncthreads();
  }
}

// Bin of the 256-bin histogram hg holding element `target` (0-based, in key
// order) and the count below that bin; run by one warp.
__device__ __forceinline__ void find_bin(const uint32_t* hg, int target, int* bin, int* below) {
  const int lane = threadIdx.x & 31;
  uint32_t c[8], s = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    c[u] = hg[lane * 8 + u];
    s += c[u];
  }
  uint32_t incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  uint32_t run = incl - s;
  const uint32_t tg = static_cast<uint32_t>(target);
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    if (run <= tg && tg < run + c[u]) {
      *bin = lane * 8 + u;
      *below = static_cast<int>(run);
    }
    run += c[u];
  }
}

constexpr int kRankMaxPerThread = 16;   // band ranking: nc <= 16 * 1024

// Band ranks of one pixel spectrum per CTA iteration.  The walk of a long
// coarse channel needs exact ranks only inside the band [r_lo, r_lo + B) of
// the middle ranks; below and above it a count suffices.  Two radix-select
// rounds over the 16 high key bits find the 16-bit buckets holding ranks r_lo
// and r_lo + B - 1; the keys from the lower bucket's start to the upper
// bucket's end (the band, its bucket mates and any ties) are compacted in
// channel order and sorted stably, so the m-th of them has the stable rank
// c_lo + m (c_lo = keys below the lower bucket), as in the full sort.  Output:
// the band's sorted values (sv [pixel][0 .. B)) and the stream of band ranks
// with the below / above codes.
template <int KPT>   // keys per thread: nc <= KPT * 1024
__global__ void __launch_bounds__(1024)
k_rank_band(const float* __restrict__ z, int n_valid, int nc, int h, int r_lo, int B, float* __restrict__ sv,
            uint32_t* __restrict__ steps) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int W = blockDim.x >> 5;
  uint32_t* hist = reinterpret_cast<uint32_t*>(smem);           // 256 * (W + 1): sort; 3 * 256 + 512: select
  uint32_t* tot = hist + 256 * (W + 1);                          // 32
  uint32_t* ka = tot + 32;
  uint32_t* kb = ka + nc;
  uint16_t* ia = reinterpret_cast<uint16_t*>(kb + nc);
  uint16_t* ib = ia + nc;
  __shared__ int sel[8];                                         // d_lo, d_hi, c1_lo, c1_hi, e_lo, e_hi, c2_lo, m
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int r_hi = r_lo + B - 1;
  for (int p = blockIdx.x; p < n_valid; p += gridDim.x) {
    const float* zp = z + static_cast<long long>(p) * nc;
    // channel i * blockDim + t in register i: a warp's lanes hold 32 consecutive channels
    uint32_t key[KPT];
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      const int k = i * blockDim.x + threadIdx.x;
      key[i] = k < nc ? f2key(__ldg(zp + k)) : 0u;
    }
    uint32_t* h1 = hist;
    uint32_t* h2lo = hist + 256;
    uint32_t* h2hi = hist + 512;
    uint32_t* cnt = hist + 768;                                  // per-chunk candidate counts
    for (int i = threadIdx.x; i < 768; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    // round 1: the top byte (shared atomics; equal digits within a warp are
    // serialised by the shared-memory pipe, not by issued instructions)
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      if (i * static_cast<int>(blockDim.x) >= nc) break;
      if (i * blockDim.x + threadIdx.x < nc) atomicAdd(&h1[key[i] >> 24], 1u);
    }
    __syncthreads();
    if (warp == 0) {
      find_bin(h1, r_lo, &sel[0], &sel[2]);
      find_bin(h1, r_hi, &sel[1], &sel[3]);
    }
    __syncthreads();
    const uint32_t d_lo = sel[0], d_hi = sel[1];
    // round 2: the second byte among keys of the two boundary top bytes
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      if (i * static_cast<int>(blockDim.x) >= nc) break;
      const bool valid = i * blockDim.x + threadIdx.x < nc;
      const uint32_t t = key[i] >> 24, d = (key[i] >> 16) & 255u;
      if (valid && t == d_lo) atomicAdd(&h2lo[d], 1u);
      else if (valid && t == d_hi) atomicAdd(&h2hi[d], 1u);
    }
    __syncthreads();
    if (warp == 0) {
      int dummy;
      find_bin(h2lo, r_lo - sel[2], &sel[4], &sel[6]);
      find_bin(d_hi == d_lo ? h2lo : h2hi, r_hi - sel[3], &sel[5], &dummy);
    }
    __syncthreads();
    const uint32_t v_lo = (d_lo << 24) | (static_cast<uint32_t>(sel[4]) << 16);
    const uint32_t v_hi = (d_hi << 24) | (static_cast<uint32_t>(sel[5]) << 16) | 0xffffu;
    const int c_lo = sel[2] + sel[6];                            // keys below v_lo
    // compaction of the candidates in channel order: chunk (i, warp) is
    // channels [i * blockDim + 32 warp, + 32)
    const int n_chunks = (nc + blockDim.x - 1) / blockDim.x * W;
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      if (i * static_cast<int>(blockDim.x) >= nc) break;
      const bool valid = i * blockDim.x + threadIdx.x < nc;
      const bool cand = valid && key[i] >= v_lo && key[i] <= v_hi;
      const unsigned bc = __ballot_sync(0xffffffffu, cand);
      if (lane == 0) cnt[i * W + warp] = __popc(bc);
    }
    __syncthreads();
    if (warp == 0) {
      // exclusive scan of the n_chunks (<= 512) counts, 16 per lane
      const int per = (n_chunks + 31) / 32;
      uint32_t s = 0;
      for (int u = 0; u < per; ++u) {
        const int j = lane * per + u;
        if (j < n_chunks) s += cnt[j];
      }
      uint32_t incl = s;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      uint32_t run = incl - s;
      for (int u = 0; u < per; ++u) {
        const int j = lane * per + u;
        if (j < n_chunks) {
          const uint32_t c = cnt[j];
          cnt[j] = run;
          run += c;
        }
      }
      if (lane == 31) sel[7] = static_cast<int>(incl);
    }
    __syncthreads();
    const int m = sel[7];
    uint16_t* rk = ib;                                           // channel -> band rank or code, after the sort
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      if (i * static_cast<int>(blockDim.x) >= nc) break;
      const int k = i * blockDim.x + threadIdx.x;
      const bool valid = k < nc;
      const bool cand = valid && key[i] >= v_lo && key[i] <= v_hi;
      const unsigned bc = __ballot_sync(0xffffffffu, cand);
      if (cand) {
        const uint32_t pos = cnt[i * W + warp] + __popc(bc & lt_mask);
        ka[pos] = key[i];
        ia[pos] = static_cast<uint16_t>(k);
      }
    }
    __syncthreads();
    lsd_sort(ka, ia, kb, ib, m, hist, tot, W);
    // candidate j has stable rank c_lo + j, band rank j - (r_lo - c_lo)
    const int off = r_lo - c_lo;
    float* svp = sv + static_cast<long long>(p) * nc;
    for (int j = threadIdx.x; j < B; j += blockDim.x) svp[j] = key2f(ka[off + j]);
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      const int b = j - off;
      rk[ia[j]] = static_cast<uint16_t>(b < 0 ? kRankBelow : (b >= B ? kRankAbove : static_cast<uint32_t>(b)));
    }
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      const int k = i * blockDim.x + threadIdx.x;
      if (k < nc && (key[i] < v_lo || key[i] > v_hi))
        rk[k] = static_cast<uint16_t>(key[i] < v_lo ? kRankBelow : kRankAbove);
    }
    __syncthreads();
    write_stream(rk, nc, h, steps + static_cast<long long>(p) * walk_stride(nc, h));
    __syncthreads();
  }
}

// --------------------------------------------------------- a9 running median
// The walk keeps, per pixel spectrum, the set of ranks inside the current
// window as a bitset over B ranks (the full walk: every rank, B >= nc; the
// band walk: the middle 2048 ranks of the band stream, whose elements below
// and above the band are only counted).  A cursor word W with lt = the number of
// set bits in words below W finds any order statistic of the band in a few
// word steps, since consecutive windows move it by at most one element; an
// insert or remove below W moves lt by one, so no step needs a search for a
// removed element.  A pixel's outputs may be split into S segments of
// consecutive channels, each walked by its own thread from the window before
// its first output (built from the inserts of the stream), so the chain of
// dependent steps a thread runs is about nc / S + w instead of nc + w / 2.

// Position of the n-th (0-based) set bit of x, n < popc(x): binary search on
// the population counts of the low halves.
__device__ __forceinline__ int select_bit(uint32_t x, int n) {
  int pos = 0;
  int c = __popc(x & 0xffffu);
  if (n >= c) { n -= c; pos += 16; x >>= 16; }
  c = __popc(x & 0xffu);
  if (n >= c) { n -= c; pos += 8; x >>= 8; }
  c = __popc(x & 0xfu);
  if (n >= c) { n -= c; pos += 4; x >>= 4; }
  c = __popc(x & 0x3u);
  if (n >= c) { n -= c; pos += 2; x >>= 2; }
  return pos + (n >= static_cast<int>(x & 1u) ? 1 : 0);
}

struct WalkState {
  int below, above, band;   // window elements below, above and inside the band
  int W, lt;                // cursor word; set bits in the words below it
};

// Insert (sgn = +1) or remove (sgn = -1) band rank r (r < 0: below the band,
// r >= B: above it).  Ranks are distinct, so both flip one bit.  Bit b of a
// thread's set is word b / 32 at bits[(b / 32) * T] (the words of the
// threads of a CTA interleave).
template <bool BAND, int T>
__device__ __forceinline__ void walk_update(uint32_t* bits, int r, int B, int sgn, WalkState& s) {
  const bool inb = !BAND || static_cast<unsigned>(r) < static_cast<unsigned>(B);
  if (BAND) {
    s.below += r < 0 ? sgn : 0;
    s.above += r >= B ? sgn : 0;
  }
  if (inb) bits[(r >> 5) * T] ^= 1u << (r & 31);
  s.band += inb ? sgn : 0;
  s.lt += (inb && (r >> 5) < s.W) ? sgn : 0;
}

// Band positions of the window's lower and upper median (equal for an odd
// window); false if either lies outside the band.
template <bool BAND, int T>
__device__ __forceinline__ bool walk_median(const uint32_t* bits, WalkState& s, int& lo, int& hi) {
  const int below = BAND ? s.below : 0;
  const int size = below + s.band + (BAND ? s.above : 0);
  const int tb = ((size - 1) >> 1) - below;
  const bool even = (size & 1) == 0;
  if (tb < 0 || tb + (even ? 1 : 0) >= s.band) return false;
  // lt > tb >= 0 means a set bit below W; lt + popc(word W) <= tb < band means
  // a set bit above it: the cursor stays inside the set's words
  while (s.lt > tb) {
    --s.W;
    s.lt -= __popc(bits[s.W * T]);
  }
  uint32_t x = bits[s.W * T];
  int pc = __popc(x);
  while (s.lt + pc <= tb) {
    s.lt += pc;
    ++s.W;
    x = bits[s.W * T];
    pc = __popc(x);
  }
  const int b = select_bit(x, tb - s.lt);
  lo = (s.W << 5) + b;
  hi = lo;
  if (even) {
    // the next set bit: in this word above b, else in a following word
    const uint32_t rest = b < 31 ? x & (0xfffffffeu << b) : 0u;
    if (rest) {
      hi = (s.W << 5) + __ffs(rest) - 1;
    } else {
      int w2 = s.W + 1;
      uint32_t y = bits[w2 * T];
      while (y == 0u) y = bits[++w2 * T];
      hi = (w2 << 5) + __ffs(y) - 1;
    }
  }
  return true;
}

// Applies f(index, word) to words [w0, w1) of a pixel's step stream, read in
// 16-byte chunks two chunks ahead; stops when f returns false.
template <class F>
__device__ __forceinline__ bool for_steps(const uint4* __restrict__ st4, int w0, int w1, F&& f) {
  const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
  const int ce = (w1 + 3) >> 2;
  int c = w0 >> 2;
  uint4 a = c < ce ? st4[c] : zero4, b = c + 1 < ce ? st4[c + 1] : zero4;
  for (; c < ce; ++c) {
    const uint4 nx = c + 2 < ce ? st4[c + 2] : zero4;
    const uint32_t sw[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = (c << 2) + q;
      if (i >= w0 && i < w1 && !f(i, sw[q])) return false;
    }
    a = b;
    b = nx;
  }
  return true;
}

constexpr int kWalkThreads = 64;   // full walk: nc / 32 words per thread
constexpr int kBandWordsMax = 64;  // band walk: up to 2048 ranks
constexpr int kBandThreads = 128;

// One thread per (pixel, segment) walks the segment's outputs over the step
// stream written by k_rank / k_rank_band and writes each window's median
// ranks, lower | upper << 16 (equal for an odd window; band ranks for a band
// stream), to med [pixel][nc]; k_median_sub then applies them with all
// threads (the gathers of the sorted values would otherwise sit in the walk's
// chain of dependent steps).
//   BAND: the band stream (nwords * 32 band ranks); a segment whose median
//     leaves the band gives up, and its pixel is listed once in fail (k_rank
//     and the full walk redo it).
//   !BAND: the full rank set (nwords = nc / 32 rounded up); with a pixel list
//     (the band walk's failures) item i walks list[i], i < *n_list.
// seg_len is a multiple of 4, so every segment's steps start on a chunk.
template <bool BAND, int T>
__global__ void __launch_bounds__(T)
k_walk(const uint32_t* __restrict__ steps, int n_valid, int nc, int h, int n_seg, int seg_len, int nwords,
       uint32_t* __restrict__ med, const int* __restrict__ list, const int* __restrict__ n_list,
       int* __restrict__ fail, int* __restrict__ n_fail) {
  extern __shared__ uint32_t bits_all[];
  const int t = threadIdx.x;
  const int item = (blockIdx.x * T + t) / n_seg;
  const int sg = (blockIdx.x * T + t) - item * n_seg;
  uint32_t* bits = bits_all + t;
  int p = item;
  bool live = item < n_valid;
  if (!BAND && list) {
    live = item < min(*n_list, n_valid);
    p = live ? list[item] : 0;
  }
  bool gave_up = false;
  if (live) {
    for (int w = 0; w < nwords; ++w) bits[w * T] = 0u;
    const int B = nwords * 32;
    const int H = (h + 3) & ~3;
    const int k0 = sg * seg_len, k1 = min(nc, k0 + seg_len);
    const uint4* st4 = reinterpret_cast<const uint4*>(steps + static_cast<long long>(p) * walk_stride(nc, h));
    uint32_t* mo = med + static_cast<long long>(p) * nc - H;
    WalkState s{0, 0, 0, 0, 0};
    auto rank_of = [&](uint32_t r) {
      if (!BAND) return static_cast<int>(r);
      return r == kRankBelow ? -1 : (r == kRankAbove ? B : static_cast<int>(r));
    };
    // the window before output k0: channels [k0 - 1 - h, k0 - 1 + h]; channel
    // j is inserted by word j - h + H (the words below H build the first window)
    const int wa = max(H - h, H + k0 - 1 - 2 * h), wb = H + k0;
    bool ok = for_steps(st4, wa, wb, [&](int, uint32_t word) {
      const uint32_t rin = word & 0xffffu;
      if (rin != kRankNone) walk_update<BAND, T>(bits, rank_of(rin), B, 1, s);
      return true;
    });
    ok = ok && for_steps(st4, H + k0, H + k1, [&](int i, uint32_t word) {
      const uint32_t rin = word & 0xffffu, rout = word >> 16;
      if (rin != kRankNone) walk_update<BAND, T>(bits, rank_of(rin), B, 1, s);
      if (rout != kRankNone) walk_update<BAND, T>(bits, rank_of(rout), B, -1, s);
      int lo, hi;
      if (!walk_median<BAND, T>(bits, s, lo, hi)) return false;
      mo[i] = static_cast<uint32_t>(lo) | (static_cast<uint32_t>(hi) << 16);
      return true;
    });
    if (!ok) {
      if (BAND) gave_up = true;
      else atomicExch(&g_detect_status, 3);            // the full set always holds the median
    }
  }
  if (BAND) {
    // a pixel's segments are adjacent threads of one warp (n_seg divides 32)
    const unsigned any = __ballot_sync(0xffffffffu, gave_up);
    const int lane = t & 31, first = lane - sg;
    const unsigned mine = ((n_seg >= 32) ? 0xffffffffu : ((1u << n_seg) - 1u)) << first;
    if (live && sg == 0 && (any & mine)) {
      const int slot = atomicAdd(n_fail, 1);
      if (slot < n_valid) fail[slot] = p;
    }
  }
}

// z' = z - (v[lower] + v[upper]) / 2 for every voxel, v the pixel's sorted
// values (the band's for a band stream) and med the median ranks the walk left.
__global__ void k_median_sub(float* __restrict__ zbuf, const float* __restrict__ sv,
                             const uint32_t* __restrict__ med, int n_valid, int nc) {
  if ((nc & 3) == 0) {
    // four channels per thread: 16-byte reads of z and of the rank words
    const int nq = nc >> 2;
    const long long n = static_cast<long long>(n_valid) * nq;
    for (long long v = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; v < n;
         v += static_cast<long long>(gridDim.x) * blockDim.x) {
      const int p = static_cast<int>(v / nq);
      const uint4 r = __ldg(reinterpret_cast<const uint4*>(med) + v);
      const float* svp = sv + static_cast<long long>(p) * nc;
      float4* zq = reinterpret_cast<float4*>(zbuf) + v;
      float4 x = *zq;
      x.x -= 0.5f * (__ldg(svp + (r.x & 0xffffu)) + __ldg(svp + (r.x >> 16)));
      x.y -= 0.5f * (__ldg(svp + (r.y & 0xffffu)) + __ldg(svp + (r.y >> 16)));
      x.z -= 0.5f * (__ldg(svp + (r.z & 0xffffu)) + __ldg(svp + (r.z >> 16)));
      x.w -= 0.5f * (__ldg(svp + (r.w & 0xffffu)) + __ldg(svp + (r.w >> 16)));
      *zq = x;
    }
    return;
  }
  const long long n = static_cast<long long>(n_valid) * nc;
  for (long long v = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; v < n;
       v += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int p = static_cast<int>(v / nc);
    const uint32_t r = __ldg(med + v);
    const float* svp = sv + static_cast<long long>(p) * nc;
    const float m = 0.5f * (__ldg(svp + (r & 0xffffu)) + __ldg(svp + (r >> 16)));
    zbuf[v] -= m;
  }
}

// -------------------------------------------------------- a10 matched filter
// Shared-memory slot of staged spectrum index i: one pad word after every 8,
// so thread t's window (starting at index 8t, slot 9t) lies in its own banks
// and every load of the window is the thread's base slot plus a constant.
__host__ __device__ constexpr int mf_slot(int i) { return i + (i >> 3); }

// Boxcars for kVox consecutive channels from the register prefix P; BOUNDS
// keeps only widths that fit inside the coarse channel (edge chunks).
template <bool BOUNDS>
__device__ __forceinline__ void mf_chunk(const float (&P)[kWin + 1], int k0, int nc, float (&best)[kVox],
                                         int (&bw)[kVox]) {
#pragma unroll
  for (int j = 0; j < kVox; ++j) { best[j] = -INFINITY; bw[j] = 0; }
#pragma unroll
  for (int wi = 0; wi < kNW; ++wi) {
    const int w = width_of(wi);
    const int lo = (w - 1) / 2, hi = w - 1 - lo;
#pragma unroll
    for (int j = 0; j < kVox; ++j) {
      if (!BOUNDS || (k0 + j - lo >= 0 && k0 + j + hi <= nc - 1)) {
        const float S = P[j + kMaxLo + hi + 1] - P[j + kMaxLo - lo];
        const float v = S * rsqrt_width(wi);
        if (v > best[j]) { best[j] = v; bw[j] = w; }
      }
    }
  }
}

__global__ void __launch_bounds__(128)
k_mf(const float* __restrict__ zbuf, int n_valid, int nc, float* __restrict__ snr,
     uint8_t* __restrict__ width, uint32_t hist_key0, int n_bins, unsigned long long* __restrict__ ghist) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n_s = kMaxLo + nc + kMaxHi + kVox;
  float* s = reinterpret_cast<float*>(smem);                 // [mf_slot(n_s)]
  uint32_t* hist = reinterpret_cast<uint32_t*>(s + mf_slot(n_s) + 1);
  for (int i = threadIdx.x; i < n_bins; i += blockDim.x) hist[i] = 0;
  const float floor_snr = key2f(hist_key0 << kHistShift);
  for (int p = blockIdx.x; p < n_valid; p += gridDim.x) {
    const float* zp = zbuf + static_cast<long long>(p) * nc;
    __syncthreads();
    // stage the spectrum at slots kMaxLo .. kMaxLo + nc - 1, zeros around it;
    // 16-byte loads, several in flight per thread
    if ((nc & 3) == 0 && (reinterpret_cast<uintptr_t>(zp) & 15) == 0) {
      const float4* z4 = reinterpret_cast<const float4*>(zp);
      const int n4 = nc >> 2;
#pragma unroll 4
      for (int v = threadIdx.x; v < n4; v += blockDim.x) {
        const float4 q = __ldg(z4 + v);
        const int i = kMaxLo + 4 * v;
        s[mf_slot(i)] = q.x;
        s[mf_slot(i + 1)] = q.y;
        s[mf_slot(i + 2)] = q.z;
        s[mf_slot(i + 3)] = q.w;
      }
      for (int i = threadIdx.x; i < kMaxLo; i += blockDim.x) s[mf_slot(i)] = 0.f;
      for (int i = kMaxLo + nc + threadIdx.x; i < n_s; i += blockDim.x) s[mf_slot(i)] = 0.f;
    } else {
#pragma unroll 4
      for (int i = threadIdx.x; i < n_s; i += blockDim.x) {
        const int k = i - kMaxLo;
        s[mf_slot(i)] = (k >= 0 && k < nc) ? __ldg(zp + k) : 0.f;
      }
    }
    __syncthreads();
    for (int k0 = threadIdx.x * kVox; k0 < nc; k0 += blockDim.x * kVox) {
      const float* sw = s + mf_slot(k0);                     // k0 is a multiple of 8
      float P[kWin + 1];
      P[0] = 0.f;
#pragma unroll
      for (int i = 0; i < kWin; ++i) P[i + 1] = P[i] + sw[mf_slot(i)];   // channel k0 - 49 + i
      float best[kVox];
      int bw[kVox];
      if (k0 >= kMaxLo && k0 + kVox - 1 + kMaxHi <= nc - 1) mf_chunk<false>(P, k0, nc, best, bw);
      else mf_chunk<true>(P, k0, nc, best, bw);
      float* so = snr + static_cast<long long>(p) * nc + k0;
      uint8_t* wo = width + static_cast<long long>(p) * nc + k0;
      if (k0 + kVox <= nc && (reinterpret_cast<uintptr_t>(so) & 15) == 0 &&
          (reinterpret_cast<uintptr_t>(wo) & 7) == 0) {
        reinterpret_cast<float4*>(so)[0] = make_float4(best[0], best[1], best[2], best[3]);
        reinterpret_cast<float4*>(so)[1] = make_float4(best[4], best[5], best[6], best[7]);
        uint2 wb;
        wb.x = static_cast<uint32_t>(bw[0]) | (static_cast<uint32_t>(bw[1]) << 8) |
               (static_cast<uint32_t>(bw[2]) << 16) | (static_cast<uint32_t>(bw[3]) << 24);
        wb.y = static_cast<uint32_t>(bw[4]) | (static_cast<uint32_t>(bw[5]) << 8) |
               (static_cast<uint32_t>(bw[6]) << 16) | (static_cast<uint32_t>(bw[7]) << 24);
        *reinterpret_cast<uint2*>(wo) = wb;
      } else {
#pragma unroll
        for (int j = 0; j < kVox; ++j)
          if (k0 + j < nc) {
            so[j] = best[j];
            wo[j] = static_cast<uint8_t>(bw[j]);
          }
      }
#pragma unroll
      for (int j = 0; j < kVox; ++j) {
        if (k0 + j < nc && best[j] >= floor_snr) {
          int b = static_cast<int>((f2key(best[j]) >> kHistShift) - hist_key0);
          if (b >= n_bins) b = n_bins - 1;
          atomicAdd(&hist[b], 1u);
        }
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n_bins; i += blockDim.x)
    if (hist[i]) atomicAdd(ghist + i, static_cast<unsigned long long>(hist[i]));
}

// ------------------------------------------------- a11 exact BH cut, a12 NMS
// ln Q(s), Q the upper Gaussian tail (same formula as the host side).
__device__ double log_q_dev(double s) {
  if (s < 25.0) return log(0.5 * erfc(s * 0.70710678118654752440));
  const double s2 = s * s;
  const double series = 1.0 - 1.0 / s2 + 3.0 / (s2 * s2) - 15.0 / (s2 * s2 * s2) + 105.0 / (s2 * s2 * s2 * s2);
  return -0.5 * s2 - log(s * 2.50662827463100050242) + log(series);
}

// Values of one histogram bin (key >> kHistShift == kb; the top bin takes
// every larger key as well), for the exact BH step-up inside that bin.
__global__ void k_gather_bin(const float* __restrict__ snr, long long n, uint32_t kb, int top,
                             float* __restrict__ out, int cap, int* __restrict__ count) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float v = snr[i];
    const uint32_t b = f2key(v) >> kHistShift;
    if (b == kb || (top && b > kb)) {
      const int slot = atomicAdd(count, 1);
      if (slot < cap) out[slot] = v;
    }
  }
}

// Values of every histogram bin b with want[b] != 0 in one pass (keys at or
// above the top bin count as the top bin, as in k_gather_bin).
__global__ void k_gather_bins(const float* __restrict__ snr, long long n, uint32_t key0, int nb,
                              const uint8_t* __restrict__ want, float* __restrict__ out, int cap,
                              int* __restrict__ count) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float v = snr[i];
    const uint32_t kb = f2key(v) >> kHistShift;
    if (kb < key0) continue;
    const uint32_t b = min(kb - key0, static_cast<uint32_t>(nb - 1));
    if (want[b]) {
      const int slot = atomicAdd(count, 1);
      if (slot < cap) out[slot] = v;
    }
  }
}

// One detection as the kernels hand it to the host.
struct CandRec {
  int coarse, p, k, width;
  float snr, pad;
  double log10_p;
};

constexpr int kNmsCap = 256;          // detections a warp holds for one (pixel, coarse) pair
constexpr int kNmsWarps = 8;

// a12, one warp per (pixel, coarse) pair, pair q = p * n_coarse + c (the output
// order).  The pair's detections (SNR >= cut) are gathered in channel order;
// greedy NMS repeatedly accepts the undecided detection of highest SNR
// (lowest channel on ties) and suppresses the undecided ones within
// max(1, w / 2) channels of it, w the accepted width -- the same decisions as
// walking the list in descending SNR.  The accepted detections are written in
// channel order to a range reserved with one atomic per pair (counters[1]);
// pairs with more than kNmsCap detections go to the overflow list
// (counters[0]) for k_nms_big.
__global__ void __launch_bounds__(kNmsWarps * 32)
k_nms_warp(const float* __restrict__ snr, const uint8_t* __restrict__ width, const long long* __restrict__ vox0,
           const int* __restrict__ nfft, int n_coarse, long long n_pairs, float cut, int* __restrict__ ovf,
           int* __restrict__ counters, CandRec* __restrict__ out, int out_cap) {
  __shared__ uint32_t lk[kNmsWarps][kNmsCap];       // (k << 8) | width
  __shared__ float lv[kNmsWarps][kNmsCap];
  __shared__ uint8_t st[kNmsWarps][kNmsCap];        // 0 undecided, 1 accepted, 2 suppressed
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long q = static_cast<long long>(blockIdx.x) * kNmsWarps + warp;
  if (q >= n_pairs) return;                         // whole warps leave together
  const int p = static_cast<int>(q / n_coarse), c = static_cast<int>(q - static_cast<long long>(p) * n_coarse);
  const int nc = nfft[c];
  const long long base = vox0[c] + static_cast<long long>(p) * nc;
  const unsigned full = 0xffffffffu, lt = (1u << lane) - 1u;
  uint32_t* K = lk[warp];
  float* V = lv[warp];
  uint8_t* S = st[warp];
  int n = 0;
  bool over = false;
  // kNmsAhead chunks of 32 channels per iteration, their reads issued together
  constexpr int kNmsAhead = 8;
  for (int k0 = 0; k0 < nc && !over; k0 += 32 * kNmsAhead) {
    float v[kNmsAhead];
#pragma unroll
    for (int u = 0; u < kNmsAhead; ++u) {
      const int k = k0 + 32 * u + lane;
      v[u] = k < nc ? __ldg(snr + base + k) : -INFINITY;
    }
#pragma unroll
    for (int u = 0; u < kNmsAhead; ++u) {
      const int k = k0 + 32 * u + lane;
      const bool hit = v[u] >= cut;
      const unsigned m = __ballot_sync(full, hit);
      if (!m) continue;
      if (n + __popc(m) > kNmsCap) { over = true; break; }
      if (hit) {
        const int i = n + __popc(m & lt);
        K[i] = (static_cast<uint32_t>(k) << 8) | width[base + k];
        V[i] = v[u];
        S[i] = 0;
      }
      n += __popc(m);
    }
  }
  if (over) {
    if (lane == 0) ovf[atomicAdd(counters, 1)] = static_cast<int>(q);   // for k_nms_big
    return;
  }
  __syncwarp();
  int n_acc = 0;
  for (;;) {
    float bv = -INFINITY;
    int bi = -1;
    for (int i = lane; i < n; i += 32)
      if (S[i] == 0 && (bi < 0 || V[i] > bv)) { bv = V[i]; bi = i; }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const float ov = __shfl_xor_sync(full, bv, o);
      const int oi = __shfl_xor_sync(full, bi, o);
      if (oi >= 0 && (bi < 0 || ov > bv || (ov == bv && oi < bi))) { bv = ov; bi = oi; }
    }
    if (bi < 0) break;
    const int ka = static_cast<int>(K[bi] >> 8);
    const int r = max(1, static_cast<int>(K[bi] & 255u) / 2);
    for (int i = lane; i < n; i += 32)
      if (S[i] == 0) {
        if (i == bi) S[i] = 1;
        else if (abs(static_cast<int>(K[i] >> 8) - ka) <= r) S[i] = 2;
      }
    __syncwarp();
    ++n_acc;
  }
  // the pair's accepted detections go to a range reserved here, in channel
  // order (pairs land in any order; the host orders them)
  int j = 0;
  if (lane == 0 && n_acc) j = atomicAdd(counters + 1, n_acc);
  j = __shfl_sync(full, j, 0);
  for (int i0 = 0; i0 < n; i0 += 32) {
    const int i = i0 + lane;
    const bool a = i < n && S[i] == 1;
    const unsigned m = __ballot_sync(full, a);
    if (a) {
      const int o = j + __popc(m & lt);
      if (o < out_cap) {
        CandRec rc;
        rc.coarse = c;
        rc.p = p;
        rc.k = static_cast<int>(K[i] >> 8);
        rc.width = static_cast<int>(K[i] & 255u);
        rc.snr = V[i];
        rc.pad = 0.f;
        rc.log10_p = log_q_dev(static_cast<double>(V[i])) * 0.43429448190325182765;
        out[o] = rc;
      }
    }
    j += __popc(m);
  }
}

// a12 for pairs with more than kNmsCap detections: one CTA per pair.  The
// detections are sorted by (SNR descending, channel ascending) with a bitonic
// sort in shared memory, then one warp walks them in that order against a
// bitmap of covered channels.  Shared memory: p2max 64-bit keys and two
// bitmaps of nc_max bits.
__global__ void __launch_bounds__(1024)
k_nms_big(const float* __restrict__ snr, const uint8_t* __restrict__ width, const long long* __restrict__ vox0,
          const int* __restrict__ nfft, int n_coarse, const int* __restrict__ ovf, int* __restrict__ counters,
          int p2max, float cut, CandRec* __restrict__ out, int out_cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(smem);       // [p2max]
  uint32_t* cov = reinterpret_cast<uint32_t*>(keys + p2max);                     // [p2max / 32]
  uint32_t* acc = cov + p2max / 32;                                              // [p2max / 32]
  uint32_t* scan = acc + p2max / 32;                                             // [1024]
  uint32_t* wtot = scan + 1024;                                                  // [32]
  __shared__ int s_n;
  if (blockIdx.x >= counters[0]) return;
  const int q = ovf[blockIdx.x];
  const int p = q / n_coarse, c = q - p * n_coarse;
  const int nc = nfft[c];
  const long long base = vox0[c] + static_cast<long long>(p) * nc;
  const int tid = threadIdx.x, T = blockDim.x;
  if (tid == 0) s_n = 0;
  for (int i = tid; i < p2max / 32; i += T) { cov[i] = 0u; acc[i] = 0u; }
  __syncthreads();
  // gather in channel order
  for (int k0 = 0; k0 < nc; k0 += T) {
    const int k = k0 + tid;
    const float v = k < nc ? snr[base + k] : -INFINITY;
    const bool hit = v >= cut;
    scan[tid] = hit ? 1u : 0u;
    __syncthreads();
    block_exclusive_scan(scan, T, wtot);
    const int n0 = s_n;
    if (hit) {
      const uint32_t lo = (static_cast<uint32_t>(k) << 8) | width[base + k];
      keys[n0 + scan[tid]] = (static_cast<unsigned long long>(~f2key(v)) << 32) | lo;
    }
    __syncthreads();
    if (tid == T - 1) s_n = n0 + static_cast<int>(scan[tid]) + (hit ? 1 : 0);
    __syncthreads();
  }
  const int n = s_n;
  int p2 = 1;
  while (p2 < n) p2 <<= 1;
  for (int i = n + tid; i < p2; i += T) keys[i] = ~0ull;
  __syncthreads();
  for (int size = 2; size <= p2; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = tid; t < p2 / 2; t += T) {
        const int i = (t / stride) * 2 * stride + (t % stride);
        const int j = i + stride;
        const bool up = (i & size) == 0;
        const unsigned long long a = keys[i], b = keys[j];
        if ((a > b) == up) { keys[i] = b; keys[j] = a; }
      }
      __syncthreads();
    }
  if (tid < 32) {
    for (int i = 0; i < n; ++i) {
      const uint32_t lo = static_cast<uint32_t>(keys[i]);
      const int k = static_cast<int>(lo >> 8);
      if ((cov[k >> 5] >> (k & 31)) & 1u) continue;
      const int r = max(1, static_cast<int>(lo & 255u) / 2);
      const int a = max(0, k - r), b = min(nc - 1, k + r);
      for (int x = a + tid; x <= b; x += 32) atomicOr(&cov[x >> 5], 1u << (x & 31));
      if (tid == 0) acc[k >> 5] |= 1u << (k & 31);
      __syncwarp();
    }
  }
  __syncthreads();
  const int words = (nc + 31) / 32;
  // reserve the pair's output range: count the accepted detections
  {
    int my = 0;
    for (int i = tid; i < words; i += T) my += __popc(acc[i]);
    for (int o = 16; o; o >>= 1) my += __shfl_xor_sync(0xffffffffu, my, o);
    if (tid == 0) s_n = 0;
    __syncthreads();
    if ((tid & 31) == 0 && my) atomicAdd(&s_n, my);
    __syncthreads();
    if (tid == 0) s_n = s_n ? atomicAdd(counters + 1, s_n) : 0;
    __syncthreads();
  }
  int j0 = s_n;
  for (int w0 = 0; w0 < words; w0 += T) {
    const int wi = w0 + tid;
    const uint32_t bits = wi < words ? acc[wi] : 0u;
    scan[tid] = __popc(bits);
    __syncthreads();
    block_exclusive_scan(scan, T, wtot);
    int o = j0 + static_cast<int>(scan[tid]);
    for (uint32_t b = bits; b; b &= b - 1) {
      const int k = wi * 32 + __ffs(b) - 1;
      if (o < out_cap) {
        CandRec rc;
        rc.coarse = c;
        rc.p = p;
        rc.k = k;
        rc.width = width[base + k];
        rc.snr = snr[base + k];
        rc.pad = 0.f;
        rc.log10_p = log_q_dev(static_cast<double>(rc.snr)) * 0.43429448190325182765;
        out[o] = rc;
      }
      ++o;
    }
    __syncthreads();
    if (tid == T - 1) scan[0] = scan[tid] + __popc(bits);
    __syncthreads();
    j0 += static_cast<int>(scan[0]);
    __syncthreads();
  }
}

// scatter [pixel][k] arrays of one coarse block into [chan][N][N] (stage isolation)
template <class T>
__global__ void k_scatter(const T* __restrict__ src, const int* __restrict__ pix, int n_valid, int nc,
                          int chan0, long long npix, T* __restrict__ dst) {
  const long long n = static_cast<long long>(n_valid) * nc;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int p = static_cast<int>(i / nc), k = static_cast<int>(i - static_cast<long long>(p) * nc);
    dst[static_cast<long long>(chan0 + k) * npix + pix[p]] = src[i];
  }
}

__global__ void k_u8_to_i32(const uint8_t* __restrict__ a, long long n, int32_t* __restrict__ b) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    b[i] = a[i];
}

// ------------------------------------------------------------------ host side
double log_q(double s) {
  // ln of the upper Gaussian tail Q(s)
  if (s < 25.0) return std::log(0.5 * std::erfc(s / std::sqrt(2.0)));
  const double s2 = s * s;
  const double series = 1.0 - 1.0 / s2 + 3.0 / (s2 * s2) - 15.0 / (s2 * s2 * s2) + 105.0 / (s2 * s2 * s2 * s2);
  return -0.5 * s2 - std::log(s * std::sqrt(2.0 * M_PI)) + std::log(series);
}

double q_inverse(double p) {
  // upper-tail Gaussian quantile by bisection on log_q
  double lo = -10.0, hi = 60.0;
  const double lp = std::log(p);
  for (int i = 0; i < 200; ++i) {
    const double mid = 0.5 * (lo + hi);
    if (log_q(mid) > lp) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

int window_channels(double df, double span) {
  int w = static_cast<int>(std::floor(span / df)) + 1;
  while (w * df <= span) ++w;
  if (w % 2 == 0) ++w;
  return w;
}

constexpr int kGatherCap = 1 << 23;     // values of the open histogram bins (exact BH step-up), at least
constexpr int kCandCap = 1 << 21;       // candidates written by the NMS kernels, at least

struct DetectPlan {
  int n, n_coarse, n_chan;
  long long npix;
  std::vector<int> pix;        // in-horizon pixel indices
  std::vector<int> nfft, chan0, half;
  std::vector<long long> vox0; // voxel offset of each coarse block in snr/width
  long long n_vox = 0;
  int max_nc = 0;
  int max_steps = 0;
  int n_valid = 0;
  bool stats_in_smem = false;
  int gather_cap = 0;          // values of the open histogram bins gathered at once
  int cand_cap = 0;            // candidate records written by the NMS kernels
};

DetectPlan make_plan(int n_chan, int n, double cell, int n_coarse, const int32_t* nfft,
                     double coarse_bw, double span) {
  DetectPlan p;
  p.n = n;
  p.n_coarse = n_coarse;
  p.n_chan = n_chan;
  p.npix = static_cast<long long>(n) * n;
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      const double l = static_cast<double>(c - n / 2) * cell;
      const double m = static_cast<double>(r - n / 2) * cell;
      if (l * l + m * m < 1.0) p.pix.push_back(r * n + c);
    }
  p.n_valid = static_cast<int>(p.pix.size());
  int c0 = 0;
  for (int c = 0; c < n_coarse; ++c) {
    p.nfft.push_back(nfft[c]);
    p.chan0.push_back(c0);
    p.vox0.push_back(p.n_vox);
    p.half.push_back(window_channels(coarse_bw / nfft[c], span) / 2);
    p.n_vox += static_cast<long long>(p.n_valid) * nfft[c];
    p.max_nc = std::max(p.max_nc, static_cast<int>(nfft[c]));
    p.max_steps = std::max(p.max_steps, walk_stride(nfft[c], p.half.back()));
    c0 += nfft[c];
  }
  p.stats_in_smem = (static_cast<size_t>(p.n_valid) * 4 + 8192 + 256 + 32 + 16384) <= 231000;
  // the capacities grow with the search: a search of few spectra per channel
  // (skewed noise images) can pass about one test in a thousand
  const long long grow = std::min<long long>(p.n_vox / 512, 1LL << 26);
  p.gather_cap = static_cast<int>(std::max<long long>(kGatherCap, grow));
  p.cand_cap = static_cast<int>(std::max<long long>(kCandCap, grow));
  return p;
}

constexpr int kMaxBins = 2048;

struct DetectWs {
  int* pix;
  double* stats64;
  float* stats32;
  float* zbuf;
  float* sv;
  uint32_t* steps;
  uint32_t* med;         // [pixel][channel] median ranks of the current coarse block
  int* fail;             // pixels whose band walk gave up
  float* snr;
  uint8_t* width;
  unsigned long long* hist;
  float* vals;
  long long* vox0;
  int* nfft;
  int* ovf;
  CandRec* recs;
  int* count;            // [0] gathered values, [1] overflow pairs, [2] candidates, [3] band-walk failures
  uint8_t* want;         // [kMaxBins] bins gathered in one pass
};

long long n_pairs_of(const DetectPlan& p) { return static_cast<long long>(p.n_valid) * p.n_coarse; }

DetectWs carve_detect(void* ws, size_t bytes, const DetectPlan& p, size_t* need) {
  Carver c(ws, bytes);
  DetectWs w;
  const size_t blk = static_cast<size_t>(p.n_valid) * p.max_nc;
  const long long np = std::max(1LL, n_pairs_of(p));
  w.pix = c.take<int>(p.n_valid > 0 ? p.n_valid : 1);
  w.stats64 = c.take<double>(2 * static_cast<size_t>(p.n_chan));
  w.stats32 = c.take<float>(2 * static_cast<size_t>(p.n_chan));
  w.zbuf = c.take<float>(blk);
  w.sv = c.take<float>(blk);
  w.steps = c.take<uint32_t>(static_cast<size_t>(p.n_valid) * p.max_steps);
  w.med = c.take<uint32_t>(blk);
  w.fail = c.take<int>(p.n_valid > 0 ? p.n_valid : 1);
  w.snr = c.take<float>(static_cast<size_t>(p.n_vox));
  w.width = c.take<uint8_t>(static_cast<size_t>(p.n_vox));
  w.hist = c.take<unsigned long long>(kMaxBins);
  w.vals = c.take<float>(p.gather_cap);
  w.vox0 = c.take<long long>(p.n_coarse);
  w.nfft = c.take<int>(p.n_coarse);
  w.ovf = c.take<int>(np);
  w.recs = c.take<CandRec>(p.cand_cap);
  w.count = c.take<int>(4);
  w.want = c.take<uint8_t>(kMaxBins);
  *need = c.used;
  return w;
}

int validate(int n_chan, int n, double cell, int n_coarse, const int32_t* nfft) {
  if (n_chan <= 0 || n_coarse <= 0 || !nfft || !(cell > 0.0)) return OVRO_ERR_INVALID_ARG;
  if (!is_pow2(n) || n < 16 || n > 1024) return OVRO_ERR_UNSUPPORTED;
  long long tot = 0;
  for (int c = 0; c < n_coarse; ++c) {
    if (nfft[c] <= 0) return OVRO_ERR_INVALID_ARG;
    if (nfft[c] > 16384) return OVRO_ERR_UNSUPPORTED;
    tot += nfft[c];
  }
  if (tot != n_chan) return OVRO_ERR_INVALID_ARG;
  return OVRO_OK;
}

// a8 for nc consecutive channel images starting at img; statistics to s64/s32.
int run_stats_block(const float* img, int nc, double* s64, float* s32, const DetectPlan& p, const DetectWs& w,
                    cudaStream_t st) {
  const size_t base = 2048 * 4 + 64 * 4 + 8 * 4 + 2048 * 8;
  // staged: the channel's in-horizon pixels copied to shared memory once (one
  // CTA per SM); unstaged: every pass re-reads them through L2, and two CTAs
  // share an SM, one loading while the other selects
  auto stats = [&](int staged) -> int {
    const size_t sm = base + (staged ? static_cast<size_t>(p.n_valid) * 4 : 0);
    OVRO_CUDA_TRY(cudaFuncSetAttribute(k_stats, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm)));
    OVRO_PROF("k_stats", st);
    k_stats<<<nc, 1024, sm, st>>>(img, w.pix, p.n_valid, p.npix, staged, s64, s32);
    OVRO_LAUNCH_CHECK();
    return OVRO_OK;
  };
  if (!p.stats_in_smem) return stats(0);
  const std::string key = tune_key("k_stats", {p.n_valid, nc});
  int staged = tuned(key, 0);                       // L2 reads won at 256^2 x 8192 channels
  if (tuning(st))
    if (int e = tune_pick(key, {1, 0}, stats, st, &staged)) return e;
  return stats(staged);
}

// a9 + a10 for coarse block c, whose nfft[c] images start at img_block:
// snr/width [pixel][k] at vox0[c] in the workspace; the histogram accumulates.
int run_filter_coarse(int c, const float* img_block, const DetectPlan& p, const DetectWs& w, uint32_t hist_key0,
                      int n_bins, float* d_zp_out, cudaStream_t st) {
  const int nsm = num_sms();
  const int nc = p.nfft[c];
  {
    dim3 g((p.n_valid + 31) / 32, (nc + kZtK - 1) / kZtK);
    OVRO_PROF("k_ztrans", st);
    k_ztrans<<<g, 256, 0, st>>>(img_block, w.pix, p.n_valid, p.npix, 0, nc, w.stats32 + 2LL * p.chan0[c], w.zbuf);
    OVRO_LAUNCH_CHECK();
  }
  {
    // Coarse channels longer than the band: band ranks and the band walk for
    // every pixel, then full ranks and the full walk for the pixels whose
    // median left the band.  Shorter ones: full ranks and the full walk.
    // the band: the middle 2048 ranks (a window median's rank wanders about
    // nc / (2 sqrt(W)) from the middle for a stationary spectrum: 99 ranks at
    // 8192 channels, W = 1707; on the skewed noise images of the full workload
    // a band of 1024 sent enough pixels to the full walk to cost more than the
    // smaller sort saved: 13.7 against 12.6 ms per step for ranks and walk)
    const int band_words = kBandWordsMax;
    const int band = band_words * 32;
    const bool use_band = nc > band && nc <= kRankMaxPerThread * 1024;
    const int threads = 1024, W = threads / 32;      // one CTA per SM (shared memory): all 32 warps
    const size_t sm_rank = (256 * (W + 1) + 32) * 4 + static_cast<size_t>(nc) * 12;
    OVRO_CUDA_TRY(cudaFuncSetAttribute(k_rank, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sm_rank)));
    OVRO_CUDA_TRY(cudaFuncSetAttribute(k_rank_band<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sm_rank)));
    OVRO_CUDA_TRY(cudaFuncSetAttribute(k_rank_band<kRankMaxPerThread>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sm_rank)));
    // CTAs per SM (each CTA loops over pixels; the outputs do not depend on it)
    auto rank = [&](int per_sm) -> int {
      const int blocks = std::min(p.n_valid, per_sm * nsm);
      OVRO_PROF("k_rank", st);
      if (use_band && nc <= 8 * 1024)
        k_rank_band<8><<<blocks, threads, sm_rank, st>>>(w.zbuf, p.n_valid, nc, p.half[c], nc / 2 - band / 2, band,
                                                         w.sv, w.steps);
      else if (use_band)
        k_rank_band<kRankMaxPerThread><<<blocks, threads, sm_rank, st>>>(w.zbuf, p.n_valid, nc, p.half[c],
                                                                         nc / 2 - band / 2, band, w.sv, w.steps);
      else
        k_rank<<<blocks, threads, sm_rank, st>>>(w.zbuf, p.n_valid, nc, p.half[c], w.sv, w.steps, nullptr, nullptr);
      OVRO_LAUNCH_CHECK();
      return OVRO_OK;
    };
    const std::string rkey = tune_key(use_band ? "k_rank_band" : "k_rank", {p.n_valid, nc});
    int per_sm = tuned(rkey, 16);
    if (tuning(st))
      if (int e = tune_pick(rkey, {1, 2, 4, 16}, rank, st, &per_sm)) return e;

    // S segments per pixel (S divides 32), tuned per shape; a trial ranks
    // again, since the fallback rewrites the failed pixels' streams
    const int nwords = (nc + 31) / 32;
    const size_t sm_full = static_cast<size_t>(nwords) * kWalkThreads * 4;
    const size_t sm_band = static_cast<size_t>(band_words) * kBandThreads * 4;
    OVRO_CUDA_TRY(cudaFuncSetAttribute(k_walk<false, kWalkThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sm_full)));
    auto rank_walk = [&](int n_seg) -> int {
      if (int e = rank(per_sm)) return e;
      const int seg_len = ((nc + n_seg - 1) / n_seg + 3) & ~3;
      const long long thr = static_cast<long long>(p.n_valid) * n_seg;
      if (use_band) {
        OVRO_CUDA_TRY(cudaMemsetAsync(w.count + 3, 0, sizeof(int), st));
        {
          OVRO_PROF("k_walk", st);
          k_walk<true, kBandThreads><<<static_cast<int>((thr + kBandThreads - 1) / kBandThreads), kBandThreads,
                                       sm_band, st>>>(w.steps, p.n_valid, nc, p.half[c], n_seg, seg_len, band_words,
                                                      w.med, nullptr, nullptr, w.fail, w.count + 3);
          OVRO_LAUNCH_CHECK();
        }
        OVRO_PROF("k_rank", st);
        k_rank<<<std::min(p.n_valid, nsm), threads, sm_rank, st>>>(w.zbuf, p.n_valid, nc, p.half[c], w.sv, w.steps,
                                                                   w.fail, w.count + 3);
        OVRO_LAUNCH_CHECK();
      }
      OVRO_PROF("k_walk", st);
      k_walk<false, kWalkThreads><<<static_cast<int>((thr + kWalkThreads - 1) / kWalkThreads), kWalkThreads,
                                    sm_full, st>>>(w.steps, p.n_valid, nc, p.half[c], n_seg, seg_len, nwords, w.med,
                                                   use_band ? w.fail : nullptr, use_band ? w.count + 3 : nullptr,
                                                   nullptr, nullptr);
      OVRO_LAUNCH_CHECK();
      return OVRO_OK;
    };
    const std::string key = tune_key("k_walk", {p.n_valid, nc});
    int n_seg = tuned(key, 2);
    if (tuning(st))
      if (int e = tune_pick(key, {1, 2, 4}, rank_walk, st, &n_seg)) return e;
    if (int e = rank_walk(n_seg)) return e;
    OVRO_PROF("k_median_sub", st);
    k_median_sub<<<8 * nsm, 256, 0, st>>>(w.zbuf, w.sv, w.med, p.n_valid, nc);
    OVRO_LAUNCH_CHECK();
  }
  if (d_zp_out) {
    k_scatter<float><<<4 * nsm, 256, 0, st>>>(w.zbuf, w.pix, p.n_valid, nc, p.chan0[c], p.npix, d_zp_out);
    OVRO_LAUNCH_CHECK();
  }
  {
    const size_t sm = static_cast<size_t>(mf_slot(kMaxLo + nc + kMaxHi + kVox) + 1) * 4 +
                      static_cast<size_t>(n_bins) * 4;
    OVRO_CUDA_TRY(cudaFuncSetAttribute(k_mf, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm)));
    // CTAs per SM; trial launches histogram into scratch (the real histogram
    // accumulates over coarse channels and must count every voxel once)
    auto mf = [&](int per_sm, unsigned long long* hist) -> int {
      const int blocks = std::min(p.n_valid, per_sm * nsm);
      OVRO_PROF("k_mf", st);
      k_mf<<<blocks, 128, sm, st>>>(w.zbuf, p.n_valid, nc, w.snr + p.vox0[c], w.width + p.vox0[c], hist_key0,
                                    n_bins, hist);
      OVRO_LAUNCH_CHECK();
      return OVRO_OK;
    };
    const std::string key = tune_key("k_mf", {p.n_valid, nc});
    int per_sm = tuned(key, 24);
    if (tuning(st)) {
      unsigned long long* scratch = reinterpret_cast<unsigned long long*>(w.vals);
      if (int e = tune_pick(key, {6, 12, 24, 48}, [&](int v) { return mf(v, scratch); }, st, &per_sm)) return e;
    }
    if (int e = mf(per_sm, w.hist)) return e;
  }
  return OVRO_OK;
}

int run_filter(const float* d_img, const DetectPlan& p, const DetectWs& w, uint32_t hist_key0, int n_bins,
               float* d_zp_out, cudaStream_t st) {
  for (int c = 0; c < p.n_coarse; ++c)
    if (int e = run_filter_coarse(c, d_img + static_cast<long long>(p.chan0[c]) * p.npix, p, w, hist_key0, n_bins,
                                  d_zp_out, st))
      return e;
  return OVRO_OK;
}

// Device address of the detection status word (per device).
int* detect_status_ptr() {
  static int* cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (!cache[dev]) {
    void* q = nullptr;
    if (cudaGetSymbolAddress(&q, g_detect_status) != cudaSuccess) return nullptr;
    cache[dev] = static_cast<int*>(q);
  }
  return cache[dev];
}

uint32_t host_f2key(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
float host_key2f(uint32_t k) {
  const uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// histogram floor and bin count for a mode
void hist_range(const ovro_detect_params& prm, uint32_t* key0, int* n_bins) {
  double floor_snr;
  if (prm.mode == OVRO_DETECT_FIXED) floor_snr = prm.nsigma;
  else floor_snr = q_inverse(prm.alpha) - 0.01;
  if (floor_snr < 0.25) floor_snr = 0.25;
  // round the floor down to a bin edge
  *key0 = host_f2key(static_cast<float>(floor_snr)) >> kHistShift;
  const uint32_t top = (host_f2key(64.0f) >> kHistShift);
  int nb = static_cast<int>(top > *key0 ? top - *key0 : 0) + 1;   // + overflow bin
  if (nb > kMaxBins) nb = kMaxBins;
  *n_bins = nb;
}

// Exact Benjamini-Hochberg cut from the SNR histogram.  count(SNR >= s) is
// known exactly at every bin edge, so a bin either surely holds the step-up
// threshold's rank range (every value in it passes: cut at its lower edge),
// surely cannot (no value passes), or is ambiguous -- then its values are
// gathered and ranked exactly.  Bins are taken from the lowest one where a
// rejection is possible upwards; the first passing value found is the cut
// (the largest rank that passes).
//
// Verdict for bin b: 0 no value can pass, 1 every value passes (*lo_edge is
// the cut), 2 ambiguous, 3 empty bin.
int bh_bin_verdict(const unsigned long long* hist, int nb, uint32_t key0, double m, double alpha, int b,
                   float* lo_edge, unsigned long long* above_next) {
  unsigned long long above = 0;                    // count(SNR >= upper edge of bin b)
  for (int x = nb - 1; x > b; --x) above += hist[x];
  *above_next = above;
  *lo_edge = host_key2f((key0 + b) << kHistShift);
  if (hist[b] == 0) return 3;
  auto passes = [&](double s, unsigned long long rank) {
    return log_q(s) <= std::log(alpha * static_cast<double>(rank) / m);
  };
  const bool top = b == nb - 1;
  if (!top && !passes(static_cast<double>(host_key2f((key0 + b + 1) << kHistShift)), above + hist[b])) return 0;
  if (passes(static_cast<double>(*lo_edge), above + 1)) return 1;
  return 2;
}

// The lowest passing value among the values of one bin (descending order),
// ranks above_next + 1, above_next + 2, ...; returns 1 and *cut, or 0.
int bh_resolve(const float* v_desc, long long n, unsigned long long above_next, double m, double alpha,
               float* cut) {
  long long best = -1;
  for (long long j = 0; j < n; ++j)
    if (log_q(v_desc[j]) <= std::log(alpha * static_cast<double>(above_next + j + 1) / m)) best = j;
  if (best < 0) return 0;
  *cut = v_desc[best];
  return 1;
}

// Values of bin b of this search (device gather; synchronises).
int gather_bin(const DetectWs& w, const DetectPlan& p, uint32_t key0, int nb, int b, std::vector<float>& v,
               cudaStream_t st) {
  const int nsm = num_sms();
  OVRO_CUDA_TRY(cudaMemsetAsync(w.count, 0, sizeof(int), st));
  k_gather_bin<<<8 * nsm, 256, 0, st>>>(w.snr, p.n_vox, key0 + b, b == nb - 1 ? 1 : 0, w.vals, p.gather_cap,
                                        w.count);
  OVRO_LAUNCH_CHECK();
  int nv = 0;
  OVRO_CUDA_TRY(cudaMemcpyAsync(&nv, w.count, sizeof(int), cudaMemcpyDeviceToHost, st));
  OVRO_CUDA_TRY(cudaStreamSynchronize(st));
  if (nv > p.gather_cap) return OVRO_ERR_CAPACITY;
  v.resize(nv);
  if (nv) OVRO_CUDA_TRY(cudaMemcpy(v.data(), w.vals, nv * sizeof(float), cudaMemcpyDeviceToHost));
  return OVRO_OK;
}

// Values of one histogram bin in descending order.  Below the top bin every
// key of the bin shares its upper 16 bits, so a counting sort over the lower
// 16 bits orders them (keys are monotone in the value, equal keys equal values).
void sort_bin_desc(std::vector<float>& v, bool top) {
  if (top || v.size() < 4096) {
    std::sort(v.begin(), v.end(), std::greater<float>());
    return;
  }
  const uint32_t hi = host_f2key(v[0]) >> kHistShift;
  std::vector<uint32_t> cnt(1u << kHistShift, 0);
  for (float x : v) ++cnt[host_f2key(x) & ((1u << kHistShift) - 1)];
  size_t o = 0;
  for (int k = (1 << kHistShift) - 1; k >= 0; --k)
    for (uint32_t c = cnt[k]; c; --c) v[o++] = host_key2f((hi << kHistShift) | static_cast<uint32_t>(k));
}

// Single-search cut.  Returns 0 with *cut set, 1 when nothing is rejected, or
// an error status.  Bins are visited upwards: the first bin every value of
// which passes gives the cut; an open bin below it is resolved from its
// values.  The values of all the open bins below that one are gathered in one
// pass over the SNR cube (per bin if together they exceed the gather buffer).
int bh_cut(const std::vector<unsigned long long>& hist, uint32_t key0, int nb, double m, double alpha,
           const DetectWs& w, const DetectPlan& p, cudaStream_t st, float* cut) {
  std::vector<int> verdict(nb);
  std::vector<float> lo(nb);
  std::vector<unsigned long long> above(nb);
  int b1 = nb;
  unsigned long long open_total = 0;
  int n_open = 0;
  for (int b = 0; b < nb; ++b) {
    verdict[b] = bh_bin_verdict(hist.data(), nb, key0, m, alpha, b, &lo[b], &above[b]);
    if (verdict[b] == 1) {
      b1 = b;
      break;
    }
    if (verdict[b] == 2) {
      open_total += hist[b];
      ++n_open;
    }
  }
  std::vector<std::vector<float>> bins(nb);
  const bool one_pass = n_open > 1 && open_total <= static_cast<unsigned long long>(p.gather_cap);
  if (one_pass) {
    std::vector<uint8_t> want(nb, 0);
    for (int b = 0; b < b1; ++b) want[b] = verdict[b] == 2;
    OVRO_CUDA_TRY(cudaMemcpyAsync(w.want, want.data(), nb, cudaMemcpyHostToDevice, st));
    OVRO_CUDA_TRY(cudaMemsetAsync(w.count, 0, sizeof(int), st));
    k_gather_bins<<<8 * num_sms(), 256, 0, st>>>(w.snr, p.n_vox, key0, nb, w.want, w.vals, p.gather_cap, w.count);
    OVRO_LAUNCH_CHECK();
    int nv = 0;
    OVRO_CUDA_TRY(cudaMemcpyAsync(&nv, w.count, sizeof(int), cudaMemcpyDeviceToHost, st));
    OVRO_CUDA_TRY(cudaStreamSynchronize(st));
    if (static_cast<unsigned long long>(nv) != open_total) return OVRO_ERR_CAPACITY;
    std::vector<float> all(nv);
    if (nv) {
      OVRO_CUDA_TRY(cudaMemcpyAsync(all.data(), w.vals, nv * sizeof(float), cudaMemcpyDeviceToHost, st));
      OVRO_CUDA_TRY(cudaStreamSynchronize(st));
    }
    for (float v : all) {
      const uint32_t kb = host_f2key(v) >> kHistShift;
      bins[std::min<uint32_t>(kb - key0, static_cast<uint32_t>(nb - 1))].push_back(v);
    }
  }
  for (int b = 0; b < b1; ++b) {
    if (verdict[b] != 2) continue;
    std::vector<float>& vals = bins[b];
    if (!one_pass) {
      if (hist[b] > static_cast<unsigned long long>(p.gather_cap)) return OVRO_ERR_CAPACITY;
      if (int e = gather_bin(w, p, key0, nb, b, vals, st)) return e;
    }
    if (static_cast<unsigned long long>(vals.size()) != hist[b]) return OVRO_ERR_CAPACITY;
    sort_bin_desc(vals, b == nb - 1);
    if (bh_resolve(vals.data(), static_cast<long long>(vals.size()), above[b], m, alpha, cut)) return 0;
  }
  if (b1 < nb) {
    *cut = lo[b1];
    return 0;
  }
  return 1;
}

}  // namespace
}  // namespace ovro

extern "C" {

int ovro_default_widths(int32_t* h_out_or_null) {
  if (h_out_or_null)
    for (int i = 0; i < ovro::kNW; ++i) h_out_or_null[i] = ovro::width_of(i);
  return ovro::kNW;
}

size_t ovro_detect_workspace_size(int n_chan, int image_size, int n_coarse, const int32_t* h_nfft) {
  using namespace ovro;
  // the in-horizon pixel count depends on the cell; size for the largest (all pixels)
  if (validate(n_chan, image_size, 1.0, n_coarse, h_nfft) != OVRO_OK) return 0;
  DetectPlan p = make_plan(n_chan, image_size, 1e-9, n_coarse, h_nfft, 24000.0, 5000.0);
  size_t need = 0;
  carve_detect(nullptr, 0, p, &need);
  return need;
}

int ovro_detect_stats(const float* d_img, int n_chan, int image_size, double cell_dircos, double* d_stats,
                      void* d_ws, size_t ws_bytes, void* stream) {
  using namespace ovro;
  if (!d_img || !d_stats) return OVRO_ERR_INVALID_ARG;
  const int32_t one[1] = {n_chan};
  if (int e = validate(n_chan, image_size, cell_dircos, 1, one)) return e;
  DetectPlan p = make_plan(n_chan, image_size, cell_dircos, 1, one, 24000.0, 5000.0);
  if (p.n_valid == 0) return OVRO_ERR_INVALID_ARG;
  size_t need = 0;
  DetectWs w = carve_detect(d_ws, ws_bytes, p, &need);
  if (int e = check_workspace(d_ws, ws_bytes, need)) return e;
  cudaStream_t st = as_stream(stream);
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.pix, p.pix.data(), p.pix.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  if (int e = run_stats_block(d_img, n_chan, w.stats64, w.stats32, p, w, st)) return e;
  OVRO_CUDA_TRY(cudaMemcpyAsync(d_stats, w.stats64, 2 * sizeof(double) * n_chan, cudaMemcpyDeviceToDevice, st));
  return OVRO_OK;
}

int ovro_detect_filter(const float* d_img, const double* d_stats, int n_chan, int image_size,
                       double cell_dircos, int n_coarse, const int32_t* h_nfft,
                       const ovro_detect_params* params, float* d_zp_or_null, float* d_snr,
                       int32_t* d_width, void* d_ws, size_t ws_bytes, void* stream) {
  using namespace ovro;
  if (!d_img || !d_stats || !params || !d_snr || !d_width) return OVRO_ERR_INVALID_ARG;
  if (int e = validate(n_chan, image_size, cell_dircos, n_coarse, h_nfft)) return e;
  DetectPlan p = make_plan(n_chan, image_size, cell_dircos, n_coarse, h_nfft, params->coarse_bw_hz,
                           params->highpass_hz);
  if (p.n_valid == 0) return OVRO_ERR_INVALID_ARG;
  size_t need = 0;
  DetectWs w = carve_detect(d_ws, ws_bytes, p, &need);
  if (int e = check_workspace(d_ws, ws_bytes, need)) return e;
  cudaStream_t st = as_stream(stream);
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.pix, p.pix.data(), p.pix.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  k_stats32<<<(n_chan + 255) / 256, 256, 0, st>>>(d_stats, n_chan, w.stats32);
  OVRO_LAUNCH_CHECK();
  uint32_t key0;
  int nb;
  hist_range(*params, &key0, &nb);
  OVRO_CUDA_TRY(cudaMemsetAsync(w.hist, 0, kMaxBins * sizeof(unsigned long long), st));
  if (d_zp_or_null) OVRO_CUDA_TRY(cudaMemsetAsync(d_zp_or_null, 0, sizeof(float) * n_chan * p.npix, st));
  OVRO_CUDA_TRY(cudaMemsetAsync(d_snr, 0, sizeof(float) * n_chan * p.npix, st));
  OVRO_CUDA_TRY(cudaMemsetAsync(d_width, 0, sizeof(int32_t) * n_chan * p.npix, st));
  if (int e = run_filter(d_img, p, w, key0, nb, d_zp_or_null, st)) return e;
  const int nsm = num_sms();
  for (int c = 0; c < p.n_coarse; ++c) {
    k_scatter<float><<<4 * nsm, 256, 0, st>>>(w.snr + p.vox0[c], w.pix, p.n_valid, p.nfft[c], p.chan0[c],
                                               p.npix, d_snr);
    OVRO_LAUNCH_CHECK();
    // widths: widen to int32 in the zbuf scratch, then scatter
    const long long nv = static_cast<long long>(p.n_valid) * p.nfft[c];
    int32_t* tmp = reinterpret_cast<int32_t*>(w.zbuf);
    k_u8_to_i32<<<4 * nsm, 256, 0, st>>>(w.width + p.vox0[c], nv, tmp);
    OVRO_LAUNCH_CHECK();
    k_scatter<int32_t><<<4 * nsm, 256, 0, st>>>(tmp, w.pix, p.n_valid, p.nfft[c], p.chan0[c], p.npix, d_width);
    OVRO_LAUNCH_CHECK();
  }
  return OVRO_OK;
}

}  // extern "C"

namespace ovro {

struct DetectCtx {
  DetectPlan p;
  DetectWs w;
  ovro_detect_params prm;
  uint32_t key0 = 0;
  int nb = 0;
  int n_chan = 0, image_size = 0;
  // host staging of the candidate records and their ordering, kept across
  // calls (their pages stay mapped)
  std::vector<CandRec> recs;
  std::vector<int> q_start, order;
};

size_t detect_ctx_workspace(int n_chan, int image_size, int n_coarse, const int32_t* h_nfft) {
  // the in-horizon pixel count depends on the cell; size for the largest (all pixels)
  if (validate(n_chan, image_size, 1.0, n_coarse, h_nfft) != OVRO_OK) return 0;
  DetectPlan p = make_plan(n_chan, image_size, 1e-9, n_coarse, h_nfft, 24000.0, 5000.0);
  size_t need = 0;
  carve_detect(nullptr, 0, p, &need);
  return need;
}

int detect_ctx_init(DetectCtx** out, int n_chan, int image_size, double cell, int n_coarse, const int32_t* h_nfft,
                    const ovro_detect_params* params, void* d_ws, size_t ws_bytes) {
  if (!out || !params) return OVRO_ERR_INVALID_ARG;
  *out = nullptr;
  if (params->mode != OVRO_DETECT_BH && params->mode != OVRO_DETECT_FIXED) return OVRO_ERR_INVALID_ARG;
  if (params->mode == OVRO_DETECT_BH && !(params->alpha > 0.0 && params->alpha <= 0.4))
    return OVRO_ERR_INVALID_ARG;
  if (!(params->highpass_hz > 0.0) || !(params->coarse_bw_hz > 0.0)) return OVRO_ERR_INVALID_ARG;
  if (int e = validate(n_chan, image_size, cell, n_coarse, h_nfft)) return e;
  DetectCtx* d = new DetectCtx;
  d->p = make_plan(n_chan, image_size, cell, n_coarse, h_nfft, params->coarse_bw_hz, params->highpass_hz);
  size_t need = 0;
  d->w = carve_detect(d_ws, ws_bytes, d->p, &need);
  if (d->p.n_valid > 0)
    if (int e = check_workspace(d_ws, ws_bytes, need)) {
      delete d;
      return e;
    }
  d->prm = *params;
  hist_range(*params, &d->key0, &d->nb);
  d->n_chan = n_chan;
  d->image_size = image_size;
  *out = d;
  return OVRO_OK;
}

int detect_ctx_valid_pixels(const DetectCtx* d) { return d ? d->p.n_valid : 0; }

int detect_ctx_upload(DetectCtx* d, cudaStream_t st) {
  if (!d) return OVRO_ERR_INVALID_ARG;
  const DetectPlan& p = d->p;
  if (p.n_valid == 0) return OVRO_OK;
  OVRO_CUDA_TRY(cudaMemcpyAsync(d->w.pix, p.pix.data(), p.pix.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  OVRO_CUDA_TRY(cudaMemcpyAsync(d->w.vox0, p.vox0.data(), p.n_coarse * sizeof(long long), cudaMemcpyHostToDevice, st));
  OVRO_CUDA_TRY(cudaMemcpyAsync(d->w.nfft, p.nfft.data(), p.n_coarse * sizeof(int), cudaMemcpyHostToDevice, st));
  return OVRO_OK;
}

int detect_ctx_begin(DetectCtx* d, cudaStream_t st) {
  if (!d) return OVRO_ERR_INVALID_ARG;
  if (d->p.n_valid == 0) return OVRO_OK;
  int* sp = detect_status_ptr();
  if (!sp) return OVRO_ERR_CUDA;
  OVRO_CUDA_TRY(cudaMemsetAsync(sp, 0, sizeof(int), st));
  OVRO_CUDA_TRY(cudaMemsetAsync(d->w.hist, 0, kMaxBins * sizeof(unsigned long long), st));
  return OVRO_OK;
}

int detect_ctx_coarse(DetectCtx* d, int c, const float* d_img_block, cudaStream_t st) {
  if (!d || !d_img_block || c < 0 || c >= d->p.n_coarse) return OVRO_ERR_INVALID_ARG;
  const DetectPlan& p = d->p;
  if (p.n_valid == 0) return OVRO_OK;
  const long long off = 2LL * p.chan0[c];
  if (int e = run_stats_block(d_img_block, p.nfft[c], d->w.stats64 + off, d->w.stats32 + off, p, d->w, st))
    return e;
  return run_filter_coarse(c, d_img_block, p, d->w, d->key0, d->nb, nullptr, st);
}

// a8-a10 for coarse channel c, also scattering z' into d_zp [n_chan][N][N].
int detect_ctx_coarse_zp(DetectCtx* d, int c, const float* d_img_block, float* d_zp, cudaStream_t st) {
  if (!d || !d_img_block || c < 0 || c >= d->p.n_coarse) return OVRO_ERR_INVALID_ARG;
  const DetectPlan& p = d->p;
  if (p.n_valid == 0) return OVRO_OK;
  const long long off = 2LL * p.chan0[c];
  if (int e = run_stats_block(d_img_block, p.nfft[c], d->w.stats64 + off, d->w.stats32 + off, p, d->w, st))
    return e;
  return run_filter_coarse(c, d_img_block, p, d->w, d->key0, d->nb, d_zp, st);
}

// The search's SNR histogram (synchronises; checks the device status word).
int detect_ctx_histogram(DetectCtx* d, std::vector<unsigned long long>& hist, cudaStream_t st) {
  hist.assign(d->nb, 0ull);
  if (d->p.n_valid == 0) return OVRO_OK;
  OVRO_CUDA_TRY(cudaMemcpyAsync(hist.data(), d->w.hist, d->nb * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                st));
  int status = 0;
  OVRO_CUDA_TRY(cudaMemcpyFromSymbolAsync(&status, g_detect_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
  OVRO_CUDA_TRY(cudaStreamSynchronize(st));
  return status ? OVRO_ERR_CAPACITY : OVRO_OK;
}

int detect_ctx_finish(DetectCtx* d, const double* h_chan_freq_hz, ovro_candidate* h_out, int max_out, int* n_out,
                      cudaStream_t st) {
  if (!d || !n_out || (max_out > 0 && !h_out) || max_out < 0 || !h_chan_freq_hz) return OVRO_ERR_INVALID_ARG;
  *n_out = 0;
  if (d->p.n_valid == 0) return OVRO_OK;
  // ---- a11: threshold
  std::vector<unsigned long long> hist;
  if (int e = detect_ctx_histogram(d, hist, st)) return e;
  const double m = static_cast<double>(d->p.n_valid) * d->n_chan;
  float cut;
  if (d->prm.mode == OVRO_DETECT_FIXED) {
    cut = static_cast<float>(d->prm.nsigma);
  } else {
    int e = bh_cut(hist, d->key0, d->nb, m, d->prm.alpha, d->w, d->p, st, &cut);
    if (e == 1) return OVRO_OK;        // nothing is rejected
    if (e) return e;
  }
  return detect_ctx_candidates(d, cut, h_chan_freq_hz, h_out, max_out, n_out, st);
}

// ---- a12: NMS on the device at a given cut, candidates in (pixel, coarse,
// channel) order (synchronises).
int detect_ctx_candidates(DetectCtx* d, float cut, const double* h_chan_freq_hz, ovro_candidate* h_out, int max_out,
                          int* n_out, cudaStream_t st) {
  if (!d || !n_out || (max_out > 0 && !h_out) || max_out < 0 || !h_chan_freq_hz) return OVRO_ERR_INVALID_ARG;
  *n_out = 0;
  const DetectPlan& p = d->p;
  if (p.n_valid == 0) return OVRO_OK;
  const DetectWs& w = d->w;
  const int image_size = d->image_size;
  const long long np = n_pairs_of(p);
  if (np > 0x7fffffffLL / 2) return OVRO_ERR_UNSUPPORTED;
  // one pass: each (pixel, coarse) pair's detections are written to a range
  // reserved by atomics; w.count[1] counts overflowing pairs, w.count[2] the
  // detections
  OVRO_CUDA_TRY(cudaMemsetAsync(w.count, 0, 4 * sizeof(int), st));
  const unsigned nms_blocks = static_cast<unsigned>((np + kNmsWarps - 1) / kNmsWarps);
  {
    OVRO_PROF("k_nms_warp", st);
    k_nms_warp<<<nms_blocks, kNmsWarps * 32, 0, st>>>(w.snr, w.width, w.vox0, w.nfft, p.n_coarse, np, cut, w.ovf,
                                                       w.count + 1, w.recs, p.cand_cap);
    OVRO_LAUNCH_CHECK();
  }
  int cnt[2] = {0, 0};
  OVRO_CUDA_TRY(cudaMemcpyAsync(cnt, w.count + 1, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  OVRO_CUDA_TRY(cudaStreamSynchronize(st));
  if (cnt[0] > 0) {
    int p2max = 32;
    while (p2max < p.max_nc) p2max <<= 1;
    const size_t big_sm = static_cast<size_t>(p2max) * 8 + 2 * static_cast<size_t>(p2max / 32) * 4 + 1056 * 4;
    OVRO_CUDA_TRY(cudaFuncSetAttribute(k_nms_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(big_sm)));
    k_nms_big<<<cnt[0], 1024, big_sm, st>>>(w.snr, w.width, w.vox0, w.nfft, p.n_coarse, w.ovf, w.count + 1, p2max,
                                            cut, w.recs, p.cand_cap);
    OVRO_LAUNCH_CHECK();
    OVRO_CUDA_TRY(cudaMemcpyAsync(cnt, w.count + 1, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    OVRO_CUDA_TRY(cudaStreamSynchronize(st));
  }
  const int total = cnt[1];
  *n_out = total;
  const int nw = std::min(total, p.cand_cap);
  if (nw > 0 && max_out > 0) {
    std::vector<CandRec>& recs = d->recs;
    if (recs.size() < static_cast<size_t>(nw)) recs.resize(nw);
    OVRO_CUDA_TRY(cudaMemcpyAsync(recs.data(), w.recs, nw * sizeof(CandRec), cudaMemcpyDeviceToHost, st));
    OVRO_CUDA_TRY(cudaStreamSynchronize(st));
    // (pixel, coarse) pair order, stable: a counting sort on q = p n_coarse + c
    const long long n_q = np;
    std::vector<int>& start = d->q_start;
    start.assign(static_cast<size_t>(n_q) + 1, 0);
    for (int i = 0; i < nw; ++i) ++start[static_cast<size_t>(recs[i].p) * p.n_coarse + recs[i].coarse + 1];
    for (long long q = 0; q < n_q; ++q) start[q + 1] += start[q];
    std::vector<int>& order = d->order;
    if (order.size() < static_cast<size_t>(nw)) order.resize(nw);
    for (int i = 0; i < nw; ++i) order[start[static_cast<size_t>(recs[i].p) * p.n_coarse + recs[i].coarse]++] = i;
    const int nout = std::min(nw, max_out);
    for (int q = 0; q < nout; ++q) {
      const CandRec& r = recs[order[q]];
      ovro_candidate& o = h_out[q];
      const int pixel = p.pix[r.p];
      o.coarse = r.coarse;
      o.fine = r.k;
      o.chan = p.chan0[r.coarse] + r.k;
      o.row = pixel / image_size;
      o.col = pixel % image_size;
      o.width = r.width;
      o.snr = r.snr;
      o.score = 0.f;
      o.freq_hz = h_chan_freq_hz[o.chan];
      o.log10_p = r.log10_p;
    }
  }
  if (total > max_out) return OVRO_ERR_CAPACITY;
  return total > p.cand_cap ? OVRO_ERR_CAPACITY : OVRO_OK;
}

int detect_ctx_bin_values(DetectCtx* d, int b, std::vector<float>& v, cudaStream_t st) {
  if (!d || b < 0 || b >= d->nb) return OVRO_ERR_INVALID_ARG;
  v.clear();
  if (d->p.n_valid == 0) return OVRO_OK;
  return gather_bin(d->w, d->p, d->key0, d->nb, b, v, st);
}

void detect_ctx_layout(const DetectCtx* d, uint32_t* key0, int* n_bins, long long* n_tests) {
  *key0 = d->key0;
  *n_bins = d->nb;
  *n_tests = static_cast<long long>(d->p.n_valid) * d->n_chan;
}

void detect_ctx_free(DetectCtx* d) { delete d; }

}  // namespace ovro

namespace ovro {

// Scratch of the scored search (the caller's scorer workspace).
struct ScoredWs {
  float* zp;          // [n_chan][N][N] high-passed standardised cube
  int32_t* trig;      // [max_triggers][3] (channel, row, col)
  float* x;           // [kScoreBatch][1600] cutouts
  float* logit;       // [max_triggers]
  void* sws;          // scorer kernels' own workspace (batch kScoreBatch)
  size_t sws_bytes;
};
constexpr int kScoreBatch = 1024;
constexpr int kCutout = 64 * 25;

ScoredWs carve_scored(void* ws, int n_chan, int npix, int n_coarse, int max_triggers, size_t* need) {
  Carver c(ws, ~static_cast<size_t>(0));
  ScoredWs w;
  w.zp = c.take<float>(static_cast<size_t>(n_chan) * npix);
  w.trig = c.take<int32_t>(static_cast<size_t>(std::max(1, max_triggers)) * 3);
  w.x = c.take<float>(static_cast<size_t>(kScoreBatch) * kCutout);
  w.logit = c.take<float>(std::max(1, max_triggers));
  w.sws_bytes = ovro_scorer_workspace_size(kScoreBatch, n_coarse);
  w.sws = c.take<unsigned char>(w.sws_bytes);
  *need = c.used;
  return w;
}

// a8-a12 with the learned scorer (spec addition): the fixed threshold
// trigger_nsigma proposes triggers (NMS included), each trigger's cutout of
// the high-passed cube is scored, and those whose keep probability is at least
// keep_prob are returned with it.
int detect_scored(const float* d_img, int n_chan, int image_size, double cell, int n_coarse, const int32_t* h_nfft,
                  const double* h_freq, const ovro_detect_params& params, const ovro_scorer& sc,
                  ovro_candidate* h_out, int max_out, int* n_out, void* d_ws, size_t ws_bytes, cudaStream_t st) {
  if (!sc.d_w_bf16 || !(sc.trigger_nsigma > 0.0) || sc.max_triggers <= 0 || !sc.d_ws) return OVRO_ERR_INVALID_ARG;
  if (!(sc.keep_prob >= 0.0f && sc.keep_prob <= 1.0f)) return OVRO_ERR_INVALID_ARG;
  ovro_detect_params trig_prm = params;
  trig_prm.mode = OVRO_DETECT_FIXED;
  trig_prm.nsigma = sc.trigger_nsigma;
  DetectCtx* d = nullptr;
  if (int e = detect_ctx_init(&d, n_chan, image_size, cell, n_coarse, h_nfft, &trig_prm, d_ws, ws_bytes)) return e;
  size_t need = 0;
  ScoredWs w = carve_scored(sc.d_ws, n_chan, d->p.npix, n_coarse, sc.max_triggers, &need);
  if (int e = check_workspace(sc.d_ws, sc.ws_bytes, need)) {
    detect_ctx_free(d);
    return e;
  }
  std::vector<ovro_candidate> trig(static_cast<size_t>(sc.max_triggers));
  int n_trig = 0;
  int e = detect_ctx_upload(d, st);
  if (!e) e = detect_ctx_begin(d, st);
  if (!e) {
    const cudaError_t ce = cudaMemsetAsync(w.zp, 0, sizeof(float) * static_cast<size_t>(n_chan) * d->p.npix, st);
    if (ce != cudaSuccess) {
      set_last_error("cudaMemsetAsync", ce);
      e = OVRO_ERR_CUDA;
    }
  }
  for (int c = 0; c < n_coarse && !e; ++c) {
    const float* blk = d_img + static_cast<long long>(d->p.chan0[c]) * d->p.npix;
    e = detect_ctx_coarse_zp(d, c, blk, w.zp, st);
  }
  if (!e) e = detect_ctx_finish(d, h_freq, trig.data(), sc.max_triggers, &n_trig, st);
  detect_ctx_free(d);
  if (e) return e;
  if (n_trig == 0) return OVRO_OK;
  std::vector<int32_t> t3(static_cast<size_t>(n_trig) * 3);
  for (int i = 0; i < n_trig; ++i) {
    t3[3 * i] = trig[i].chan;
    t3[3 * i + 1] = trig[i].row;
    t3[3 * i + 2] = trig[i].col;
  }
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.trig, t3.data(), t3.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  for (int b0 = 0; b0 < n_trig; b0 += kScoreBatch) {
    const int nb = std::min(kScoreBatch, n_trig - b0);
    if (int e2 = ovro_scorer_cutouts(w.zp, n_chan, image_size, n_coarse, h_nfft, w.trig + 3 * b0, nb, w.x, w.sws,
                                     w.sws_bytes, st))
      return e2;
    if (int e2 = ovro_scorer_forward(sc.d_w_bf16, w.x, nb, w.logit + b0, w.sws, w.sws_bytes, st)) return e2;
  }
  std::vector<float> logit(n_trig);
  OVRO_CUDA_TRY(cudaMemcpyAsync(logit.data(), w.logit, n_trig * sizeof(float), cudaMemcpyDeviceToHost, st));
  OVRO_CUDA_TRY(cudaStreamSynchronize(st));
  int n = 0;
  for (int i = 0; i < n_trig; ++i) {
    const double pk = 1.0 / (1.0 + std::exp(-static_cast<double>(logit[i])));
    if (pk < sc.keep_prob) continue;
    if (n < max_out) {
      h_out[n] = trig[i];
      h_out[n].score = static_cast<float>(pk);
    }
    ++n;
  }
  *n_out = n;
  return n > max_out ? OVRO_ERR_CAPACITY : OVRO_OK;
}

}  // namespace ovro

extern "C" {

int ovro_detect(const float* d_img, int n_chan, int image_size, double cell_dircos, int n_coarse,
                const int32_t* h_nfft, const double* h_chan_freq_hz, const ovro_detect_params* params,
                const ovro_scorer* scorer_or_null, ovro_candidate* h_out, int max_out, int* n_out, void* d_ws,
                size_t ws_bytes, void* stream) {
  using namespace ovro;
  if (!d_img || !params || !n_out || (max_out > 0 && !h_out) || max_out < 0 || !h_chan_freq_hz)
    return OVRO_ERR_INVALID_ARG;
  *n_out = 0;
  if (scorer_or_null)
    return detect_scored(d_img, n_chan, image_size, cell_dircos, n_coarse, h_nfft, h_chan_freq_hz, *params,
                         *scorer_or_null, h_out, max_out, n_out, d_ws, ws_bytes, as_stream(stream));
  DetectCtx* d = nullptr;
  if (int e = detect_ctx_init(&d, n_chan, image_size, cell_dircos, n_coarse, h_nfft, params, d_ws, ws_bytes))
    return e;
  cudaStream_t st = as_stream(stream);
  int e = detect_ctx_upload(d, st);
  if (!e) e = detect_ctx_begin(d, st);
  for (int c = 0; c < n_coarse && !e; ++c)
    e = detect_ctx_coarse(d, c, d_img + static_cast<long long>(d->p.chan0[c]) * d->p.npix, st);
  if (!e) e = detect_ctx_finish(d, h_chan_freq_hz, h_out, max_out, n_out, st);
  detect_ctx_free(d);
  return e;
}

size_t ovro_scorer_detect_workspace_size(int n_chan, int image_size, int n_coarse, int max_triggers) {
  if (n_chan <= 0 || image_size <= 0 || n_coarse <= 0 || max_triggers <= 0) return 0;
  size_t need = 0;
  ovro::carve_scored(nullptr, n_chan, image_size * image_size, n_coarse, max_triggers, &need);
  return need;
}

// ---- sharded search (Section 2.4 threshold over several shards)
struct ovro_search {
  ovro::DetectCtx* d = nullptr;
  bool owned = true;             // false: a view of a pipeline's search
};


int ovro_search_create(int n_chan, int image_size, double cell_dircos, int n_coarse, const int32_t* h_nfft,
                       const ovro_detect_params* params, void* d_ws, size_t ws_bytes, void* stream,
                       ovro_search** out) {
  using namespace ovro;
  if (!out) return OVRO_ERR_INVALID_ARG;
  *out = nullptr;
  DetectCtx* d = nullptr;
  if (int e = detect_ctx_init(&d, n_chan, image_size, cell_dircos, n_coarse, h_nfft, params, d_ws, ws_bytes))
    return e;
  cudaStream_t st = as_stream(stream);
  int e = detect_ctx_upload(d, st);
  if (!e) e = detect_ctx_begin(d, st);
  if (e) {
    detect_ctx_free(d);
    return e;
  }
  *out = new ovro_search{d, true};
  return OVRO_OK;
}

int ovro_search_reset(ovro_search* s, void* stream) {
  if (!s) return OVRO_ERR_INVALID_ARG;
  return ovro::detect_ctx_begin(s->d, ovro::as_stream(stream));
}

int ovro_bh_layout(const ovro_detect_params* params, uint32_t* key0, int* n_bins) {
  if (!params || !key0 || !n_bins) return OVRO_ERR_INVALID_ARG;
  ovro::hist_range(*params, key0, n_bins);
  return OVRO_OK;
}

int ovro_search_add(ovro_search* s, int coarse, const float* d_img_block, void* stream) {
  if (!s) return OVRO_ERR_INVALID_ARG;
  return ovro::detect_ctx_coarse(s->d, coarse, d_img_block, ovro::as_stream(stream));
}

int ovro_search_layout(const ovro_search* s, uint32_t* key0, int* n_bins, long long* n_tests) {
  if (!s || !key0 || !n_bins || !n_tests) return OVRO_ERR_INVALID_ARG;
  ovro::detect_ctx_layout(s->d, key0, n_bins, n_tests);
  return OVRO_OK;
}

int ovro_search_histogram(ovro_search* s, unsigned long long* h_hist, int n_bins, void* stream) {
  if (!s || !h_hist) return OVRO_ERR_INVALID_ARG;
  uint32_t k0;
  int nb;
  long long nt;
  ovro::detect_ctx_layout(s->d, &k0, &nb, &nt);
  if (n_bins != nb) return OVRO_ERR_INVALID_ARG;
  std::vector<unsigned long long> h;
  if (int e = ovro::detect_ctx_histogram(s->d, h, ovro::as_stream(stream))) return e;
  std::memcpy(h_hist, h.data(), nb * sizeof(unsigned long long));
  return OVRO_OK;
}

int ovro_search_bin_values(ovro_search* s, int bin, float* h_vals, long long cap, long long* n, void* stream) {
  if (!s || !n || (cap > 0 && !h_vals)) return OVRO_ERR_INVALID_ARG;
  std::vector<float> v;
  if (int e = ovro::detect_ctx_bin_values(s->d, bin, v, ovro::as_stream(stream))) return e;
  *n = static_cast<long long>(v.size());
  if (static_cast<long long>(v.size()) > cap) return OVRO_ERR_CAPACITY;
  if (!v.empty()) std::memcpy(h_vals, v.data(), v.size() * sizeof(float));
  return OVRO_OK;
}

int ovro_search_candidates(ovro_search* s, float cut, const double* h_chan_freq_hz, ovro_candidate* h_out,
                           int max_out, int* n_out, void* stream) {
  if (!s) return OVRO_ERR_INVALID_ARG;
  return ovro::detect_ctx_candidates(s->d, cut, h_chan_freq_hz, h_out, max_out, n_out, ovro::as_stream(stream));
}

void ovro_search_destroy(ovro_search* s) {
  if (!s) return;
  if (s->owned) ovro::detect_ctx_free(s->d);
  delete s;
}

int ovro_bh_bin_verdict(const unsigned long long* h_hist, int n_bins, uint32_t key0, double n_tests, double alpha,
                        int bin, float* lo_edge, unsigned long long* above_next) {
  if (!h_hist || !lo_edge || !above_next || bin < 0 || bin >= n_bins || !(n_tests > 0.0) || !(alpha > 0.0))
    return OVRO_ERR_INVALID_ARG;
  return ovro::bh_bin_verdict(h_hist, n_bins, key0, n_tests, alpha, bin, lo_edge, above_next);
}

int ovro_bh_resolve(const float* h_vals_desc, long long n, unsigned long long above_next, double n_tests,
                    double alpha, float* cut) {
  if ((n > 0 && !h_vals_desc) || n < 0 || !cut || !(n_tests > 0.0) || !(alpha > 0.0)) return OVRO_ERR_INVALID_ARG;
  return ovro::bh_resolve(h_vals_desc, n, above_next, n_tests, alpha, cut);
}

uint32_t ovro_snr_bin_key(float snr) { return ovro::host_f2key(snr) >> ovro::kHistShift; }

}  // extern "C"

ovro_search* ovro::search_view(ovro::DetectCtx* d) { return new ovro_search{d, false}; }
