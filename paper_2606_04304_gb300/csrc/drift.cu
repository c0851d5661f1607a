// Drift-rate search over sub-integration images (the drift search the paper
// leaves as future work, Sections 2.3.4 and 4).
//
// Input: T = 2^k high-passed standardised cubes z'_t [n_chan][N][N], one per
// sub-integration (each from ovro_detect_filter).  For every in-horizon pixel
// and start channel f the search sums z'_t along the Taylor tree's digital
// lines of total drift d (positive and negative, |d| < T), keeps the largest
// SNR = sum / sqrt(T) and its drift, then thresholds and runs Stage I's
// greedy non-maximum suppression with the drifting line's width |d| + 1.
//
//   k_drift      CTA = 32 in-horizon pixels x 32 start channels: stages
//                z'_t over the channels the tile's paths touch (a halo of
//                T - 1 on each side, zero outside the coarse channel) in
//                shared memory with lanes on pixels, then sums every path
//                directly (2T - 1 drifts x T rows per output)
//   k_drift_nms  one warp per (pixel, coarse channel): ballot-gathers the
//                channels at or above the threshold, greedy NMS by warp argmax
//   k_slice      one sub-integration's block of int8 spectra, for the X-engine
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace ovro {
namespace {

constexpr int kMaxSub = 16;          // T <= 16
constexpr int kTileF = 32;           // start channels per tile
constexpr int kDriftWarps = 8;
constexpr int kNmsCapD = 256;        // detections held per (pixel, coarse) pair

struct DriftChunk {
  int c_lo, c_hi, f0, coarse;
};

struct DriftCand {
  int coarse, p, chan, drift;
  float snr, pad;
};

__global__ void k_fill_snr(float* __restrict__ snr, int8_t* __restrict__ dr, long long n) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    snr[i] = -INFINITY;
    dr[i] = 0;
  }
}

// Histogram bins of the SNR for the Benjamini-Hochberg step: the
// order-preserving 32-bit key of the FP32 value shifted right by 16 (the
// binning of ovro_snr_bin_key and ovro_bh_layout).
constexpr int kDriftHistShift = 16;
constexpr int kDriftMaxBins = 2048;

// shift table: st[d * T + t], d, t < T (Taylor paths).  With ghist, every
// voxel's best SNR at or above the floor of bin 0 is counted in its bin
// (values above the top bin in the top bin).
__global__ void __launch_bounds__(32 * kDriftWarps)
k_drift(const float* __restrict__ zp, int T, long long chan_stride, long long sub_stride,
        const int* __restrict__ pix, int n_valid, const DriftChunk* __restrict__ chunks,
        const int* __restrict__ shift_tab, float inv_sqrt_t, float* __restrict__ snr, int8_t* __restrict__ dr,
        uint32_t hist_key0, int n_bins, unsigned long long* __restrict__ ghist) {
  extern __shared__ __align__(16) float tile[];      // [T][W][32]
  __shared__ int st[kMaxSub * kMaxSub];
  __shared__ uint32_t shist[kDriftMaxBins];
  if (ghist)
    for (int i = threadIdx.x; i < n_bins; i += blockDim.x) shist[i] = 0u;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const DriftChunk ck = chunks[blockIdx.y];
  const int p = blockIdx.x * 32 + lane;
  const int W = kTileF + 2 * (T - 1);
  const int base = ck.f0 - (T - 1);                  // channel of tile column 0
  for (int i = threadIdx.x; i < T * T; i += blockDim.x) st[i] = shift_tab[i];
  const long long px = p < n_valid ? pix[p] : 0;
  for (int row = warp; row < T * W; row += kDriftWarps) {
    const int t = row / W, j = row - t * W;
    const int f = base + j;
    float v = 0.0f;
    if (p < n_valid && f >= ck.c_lo && f < ck.c_hi)
      v = __ldg(zp + t * sub_stride + static_cast<long long>(f) * chan_stride + px);
    tile[(t * W + j) * 32 + lane] = v;
  }
  __syncthreads();
  for (int o = warp; o < kTileF && p < n_valid; o += kDriftWarps) {
    const int f = ck.f0 + o;
    if (f >= ck.c_hi) break;
    const int j0 = o + (T - 1);
    float best = -INFINITY;
    int bd = 0;
    for (int d = 0; d < T; ++d) {
      for (int sgn = 1; sgn >= -1; sgn -= 2) {
        if (d == 0 && sgn < 0) continue;
        const int end = f + sgn * d;
        if (end < ck.c_lo || end >= ck.c_hi) continue;
        float s = 0.0f;
        for (int t = 0; t < T; ++t) s += tile[(t * W + j0 + sgn * st[d * T + t]) * 32 + lane];
        s *= inv_sqrt_t;
        if (s > best) {
          best = s;
          bd = sgn * d;
        }
      }
    }
    const long long idx = static_cast<long long>(f) * chan_stride + px;
    snr[idx] = best;
    dr[idx] = static_cast<int8_t>(bd);
    if (ghist) {
      const uint32_t kb = f2key(best) >> kDriftHistShift;
      if (kb >= hist_key0) atomicAdd(&shist[min(kb - hist_key0, static_cast<uint32_t>(n_bins - 1))], 1u);
    }
  }
  if (ghist) {
    __syncthreads();
    for (int i = threadIdx.x; i < n_bins; i += blockDim.x)
      if (shist[i]) atomicAdd(ghist + i, static_cast<unsigned long long>(shist[i]));
  }
}

// Values of histogram bin b of the in-horizon map (the top bin takes every
// larger key), for the exact step-up inside an open bin.
__global__ void k_drift_gather(const float* __restrict__ snr, long long chan_stride, const int* __restrict__ pix,
                               int n_valid, int n_chan, uint32_t kb, int top, float* __restrict__ out, int cap,
                               int* __restrict__ count) {
  const long long n = static_cast<long long>(n_valid) * n_chan;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long f = i / n_valid, p = i - f * n_valid;
    const float v = snr[f * chan_stride + pix[p]];
    const uint32_t k = f2key(v) >> kDriftHistShift;
    if (k == kb || (top && k > kb)) {
      const int slot = atomicAdd(count, 1);
      if (slot < cap) out[slot] = v;
    }
  }
}

// One warp per (pixel, coarse) pair q = p * n_coarse + c.
__global__ void __launch_bounds__(32 * kDriftWarps)
k_drift_nms(const float* __restrict__ snr, const int8_t* __restrict__ dr, long long chan_stride,
            const int* __restrict__ pix, int n_valid, const int* __restrict__ c_lo, const int* __restrict__ c_hi,
            int n_coarse, float cut, DriftCand* __restrict__ out, int out_cap, int* __restrict__ counters) {
  __shared__ int lf[kDriftWarps][kNmsCapD];
  __shared__ float lv[kDriftWarps][kNmsCapD];
  __shared__ uint8_t ls[kDriftWarps][kNmsCapD];     // 0 undecided, 1 accepted, 2 suppressed
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long q = static_cast<long long>(blockIdx.x) * kDriftWarps + warp;
  if (q >= static_cast<long long>(n_valid) * n_coarse) return;
  const int p = static_cast<int>(q / n_coarse), c = static_cast<int>(q % n_coarse);
  const long long px = pix[p];
  int n = 0;
  bool over = false;
  for (int f0 = c_lo[c]; f0 < c_hi[c]; f0 += 32) {
    const int f = f0 + lane;
    const float v = f < c_hi[c] ? snr[static_cast<long long>(f) * chan_stride + px] : -INFINITY;
    const bool hit = v >= cut;
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    const int pos = n + __popc(m & ((1u << lane) - 1u));
    if (hit && pos < kNmsCapD) {
      lf[warp][pos] = f;
      lv[warp][pos] = v;
      ls[warp][pos] = 0;
    }
    n += __popc(m);
  }
  if (n > kNmsCapD) {
    over = true;
    n = kNmsCapD;
  }
  if (over) {
    if (lane == 0) atomicAdd(counters + 1, 1);
    return;
  }
  __syncwarp();
  for (int iter = 0; iter < n; ++iter) {
    // argmax over undecided: larger SNR, then lower channel
    float bv = -INFINITY;
    int bi = -1;
    for (int i = lane; i < n; i += 32) {
      if (ls[warp][i] != 0) continue;
      const float v = lv[warp][i];
      if (bi < 0 || v > bv || (v == bv && lf[warp][i] < lf[warp][bi])) {
        bv = v;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      const bool take = oi >= 0 && (bi < 0 || ov > bv || (ov == bv && lf[warp][oi] < lf[warp][bi]));
      if (take) {
        bv = ov;
        bi = oi;
      }
    }
    if (bi < 0) break;
    const int fa = lf[warp][bi];
    const int da = dr[static_cast<long long>(fa) * chan_stride + px];
    const int half = max(1, (abs(da) + 1) / 2);
    __syncwarp();
    for (int i = lane; i < n; i += 32)
      if (ls[warp][i] == 0) ls[warp][i] = (i == bi) ? 1 : (abs(lf[warp][i] - fa) <= half ? 2 : 0);
    __syncwarp();
    if (lane == 0) {
      const int slot = atomicAdd(counters, 1);
      if (slot < out_cap) out[slot] = DriftCand{c, p, fa, da, bv, 0.0f};
    }
  }
}

__global__ void k_widen(const int8_t* __restrict__ a, long long n, int32_t* __restrict__ b) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    b[i] = a[i];
}

__global__ void k_slice(const int8_t* __restrict__ q, long long n_chan, long long n_spec, long long row_bytes,
                        int s0, int count, int8_t* __restrict__ out, bool vec) {
  // out[c][s][:] = q[c][s0 + s][:], row_bytes per spectrum; vec: 16-byte rows and pointers
  const long long rows = n_chan * count;
  const long long per_row = vec ? row_bytes / 16 : row_bytes;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < rows * per_row;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long r = i / per_row, e = i - r * per_row;
    const long long c = r / count, s = r - c * count;
    const long long src = (c * n_spec + s0 + s) * row_bytes, dst = r * row_bytes;
    if (vec)
      reinterpret_cast<uint4*>(out + dst)[e] = __ldg(reinterpret_cast<const uint4*>(q + src) + e);
    else
      out[dst + e] = q[src + e];
  }
}

int taylor_shift(int d, int n, int t) {
  if (n == 1) return 0;
  const int h = n / 2;
  if (t < h) return taylor_shift(d / 2, h, t);
  return (d - d / 2) + taylor_shift(d / 2, h, t - h);
}

// log10 of the one-sided Gaussian tail Q(x), FP64 (erfc below 30, the
// asymptotic series above, where erfc underflows toward denormals).
double log10_q(double x) {
  if (x < 30.0) return std::log10(0.5 * std::erfc(x / std::sqrt(2.0)));
  const double x2 = x * x;
  const double ln = -0.5 * x2 - std::log(x * std::sqrt(2.0 * M_PI)) + std::log1p(-1.0 / x2 + 3.0 / (x2 * x2));
  return ln / std::log(10.0);
}

constexpr int kDriftGatherCap = 1 << 22;

struct DriftWs {
  unsigned long long* hist;
  float* vals;
  int* pix;
  int* shift;
  DriftChunk* chunks;
  int* c_lo;
  int* c_hi;
  float* snr;
  int8_t* dr;
  DriftCand* cands;
  int* counters;
};

constexpr int kDriftCandCap = 1 << 20;

DriftWs carve_drift(void* ws, size_t bytes, int n_chan, int image_size, int n_coarse, long long n_chunks,
                    size_t* need) {
  Carver c(ws, bytes);
  const long long npix = static_cast<long long>(image_size) * image_size;
  DriftWs w;
  w.hist = c.take<unsigned long long>(kDriftMaxBins);
  w.vals = c.take<float>(kDriftGatherCap);
  w.pix = c.take<int>(npix);
  w.shift = c.take<int>(kMaxSub * kMaxSub);
  w.chunks = c.take<DriftChunk>(std::max<long long>(n_chunks, 1));
  w.c_lo = c.take<int>(n_coarse);
  w.c_hi = c.take<int>(n_coarse);
  w.snr = c.take<float>(static_cast<size_t>(n_chan) * npix);
  w.dr = c.take<int8_t>(static_cast<size_t>(n_chan) * npix);
  w.cands = c.take<DriftCand>(kDriftCandCap);
  w.counters = c.take<int>(4);
  *need = c.used;
  return w;
}

long long n_chunks_of(int n_coarse, const int32_t* nfft) {
  long long n = 0;
  for (int c = 0; c < n_coarse; ++c) n += (nfft[c] + kTileF - 1) / kTileF;
  return n;
}

}  // namespace
}  // namespace ovro

extern "C" {

size_t ovro_drift_workspace_size(int n_chan, int image_size, int n_coarse, const int32_t* h_nfft) {
  if (n_chan <= 0 || image_size <= 0 || n_coarse <= 0 || !h_nfft) return 0;
  size_t need = 0;
  ovro::carve_drift(nullptr, 0, n_chan, image_size, n_coarse, ovro::n_chunks_of(n_coarse, h_nfft), &need);
  return need;
}

int ovro_drift_search(const float* d_zp, int n_sub, int n_chan, int image_size, double cell_dircos, int n_coarse,
                      const int32_t* h_nfft, const double* h_chan_freq_hz, const ovro_detect_params* params,
                      float* d_snr_or_null, int32_t* d_drift_or_null, ovro_candidate* h_out, int32_t* h_drift_out,
                      int max_out, int* n_out, void* d_ws, size_t ws_bytes, void* stream) {
  using namespace ovro;
  if (!d_zp || !h_nfft || !h_chan_freq_hz || !n_out || !params || n_chan <= 0 || image_size <= 0 ||
      n_coarse <= 0 || !(cell_dircos > 0.0) || max_out < 0 || (max_out > 0 && (!h_out || !h_drift_out)))
    return OVRO_ERR_INVALID_ARG;
  const bool bh = params->mode == OVRO_DETECT_BH;
  if (!bh && params->mode != OVRO_DETECT_FIXED) return OVRO_ERR_INVALID_ARG;
  uint32_t key0 = 0;
  int nb = 0;
  if (bh) {
    if (int e = ovro_bh_layout(params, &key0, &nb)) return e;
    if (nb > kDriftMaxBins) return OVRO_ERR_UNSUPPORTED;
  }
  if (n_sub < 2 || n_sub > kMaxSub || (n_sub & (n_sub - 1))) return OVRO_ERR_UNSUPPORTED;
  *n_out = 0;
  std::vector<int> lo(n_coarse), hi(n_coarse);
  int c0 = 0;
  for (int c = 0; c < n_coarse; ++c) {
    if (h_nfft[c] <= 0) return OVRO_ERR_INVALID_ARG;
    lo[c] = c0;
    c0 += h_nfft[c];
    hi[c] = c0;
  }
  if (c0 != n_chan) return OVRO_ERR_INVALID_ARG;
  const int n = image_size;
  std::vector<int> pix;
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      const double l = static_cast<double>(c - n / 2) * cell_dircos;
      const double m = static_cast<double>(r - n / 2) * cell_dircos;
      if (l * l + m * m < 1.0) pix.push_back(r * n + c);
    }
  const int n_valid = static_cast<int>(pix.size());
  std::vector<DriftChunk> chunks;
  for (int c = 0; c < n_coarse; ++c)
    for (int f0 = lo[c]; f0 < hi[c]; f0 += kTileF) chunks.push_back(DriftChunk{lo[c], hi[c], f0, c});
  std::vector<int> tab(kMaxSub * kMaxSub, 0);
  for (int d = 0; d < n_sub; ++d)
    for (int t = 0; t < n_sub; ++t) tab[d * n_sub + t] = taylor_shift(d, n_sub, t);
  size_t need = 0;
  DriftWs w = carve_drift(d_ws, ws_bytes, n_chan, n, n_coarse, static_cast<long long>(chunks.size()), &need);
  if (int e = check_workspace(d_ws, ws_bytes, need)) return e;
  if (chunks.size() > 65535) return OVRO_ERR_UNSUPPORTED;
  cudaStream_t st = as_stream(stream);
  const long long npix = static_cast<long long>(n) * n;
  const long long nvox = npix * n_chan;
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.pix, pix.data(), pix.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.shift, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.chunks, chunks.data(), chunks.size() * sizeof(DriftChunk),
                                cudaMemcpyHostToDevice, st));
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.c_lo, lo.data(), lo.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  OVRO_CUDA_TRY(cudaMemcpyAsync(w.c_hi, hi.data(), hi.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  OVRO_CUDA_TRY(cudaMemsetAsync(w.counters, 0, 4 * sizeof(int), st));
  if (bh) OVRO_CUDA_TRY(cudaMemsetAsync(w.hist, 0, kDriftMaxBins * sizeof(unsigned long long), st));
  k_fill_snr<<<4 * num_sms(), 256, 0, st>>>(w.snr, w.dr, nvox);
  OVRO_LAUNCH_CHECK();
  if (n_valid > 0) {
    const size_t sm = static_cast<size_t>(n_sub) * (kTileF + 2 * (n_sub - 1)) * 32 * sizeof(float);
    OVRO_CUDA_TRY(cudaFuncSetAttribute(k_drift, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm)));
    dim3 grid((n_valid + 31) / 32, static_cast<unsigned>(chunks.size()));
    {
      OVRO_PROF("k_drift", st);
      k_drift<<<grid, 32 * kDriftWarps, sm, st>>>(d_zp, n_sub, npix, nvox, w.pix, n_valid, w.chunks, w.shift,
                                                   static_cast<float>(1.0 / std::sqrt(static_cast<double>(n_sub))),
                                                   w.snr, w.dr, key0, nb, bh ? w.hist : nullptr);
      OVRO_LAUNCH_CHECK();
    }
    // the cut: the fixed threshold, or Benjamini-Hochberg over every
    // in-horizon (pixel, channel), decided bin by bin as in Stage I
    float cut = static_cast<float>(params->nsigma);
    if (bh) {
      std::vector<unsigned long long> hist(nb);
      OVRO_CUDA_TRY(cudaMemcpyAsync(hist.data(), w.hist, nb * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                    st));
      OVRO_CUDA_TRY(cudaStreamSynchronize(st));
      const double m = static_cast<double>(n_valid) * n_chan;
      bool found = false;
      for (int b = 0; b < nb && !found; ++b) {
        float lo = 0.f;
        unsigned long long above = 0;
        const int v = ovro_bh_bin_verdict(hist.data(), nb, key0, m, params->alpha, b, &lo, &above);
        if (v == 0 || v == 3) continue;
        if (v == 1) {
          cut = lo;
          found = true;
          break;
        }
        if (hist[b] > static_cast<unsigned long long>(kDriftGatherCap)) return OVRO_ERR_CAPACITY;
        OVRO_CUDA_TRY(cudaMemsetAsync(w.counters + 2, 0, sizeof(int), st));
        k_drift_gather<<<4 * num_sms(), 256, 0, st>>>(w.snr, npix, w.pix, n_valid, n_chan, key0 + b, b == nb - 1,
                                                     w.vals, kDriftGatherCap, w.counters + 2);
        OVRO_LAUNCH_CHECK();
        int nv = 0;
        OVRO_CUDA_TRY(cudaMemcpyAsync(&nv, w.counters + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
        OVRO_CUDA_TRY(cudaStreamSynchronize(st));
        if (static_cast<unsigned long long>(nv) != hist[b]) return OVRO_ERR_CAPACITY;
        std::vector<float> vals(nv);
        OVRO_CUDA_TRY(cudaMemcpyAsync(vals.data(), w.vals, nv * sizeof(float), cudaMemcpyDeviceToHost, st));
        OVRO_CUDA_TRY(cudaStreamSynchronize(st));
        std::sort(vals.begin(), vals.end(), std::greater<float>());
        if (ovro_bh_resolve(vals.data(), nv, above, m, params->alpha, &cut)) found = true;
      }
      if (!found) cut = INFINITY;                     // nothing is rejected
      OVRO_CUDA_TRY(cudaMemsetAsync(w.counters + 2, 0, sizeof(int), st));
    }
    const long long pairs = static_cast<long long>(n_valid) * n_coarse;
    const long long blocks = (pairs + kDriftWarps - 1) / kDriftWarps;
    if (blocks > 0x7fffffffLL) return OVRO_ERR_UNSUPPORTED;
    k_drift_nms<<<static_cast<unsigned>(blocks), 32 * kDriftWarps, 0, st>>>(
        w.snr, w.dr, npix, w.pix, n_valid, w.c_lo, w.c_hi, n_coarse, cut, w.cands, kDriftCandCap, w.counters);
    OVRO_LAUNCH_CHECK();
  }
  // optional maps for the caller
  if (d_snr_or_null)
    OVRO_CUDA_TRY(cudaMemcpyAsync(d_snr_or_null, w.snr, nvox * sizeof(float), cudaMemcpyDeviceToDevice, st));
  if (d_drift_or_null) {
    k_widen<<<4 * num_sms(), 256, 0, st>>>(w.dr, nvox, d_drift_or_null);
    OVRO_LAUNCH_CHECK();
  }
  int cnt[2] = {0, 0};
  OVRO_CUDA_TRY(cudaMemcpyAsync(cnt, w.counters, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  OVRO_CUDA_TRY(cudaStreamSynchronize(st));
  if (cnt[1] > 0) {
    snprintf_last_error("ovro_drift_search: %d (pixel, coarse) pairs hold more than %d detections", cnt[1],
                        kNmsCapD);
    return OVRO_ERR_CAPACITY;
  }
  const int total = std::min(cnt[0], kDriftCandCap);
  std::vector<DriftCand> rec(total);
  if (total > 0) {
    OVRO_CUDA_TRY(cudaMemcpyAsync(rec.data(), w.cands, total * sizeof(DriftCand), cudaMemcpyDeviceToHost, st));
    OVRO_CUDA_TRY(cudaStreamSynchronize(st));
  }
  // presentation order: pixel, coarse channel, channel
  std::sort(rec.begin(), rec.end(), [](const DriftCand& a, const DriftCand& b) {
    if (a.p != b.p) return a.p < b.p;
    if (a.coarse != b.coarse) return a.coarse < b.coarse;
    return a.chan < b.chan;
  });
  *n_out = cnt[0];
  const int nw = std::min(total, max_out);
  for (int i = 0; i < nw; ++i) {
    const DriftCand& d = rec[i];
    ovro_candidate& o = h_out[i];
    o.coarse = d.coarse;
    o.fine = d.chan - lo[d.coarse];
    o.chan = d.chan;
    o.row = pix[d.p] / n;
    o.col = pix[d.p] % n;
    o.width = std::abs(d.drift) + 1;
    o.snr = d.snr;
    o.score = 0.0f;
    o.freq_hz = h_chan_freq_hz[d.chan];
    o.log10_p = log10_q(static_cast<double>(d.snr));
    h_drift_out[i] = d.drift;
  }
  if (cnt[0] > max_out || cnt[0] > kDriftCandCap) return OVRO_ERR_CAPACITY;
  return OVRO_OK;
}

int ovro_spectra_slice(const int8_t* d_q, int n_chan, int n_spec, int n_input, int s0, int count, int8_t* d_out,
                       void* stream) {
  using namespace ovro;
  if (!d_q || !d_out || n_chan <= 0 || n_spec <= 0 || n_input <= 0 || s0 < 0 || count <= 0 ||
      static_cast<long long>(s0) + count > n_spec)
    return OVRO_ERR_INVALID_ARG;
  cudaStream_t st = as_stream(stream);
  const long long row = static_cast<long long>(n_input) * 2;
  const bool vec = row % 16 == 0 && reinterpret_cast<uintptr_t>(d_q) % 16 == 0 &&
                   reinterpret_cast<uintptr_t>(d_out) % 16 == 0;
  k_slice<<<4 * num_sms(), 256, 0, st>>>(d_q, n_chan, n_spec, row, s0, count, d_out, vec);
  OVRO_LAUNCH_CHECK();
  return OVRO_OK;
}

}  // extern "C"
