// Stage I re-evaluation and the automated Stage II cuts (Section 2.4).
//
// After the non-maximum suppression each candidate is re-evaluated in a local
// spectral window: a small-scale baseline and noise level are re-estimated
// from off-line channels at its pixel and the SNR is recomputed.  Stage II
// then keeps compact narrowband sources: the candidate's line image is fitted
// with an elliptical Gaussian (centroid errors from the covariance rescaled
// by sqrt(chi2_red)), compared with the synthesized beam's fit, and
// candidates in images whose noise departs from expectation are flagged.
//
//   k_vet_psf    beam cutouts around the point-spread image's centre
//   k_vet_line   one CTA per candidate: off-line medians per pixel (a warp per
//                pixel, exact order statistics by rank counting), the line
//                image over the cutout and the re-evaluated SNR
//   k_vet_fit    one warp per fit: Levenberg-Marquardt in FP64 on <= 225
//                pixels, 6 parameters, then the covariance at the minimum
//   k_vet_noise  one CTA per candidate channel: mean and spread of the
//                standardised in-horizon pixels in FP64
// This is per-candidate work (a few thousand at most), launched after the
// search; FP64 keeps it within rounding of the definitions.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace ovro {
namespace {

constexpr double kMadToSigma = 1.482602218505602;
constexpr int kMaxOffHalf = 64;
constexpr int kMaxOff = 2 * kMaxOffHalf;
constexpr int kMaxFitHalf = 7;
constexpr int kMaxPix = (2 * kMaxFitHalf + 1) * (2 * kMaxFitHalf + 1);
constexpr int kMinOffline = 16;
constexpr int kLineWarps = 8;
constexpr int kFitOut = 12;          // p[6], sigma_x, sigma_y, chi2_red, n, chol ok, iterations
constexpr int kMaxLmIter = 400;

struct VetCand {
  int chan, w, row, col, c_lo, c_hi, coarse, pad;
};

__device__ __forceinline__ bool in_horizon(int r, int c, int n, double cell) {
  const double l = __dmul_rn(static_cast<double>(c - n / 2), cell);
  const double m = __dmul_rn(static_cast<double>(r - n / 2), cell);
  return __dadd_rn(__dmul_rn(l, l), __dmul_rn(m, m)) < 1.0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Median of v[0..n) (mean of the two middle order statistics for even n;
// 0 for n = 0).  Ranks by counting, ties broken by index, so each rank is
// held by exactly one element and a warp sum collects it.
__device__ double warp_median(const double* v, int n, int lane) {
  double lo = 0.0, hi = 0.0;
  for (int i = lane; i < n; i += 32) {
    const double x = v[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double y = v[j];
      rank += (y < x) || (y == x && j < i);
    }
    if (rank == (n - 1) / 2) lo = x;
    if (rank == n / 2) hi = x;
  }
  lo = warp_sum(lo);
  hi = warp_sum(hi);
  return n ? (lo + hi) * 0.5 : 0.0;
}

// z of channel f at pixel idx: (x - median) / (1.4826 MAD), 0 if MAD = 0.
__device__ __forceinline__ double zval(const float* __restrict__ img, const double* __restrict__ stats, long long npix,
                                       int f, long long idx) {
  const double med = stats[2 * f], mad = stats[2 * f + 1];
  if (!(mad > 0.0)) return 0.0;
  const double x = static_cast<double>(img[static_cast<long long>(f) * npix + idx]);
  return (x - med) / (kMadToSigma * mad);
}

__global__ void k_vet_psf(const float* __restrict__ psf, int n, int n_coarse, int h, double* __restrict__ L,
                          uint8_t* __restrict__ valid, double* __restrict__ p0, int* __restrict__ centre) {
  const int c = blockIdx.x;
  if (c >= n_coarse) return;
  const int side = 2 * h + 1;
  const int c0 = n / 2;
  const float* im = psf + static_cast<long long>(c) * n * n;
  for (int i = threadIdx.x; i < side * side; i += blockDim.x) {
    const int r = c0 + i / side - h, cc = c0 + i % side - h;
    const bool in = r >= 0 && r < n && cc >= 0 && cc < n;
    L[static_cast<long long>(c) * kMaxPix + i] = in ? static_cast<double>(im[r * n + cc]) : 0.0;
    valid[static_cast<long long>(c) * kMaxPix + i] = in;
  }
  if (threadIdx.x == 0) {
    double* p = p0 + 6 * c;
    p[0] = static_cast<double>(im[c0 * n + c0]);
    p[1] = c0;
    p[2] = c0;
    p[3] = 1.0;
    p[4] = 0.0;
    p[5] = 1.0;
    centre[2 * c] = c0;
    centre[2 * c + 1] = c0;
  }
}

// beam: [n_coarse][kFitOut] fit results of the beams; the candidate fit
// starts from the beam's quadratic form.
__global__ void __launch_bounds__(32 * kLineWarps)
k_vet_line(const float* __restrict__ img, const double* __restrict__ stats, int n, double cell,
           const VetCand* __restrict__ cands, int h, int m_half, const double* __restrict__ beam,
           double* __restrict__ L, uint8_t* __restrict__ valid, double* __restrict__ p0, int* __restrict__ centre,
           double* __restrict__ snr_re) {
  __shared__ int off[kMaxOff];
  __shared__ int s_n_off;
  __shared__ double vals[kLineWarps][kMaxOff];
  const VetCand cd = cands[blockIdx.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lo = cd.chan - (cd.w - 1) / 2, hi = cd.chan + (cd.w - 1) - (cd.w - 1) / 2;
  const int g = max(1, cd.w / 2);
  const int l0 = max(cd.c_lo, lo - g - m_half), l1 = max(cd.c_lo, lo - g);
  const int r0 = min(cd.c_hi, hi + g + 1), r1 = min(cd.c_hi, hi + g + m_half + 1);
  const int nl = max(0, l1 - l0), nr = max(0, r1 - r0);
  for (int i = threadIdx.x; i < nl + nr; i += blockDim.x) off[i] = i < nl ? l0 + i : r0 + (i - nl);
  const double* bm = beam + static_cast<long long>(cd.coarse) * kFitOut;
  if (threadIdx.x == 0) {
    s_n_off = nl + nr;
    // defaults, overwritten below when the candidate's own pixel is valid
    snr_re[blockIdx.x] = NAN;
    double* p = p0 + 6 * blockIdx.x;
    p[0] = 0.0;
    p[1] = cd.col;
    p[2] = cd.row;
    p[3] = bm[3];
    p[4] = bm[4];
    p[5] = bm[5];
    centre[2 * blockIdx.x] = cd.col;
    centre[2 * blockIdx.x + 1] = cd.row;
  }
  __syncthreads();
  const int n_off = s_n_off;
  const long long npix = static_cast<long long>(n) * n;
  const int side = 2 * h + 1;
  const double rw = sqrt(static_cast<double>(cd.w));
  double* Lc = L + static_cast<long long>(blockIdx.x) * kMaxPix;
  uint8_t* vc = valid + static_cast<long long>(blockIdx.x) * kMaxPix;
  for (int pix = warp; pix < side * side; pix += kLineWarps) {
    const int dr = pix / side - h, dc = pix % side - h;
    const int r = cd.row + dr, c = cd.col + dc;
    const bool ok = r >= 0 && r < n && c >= 0 && c < n && in_horizon(r, c, n, cell);
    if (!ok) {
      if (lane == 0) {
        Lc[pix] = 0.0;
        vc[pix] = 0;
      }
      continue;
    }
    const long long idx = static_cast<long long>(r) * n + c;
    double* v = vals[warp];
    for (int i = lane; i < n_off; i += 32) v[i] = zval(img, stats, npix, off[i], idx);
    __syncwarp();
    const double b = warp_median(v, n_off, lane);
    double s = 0.0;
    for (int f = lo + lane; f <= hi; f += 32) s += zval(img, stats, npix, f, idx) - b;
    s = warp_sum(s);
    if (lane == 0) {
      Lc[pix] = s / rw;
      vc[pix] = 1;
    }
    if (dr == 0 && dc == 0) {
      __syncwarp();
      for (int i = lane; i < n_off; i += 32) v[i] = fabs(v[i] - b);
      __syncwarp();
      double sig = kMadToSigma * warp_median(v, n_off, lane);
      if (n_off < kMinOffline || !(sig > 0.0)) sig = 1.0;
      if (lane == 0) {
        snr_re[blockIdx.x] = s / (sig * rw);
        p0[6 * blockIdx.x] = s / rw;
      }
    }
    __syncwarp();
  }
}

// Model A exp(-(a dx^2 + 2 b dx dy + c dy^2) / 2) and its gradient.
__device__ __forceinline__ double gauss_row(const double* p, double x, double y, double* jr) {
  const double dx = x - p[1], dy = y - p[2];
  const double e = exp(-0.5 * (p[3] * dx * dx + 2.0 * p[4] * dx * dy + p[5] * dy * dy));
  const double f = p[0] * e;
  if (jr) {
    jr[0] = e;
    jr[1] = f * (p[3] * dx + p[4] * dy);
    jr[2] = f * (p[4] * dx + p[5] * dy);
    jr[3] = -0.5 * f * dx * dx;
    jr[4] = -f * dx * dy;
    jr[5] = -0.5 * f * dy * dy;
  }
  return f;
}

// Cholesky solve of the 6 x 6 system A x = rhs (A symmetric, full storage).
// Returns false if A is not numerically positive definite.
__device__ bool chol_solve6(const double* A, const double* rhs, double* x) {
  double Lm[6][6];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) Lm[i][j] = 0.0;
  for (int j = 0; j < 6; ++j) {
    double d = A[j * 6 + j];
    for (int k = 0; k < j; ++k) d -= Lm[j][k] * Lm[j][k];
    if (!(d > 0.0) || !isfinite(d)) return false;
    const double ljj = sqrt(d);
    Lm[j][j] = ljj;
    for (int i = j + 1; i < 6; ++i) {
      double s = A[i * 6 + j];
      for (int k = 0; k < j; ++k) s -= Lm[i][k] * Lm[j][k];
      Lm[i][j] = s / ljj;
    }
  }
  double y[6];
  for (int i = 0; i < 6; ++i) {
    double s = rhs[i];
    for (int k = 0; k < i; ++k) s -= Lm[i][k] * y[k];
    y[i] = s / Lm[i][i];
  }
  for (int i = 5; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < 6; ++k) s -= Lm[k][i] * x[k];
    x[i] = s / Lm[i][i];
  }
  return true;
}

// Sums over the valid pixels of this warp's fit: rss, and (if jt) J^T J (full
// 6 x 6) and J^T r.
__device__ double fit_sums(const double* __restrict__ Lf, const uint8_t* __restrict__ vf, int side, int h, int cx,
                           int cy, const double* p, double* jtj, double* jtr, int lane) {
  double rss = 0.0;
  double a[21], g[6];
  if (jtj) {
#pragma unroll
    for (int i = 0; i < 21; ++i) a[i] = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = 0.0;
  }
  for (int i = lane; i < side * side; i += 32) {
    if (!vf[i]) continue;
    const double x = cx + (i % side - h), y = cy + (i / side - h);
    double jr[6];
    const double r = gauss_row(p, x, y, jtj ? jr : nullptr) - Lf[i];
    rss += r * r;
    if (jtj) {
      int t = 0;
#pragma unroll
      for (int u = 0; u < 6; ++u) {
        g[u] += jr[u] * r;
#pragma unroll
        for (int v = 0; v <= u; ++v) a[t++] += jr[u] * jr[v];
      }
    }
  }
  rss = warp_sum(rss);
  if (jtj) {
    int t = 0;
    for (int u = 0; u < 6; ++u) {
      jtr[u] = warp_sum(g[u]);
      for (int v = 0; v <= u; ++v) {
        const double s = warp_sum(a[t++]);
        jtj[u * 6 + v] = s;
        jtj[v * 6 + u] = s;
      }
    }
  }
  return rss;
}

// One warp per fit.  Marquardt's damping (diagonal scaling), at most
// kMaxLmIter accepted or rejected steps; every lane runs the same small
// solves, so all hold the same parameters.
__global__ void k_vet_fit(const double* __restrict__ L, const uint8_t* __restrict__ valid, const double* __restrict__ p0,
                          const int* __restrict__ centre, int n_fit, int h, double* __restrict__ out) {
  const int fit = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (fit >= n_fit) return;
  const int side = 2 * h + 1;
  const double* Lf = L + static_cast<long long>(fit) * kMaxPix;
  const uint8_t* vf = valid + static_cast<long long>(fit) * kMaxPix;
  const int cx = centre[2 * fit], cy = centre[2 * fit + 1];
  int nv = 0;
  for (int i = lane; i < side * side; i += 32) nv += vf[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nv += __shfl_xor_sync(0xffffffffu, nv, o);
  double p[6];
  for (int i = 0; i < 6; ++i) p[i] = p0[6 * fit + i];
  double jtj[36], jtr[6];
  double rss = fit_sums(Lf, vf, side, h, cx, cy, p, jtj, jtr, lane);
  double lambda = 1e-3;
  int it = 0;
  bool chol = true;
  if (nv >= 7 && isfinite(rss)) {
    while (it < kMaxLmIter) {
      ++it;
      double A[36], step[6], neg[6];
      for (int i = 0; i < 36; ++i) A[i] = jtj[i];
      for (int i = 0; i < 6; ++i) {
        A[i * 6 + i] += lambda * jtj[i * 6 + i];
        neg[i] = -jtr[i];
      }
      if (!chol_solve6(A, neg, step)) {
        lambda *= 10.0;
        if (lambda > 1e30) break;
        continue;
      }
      double pn[6];
      for (int i = 0; i < 6; ++i) pn[i] = p[i] + step[i];
      const double rn = fit_sums(Lf, vf, side, h, cx, cy, pn, nullptr, nullptr, lane);
      if (isfinite(rn) && rn < rss) {
        const double drop = rss - rn;
        for (int i = 0; i < 6; ++i) p[i] = pn[i];
        rss = fit_sums(Lf, vf, side, h, cx, cy, p, jtj, jtr, lane);
        lambda = fmax(lambda * 0.1, 1e-15);
        double sn = 0.0, pnorm = 0.0;
        for (int i = 0; i < 6; ++i) {
          sn += step[i] * step[i];
          pnorm += p[i] * p[i];
        }
        if (drop <= 1e-15 * rss && sn <= 1e-24 * (pnorm + 1e-30)) break;
      } else {
        lambda *= 10.0;
        if (lambda > 1e30) break;     // no descent left: at the minimum to rounding
      }
    }
  }
  // covariance (J^T J)^-1 chi2_red at the minimum
  double chi2 = nv > 6 ? rss / (nv - 6) : NAN;
  double sx = NAN, sy = NAN;
  if (nv >= 7) {
    double e1[6] = {0, 1, 0, 0, 0, 0}, e2[6] = {0, 0, 1, 0, 0, 0}, c1[6], c2[6];
    chol = chol_solve6(jtj, e1, c1) && chol_solve6(jtj, e2, c2);
    if (chol) {
      sx = sqrt(c1[1] * chi2);
      sy = sqrt(c2[2] * chi2);
    }
  } else {
    chol = false;
  }
  if (lane == 0) {
    double* o = out + static_cast<long long>(fit) * kFitOut;
    for (int i = 0; i < 6; ++i) o[i] = p[i];
    o[6] = sx;
    o[7] = sy;
    o[8] = chi2;
    o[9] = nv;
    o[10] = chol ? 1.0 : 0.0;
    o[11] = it;
  }
}

// out[c] = (robust sigma s, std of the standardised in-horizon pixels) of channel chans[c].
__global__ void __launch_bounds__(256) k_vet_noise(const float* __restrict__ img, const double* __restrict__ stats,
                                                   int n, double cell, const int* __restrict__ chans,
                                                   double* __restrict__ out) {
  __shared__ double part[2][256];
  const int f = chans[blockIdx.x];
  const double med = stats[2 * f], mad = stats[2 * f + 1];
  const double s = kMadToSigma * mad;
  const long long npix = static_cast<long long>(n) * n;
  const float* im = img + static_cast<long long>(f) * npix;
  double s1 = 0.0, s2 = 0.0, cnt = 0.0;
  if (s > 0.0) {
    for (long long i = threadIdx.x; i < npix; i += blockDim.x) {
      const int r = static_cast<int>(i / n), c = static_cast<int>(i % n);
      if (!in_horizon(r, c, n, cell)) continue;
      const double z = (static_cast<double>(im[i]) - med) / s;
      s1 += z;
      s2 += z * z;
      cnt += 1.0;
    }
  }
  __shared__ double pc[256];
  part[0][threadIdx.x] = s1;
  part[1][threadIdx.x] = s2;
  pc[threadIdx.x] = cnt;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      part[0][threadIdx.x] += part[0][threadIdx.x + w];
      part[1][threadIdx.x] += part[1][threadIdx.x + w];
      pc[threadIdx.x] += pc[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double sd = 0.0;
    if (s > 0.0 && pc[0] > 0.0) {
      const double mean = part[0][0] / pc[0];
      sd = sqrt(fmax(part[1][0] / pc[0] - mean * mean, 0.0));
    }
    out[2 * blockIdx.x] = s > 0.0 ? s : 0.0;
    out[2 * blockIdx.x + 1] = sd;
  }
}

struct VetWs {
  VetCand* cand;
  double* L;
  uint8_t* valid;
  double* p0;
  int* centre;
  double* fit;
  double* snr;
  int* chans;
  double* noise;
};

VetWs carve_vet(void* ws, size_t bytes, int n_cand, int n_coarse, size_t* need) {
  Carver c(ws, bytes);
  const size_t nf = static_cast<size_t>(n_cand) + n_coarse;
  VetWs w;
  w.cand = c.take<VetCand>(std::max(n_cand, 1));
  w.L = c.take<double>(nf * kMaxPix);
  w.valid = c.take<uint8_t>(nf * kMaxPix);
  w.p0 = c.take<double>(nf * 6);
  w.centre = c.take<int>(nf * 2);
  w.fit = c.take<double>(nf * kFitOut);
  w.snr = c.take<double>(std::max(n_cand, 1));
  w.chans = c.take<int>(std::max(n_cand, 1));
  w.noise = c.take<double>(2 * static_cast<size_t>(std::max(n_cand, 1)));
  *need = c.used;
  return w;
}

}  // namespace
}  // namespace ovro

extern "C" {

size_t ovro_vet_workspace_size(int n_cand, int n_coarse) {
  if (n_cand < 0 || n_coarse <= 0) return 0;
  size_t need = 0;
  ovro::carve_vet(nullptr, 0, n_cand, n_coarse, &need);
  return need;
}

void ovro_vet_default_params(ovro_vet_params* p) {
  if (!p) return;
  p->offline_half = 64;
  p->fit_half = 3;
  p->max_area_ratio = 2.0;
  p->max_noise_std = 1.5;
  p->max_sigma_dev = 2.0;
}

int ovro_vet(const float* d_img, const double* d_stats, int n_chan, int image_size, double cell_dircos,
             int n_coarse, const int32_t* h_nfft, const float* d_psf, const ovro_candidate* h_cand, int n_cand,
             float cut, const ovro_vet_params* params, ovro_vet_result* h_out, void* d_ws, size_t ws_bytes,
             void* stream) {
  using namespace ovro;
  if (!d_img || !d_stats || !h_nfft || !d_psf || n_chan <= 0 || image_size <= 0 || n_coarse <= 0 || n_cand < 0 ||
      !(cell_dircos > 0.0) || (n_cand > 0 && (!h_cand || !h_out)))
    return OVRO_ERR_INVALID_ARG;
  ovro_vet_params prm;
  ovro_vet_default_params(&prm);
  if (params) prm = *params;
  if (prm.offline_half < 1 || prm.offline_half > kMaxOffHalf || prm.fit_half < 1 || prm.fit_half > kMaxFitHalf)
    return OVRO_ERR_UNSUPPORTED;
  std::vector<int> chan0(n_coarse + 1, 0);
  for (int c = 0; c < n_coarse; ++c) {
    if (h_nfft[c] <= 0) return OVRO_ERR_INVALID_ARG;
    chan0[c + 1] = chan0[c] + h_nfft[c];
  }
  if (chan0[n_coarse] != n_chan) return OVRO_ERR_INVALID_ARG;
  std::vector<VetCand> vc(n_cand);
  std::vector<int> chans;
  std::vector<int> chan_slot(n_cand);
  for (int i = 0; i < n_cand; ++i) {
    const ovro_candidate& c = h_cand[i];
    if (c.coarse < 0 || c.coarse >= n_coarse || c.width < 1 || c.row < 0 || c.row >= image_size || c.col < 0 ||
        c.col >= image_size)
      return OVRO_ERR_INVALID_ARG;
    // the boxcar support must lie inside the coarse channel (as the search evaluates it)
    const int s_lo = c.chan - (c.width - 1) / 2, s_hi = c.chan + (c.width - 1) - (c.width - 1) / 2;
    if (s_lo < chan0[c.coarse] || s_hi >= chan0[c.coarse + 1]) return OVRO_ERR_INVALID_ARG;
    vc[i] = VetCand{c.chan, c.width, c.row, c.col, chan0[c.coarse], chan0[c.coarse + 1], c.coarse, 0};
    auto it = std::find(chans.begin(), chans.end(), c.chan);
    chan_slot[i] = static_cast<int>(it - chans.begin());
    if (it == chans.end()) chans.push_back(c.chan);
  }
  size_t need = 0;
  VetWs w = carve_vet(d_ws, ws_bytes, n_cand, n_coarse, &need);
  if (int e = check_workspace(d_ws, ws_bytes, need)) return e;
  cudaStream_t st = as_stream(stream);
  const int h = prm.fit_half;
  const int n_fit = n_cand + n_coarse;
  // fits [0, n_coarse) are the beams, [n_coarse, n_fit) the candidates
  k_vet_psf<<<n_coarse, 128, 0, st>>>(d_psf, image_size, n_coarse, h, w.L, w.valid, w.p0, w.centre);
  OVRO_LAUNCH_CHECK();
  {
    OVRO_PROF("k_vet_fit", st);
    k_vet_fit<<<(n_coarse + 3) / 4, 128, 0, st>>>(w.L, w.valid, w.p0, w.centre, n_coarse, h, w.fit);
    OVRO_LAUNCH_CHECK();
  }
  if (n_cand > 0) {
    OVRO_CUDA_TRY(cudaMemcpyAsync(w.cand, vc.data(), vc.size() * sizeof(VetCand), cudaMemcpyHostToDevice, st));
    OVRO_CUDA_TRY(cudaMemcpyAsync(w.chans, chans.data(), chans.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    {
      OVRO_PROF("k_vet_line", st);
      k_vet_line<<<n_cand, 32 * kLineWarps, 0, st>>>(
          d_img, d_stats, image_size, cell_dircos, w.cand, h, prm.offline_half, w.fit,
          w.L + static_cast<size_t>(n_coarse) * kMaxPix, w.valid + static_cast<size_t>(n_coarse) * kMaxPix,
          w.p0 + 6 * static_cast<size_t>(n_coarse), w.centre + 2 * static_cast<size_t>(n_coarse), w.snr);
      OVRO_LAUNCH_CHECK();
    }
    {
      OVRO_PROF("k_vet_fit", st);
      k_vet_fit<<<(n_cand + 3) / 4, 128, 0, st>>>(
          w.L + static_cast<size_t>(n_coarse) * kMaxPix, w.valid + static_cast<size_t>(n_coarse) * kMaxPix,
          w.p0 + 6 * static_cast<size_t>(n_coarse), w.centre + 2 * static_cast<size_t>(n_coarse), n_cand, h,
          w.fit + static_cast<size_t>(n_coarse) * kFitOut);
      OVRO_LAUNCH_CHECK();
    }
    k_vet_noise<<<static_cast<unsigned>(chans.size()), 256, 0, st>>>(d_img, d_stats, image_size, cell_dircos,
                                                                     w.chans, w.noise);
    OVRO_LAUNCH_CHECK();
  }
  std::vector<double> fit(static_cast<size_t>(n_fit) * kFitOut), snr(n_cand), noise(2 * chans.size());
  std::vector<double> stats(2 * static_cast<size_t>(n_chan));
  OVRO_CUDA_TRY(cudaMemcpyAsync(fit.data(), w.fit, fit.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  OVRO_CUDA_TRY(cudaMemcpyAsync(stats.data(), d_stats, stats.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (n_cand > 0) {
    OVRO_CUDA_TRY(cudaMemcpyAsync(snr.data(), w.snr, snr.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    OVRO_CUDA_TRY(cudaMemcpyAsync(noise.data(), w.noise, noise.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  OVRO_CUDA_TRY(cudaStreamSynchronize(st));

  // decisions: host FP64 comparisons of the device results
  std::vector<double> coarse_sigma(n_coarse);
  for (int c = 0; c < n_coarse; ++c) {
    std::vector<double> s;
    for (int f = chan0[c]; f < chan0[c + 1]; ++f) s.push_back(kMadToSigma * stats[2 * f + 1]);
    std::sort(s.begin(), s.end());
    const size_t k = s.size();
    coarse_sigma[c] = (k % 2) ? s[k / 2] : (s[k / 2 - 1] + s[k / 2]) * 0.5;
  }
  auto fit_ok = [&](const double* o, int cx, int cy) {
    bool ok = o[9] >= 7 && o[10] > 0.5;
    for (int i = 0; i < 9 && ok; ++i) ok = std::isfinite(o[i]);
    return ok && o[0] > 0 && o[3] > 0 && o[5] > 0 && o[3] * o[5] - o[4] * o[4] > 0 &&
           std::fabs(o[1] - cx) <= h && std::fabs(o[2] - cy) <= h;
  };
  const double k_fwhm = 2.0 * std::sqrt(2.0 * std::log(2.0));
  for (int i = 0; i < n_cand; ++i) {
    const ovro_candidate& c = h_cand[i];
    const double* bm = fit.data() + static_cast<size_t>(c.coarse) * kFitOut;
    const double* o = fit.data() + static_cast<size_t>(n_coarse + i) * kFitOut;
    const int c0 = image_size / 2;
    const bool bok = fit_ok(bm, c0, c0);
    const bool fok = fit_ok(o, c.col, c.row);
    ovro_vet_result& r = h_out[i];
    r.flags = 0;
    r.snr_re = static_cast<float>(snr[i]);
    if (snr[i] < static_cast<double>(cut)) r.flags |= OVRO_VET_REEVAL;
    const double s = noise[2 * chan_slot[i]], sd = noise[2 * chan_slot[i] + 1];
    const double ref = coarse_sigma[c.coarse];
    if (sd > prm.max_noise_std || s > prm.max_sigma_dev * ref || s * prm.max_sigma_dev < ref)
      r.flags |= OVRO_VET_NOISY;
    const double det_b = bm[3] * bm[5] - bm[4] * bm[4];
    if (fok && bok) {
      r.area_ratio = std::sqrt(det_b / (o[3] * o[5] - o[4] * o[4]));
      if (r.area_ratio > prm.max_area_ratio) r.flags |= OVRO_VET_EXTENDED;
    } else {
      r.area_ratio = NAN;
      r.flags |= OVRO_VET_FIT;
    }
    r.keep = r.flags == 0;
    r.amp = o[0];
    r.col = o[1];
    r.row = o[2];
    r.sigma_col = o[6];
    r.sigma_row = o[7];
    r.chi2_red = o[8];
    r.beam_fwhm = bok ? k_fwhm * std::pow(det_b, -0.25) : NAN;
    r.sigma_therm = r.beam_fwhm / (2.0 * static_cast<double>(c.snr));
    r.noise_std = sd;
    r.iterations = static_cast<int32_t>(o[11]);
  }
  return OVRO_OK;
}

}  // extern "C"
