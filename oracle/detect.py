"""Oracle: Stage I candidate identification (Section 2.4), FP64.

Steps in the paper's order:

1. Standardise each channel image with the median absolute deviation
   (Section 2.4): med = median of the in-horizon pixels,
   MAD = median |x - med|, z = (x - med) / (1.482602218505602 MAD).
   The constant is 1 / Phi^{-1}(3/4), which makes 1.4826 MAD the standard
   deviation of Gaussian noise.  A channel with MAD = 0 gives z = 0.
2. Subtract a running median along frequency at every pixel, with a window
   wider than 5 kHz (Section 2.4): W = the smallest odd number of channels with
   W * df > 5 kHz, centred, clipped at the edges of the coarse channel (the
   window shrinks there; an even count takes the mean of the two middles).
3. Convolve every pixel spectrum with unit-normalised boxcars of widths 1 to
   100 channels (Section 2.4), sampled densely at small widths:
   {1..10} u {13, 16, ..., 49} u {50, 60, ..., 100}.  Unit-normalised is read
   as 1/sqrt(w), so SNRs are comparable across widths.  Width w at channel k
   covers k - floor((w-1)/2) .. k + ceil((w-1)/2) and is only evaluated where
   that range lies inside the coarse channel.  Keep the largest SNR and its
   width (ties -> smaller width).
4. Convert SNR to a p-value under the standardised (unit Gaussian) noise
   model, p = Q(SNR), and apply Benjamini-Hochberg across all searched
   pixels and channels (Section 2.4): m = in-horizon pixels x channels,
   reject p_(i) <= i alpha / m up to the largest such i.  A fixed-threshold
   mode (SNR >= n_sigma) is provided too; the paper quotes 10 sigma.
5. One-dimensional non-maximum suppression along frequency at each pixel
   (Section 2.4): greedily accept the highest-SNR detection, suppress the
   others within max(1, floor(w/2)) channels of it (w = accepted width),
   repeat.  Ties go to the lower channel.  Done within each coarse channel.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import log_ndtr

MAD_TO_SIGMA = 1.482602218505602
WIDTHS = tuple(list(range(1, 11)) + list(range(13, 50, 3)) + list(range(50, 101, 10)))


def window_channels(df_hz: float, span_hz: float = 5000.0) -> int:
    """Smallest odd W with W * df > span."""
    w = int(math.floor(span_hz / df_hz)) + 1
    while w * df_hz <= span_hz:
        w += 1
    if w % 2 == 0:
        w += 1
    return w


def channel_stats(img: np.ndarray, mask: np.ndarray):
    """(median, MAD) in FP64 of the in-horizon pixels of one image."""
    x = img[mask].astype(np.float64)
    med = float(np.median(x))
    mad = float(np.median(np.abs(x - med)))
    return med, mad


def standardise(cube: np.ndarray, mask: np.ndarray):
    """z-cube [n_chan][N][N] (0 outside the horizon) and per-channel (med, MAD)."""
    z = np.zeros(cube.shape, dtype=np.float64)
    stats = np.zeros((cube.shape[0], 2))
    for f in range(cube.shape[0]):
        med, mad = channel_stats(cube[f], mask)
        stats[f] = med, mad
        if mad > 0:
            z[f][mask] = (cube[f][mask].astype(np.float64) - med) / (MAD_TO_SIGMA * mad)
    return z, stats


def running_median(spec: np.ndarray, w: int) -> np.ndarray:
    """Centred running median along the last axis, window clipped at the ends.

    spec: [..., n].  Interior positions use np.median over a full window; the
    h positions at each end use the shrunken window.  Leading rows are taken
    a few at a time so the window view stays small in memory.
    """
    n = spec.shape[-1]
    h = w // 2
    flat = spec.reshape(-1, n)
    out = np.empty(flat.shape, dtype=np.float64)
    rows = max(1, int(2e8 // max(1, (n * (2 * h + 1)))))
    for r0 in range(0, flat.shape[0], rows):
        blk = flat[r0:r0 + rows]
        o = out[r0:r0 + rows]
        if n > 2 * h:
            win = np.lib.stride_tricks.sliding_window_view(blk, 2 * h + 1, axis=-1)
            o[:, h:n - h] = np.median(win, axis=-1)
        for k in list(range(min(h, n))) + list(range(max(n - h, h), n)):
            lo, hi = max(0, k - h), min(n - 1, k + h)
            o[:, k] = np.median(blk[:, lo:hi + 1], axis=-1)
    return out.reshape(spec.shape)


def highpass(z: np.ndarray, chan_bounds, windows) -> np.ndarray:
    """z' = z - running median, per coarse channel.  z: [n_chan][...]."""
    out = np.empty_like(z, dtype=np.float64)
    zt = np.moveaxis(z, 0, -1)
    ot = np.moveaxis(out, 0, -1)
    for (lo, hi), w in zip(chan_bounds, windows):
        seg = zt[..., lo:hi]
        ot[..., lo:hi] = seg - running_median(seg, w)
    return out


def matched_filter(zp: np.ndarray, chan_bounds, widths=WIDTHS):
    """Max boxcar SNR over widths and its width, per voxel.  zp: [n_chan][...].

    Direct summation in FP64 (no prefix sums).  Voxels where no width fits get
    SNR = -inf and width 0 (cannot happen while width 1 is in the set).
    """
    zt = np.moveaxis(zp, 0, -1)
    snr = np.full(zt.shape, -np.inf)
    wid = np.zeros(zt.shape, dtype=np.int32)
    for lo, hi in chan_bounds:
        n = hi - lo
        seg = zt[..., lo:hi]
        for w in widths:
            a = (w - 1) // 2
            b = w - 1 - a
            if w > n:
                continue
            acc = np.zeros(seg.shape[:-1] + (n - w + 1,))
            for j in range(w):
                acc += seg[..., j:j + n - w + 1]
            s = acc / math.sqrt(w)
            dst = snr[..., lo + a:hi - b]
            better = s > dst
            dst[better] = s[better]
            wid[..., lo + a:hi - b][better] = w
    return np.moveaxis(snr, -1, 0), np.moveaxis(wid, -1, 0)


def log_p(snr) -> np.ndarray:
    """ln Q(SNR), Q the upper tail of the unit Gaussian, in FP64."""
    return log_ndtr(-np.asarray(snr, dtype=np.float64))


def bh_threshold(logp_sorted: np.ndarray, m: int, alpha: float):
    """Benjamini-Hochberg on ascending ln p: number rejected (0 if none)."""
    i = np.arange(1, logp_sorted.size + 1, dtype=np.float64)
    ok = logp_sorted <= np.log(i * alpha / m)
    return int(np.nonzero(ok)[0][-1] + 1) if ok.any() else 0


def select(snr, mask, mode="bh", alpha=0.01, nsigma=10.0):
    """Boolean voxel map of Stage I detections (before NMS).

    snr: [n_chan][N][N]; only in-horizon voxels are tests.
    """
    valid = np.broadcast_to(mask, snr.shape)
    if mode == "fixed":
        return valid & (snr >= nsigma)
    m = int(valid.sum())
    lp = log_p(snr[valid])
    order = np.argsort(lp, kind="stable")
    k = bh_threshold(lp[order], m, alpha)
    sel = np.zeros(snr.shape, dtype=bool)
    if k:
        cut = lp[order][k - 1]
        sel[valid] = lp <= cut
    return sel


@dataclass
class Candidate:
    coarse: int
    fine: int      # channel index within the coarse channel
    chan: int      # global channel index
    row: int
    col: int
    width: int
    snr: float


def nms(sel, snr, wid, chan_bounds):
    """Greedy 1D NMS along frequency per pixel, within each coarse channel."""
    out = []
    ch, rr, cc = np.nonzero(sel)
    by_pix = {}
    for f, r, c in zip(ch, rr, cc):
        by_pix.setdefault((int(r), int(c)), []).append(int(f))
    for (r, c), fl in sorted(by_pix.items()):
        for ci, (lo, hi) in enumerate(chan_bounds):
            fs = [f for f in fl if lo <= f < hi]
            fs.sort(key=lambda f: (-snr[f, r, c], f))
            accepted = []
            for f in fs:
                if any(abs(f - g) <= max(1, wid[g, r, c] // 2) for g in accepted):
                    continue
                accepted.append(f)
            for f in accepted:
                out.append(Candidate(ci, f - lo, f, r, c, int(wid[f, r, c]), float(snr[f, r, c])))
    return out


def chan_bounds_of(nfft_list):
    b, lo = [], 0
    for n in nfft_list:
        b.append((lo, lo + n))
        lo += n
    return b


def detect(cube, mask, nfft_list, coarse_bw_hz=24_000.0, mode="bh", alpha=0.01,
           nsigma=10.0, span_hz=5000.0, widths=WIDTHS, return_all=False):
    """Whole Stage I search over an image cube [n_chan][N][N]."""
    bounds = chan_bounds_of(nfft_list)
    windows = [window_channels(coarse_bw_hz / n, span_hz) for n in nfft_list]
    z, stats = standardise(cube, mask)
    zp = highpass(z, bounds, windows)
    snr, wid = matched_filter(zp, bounds, widths)
    sel = select(snr, mask, mode, alpha, nsigma)
    cands = nms(sel, snr, wid, bounds)
    if return_all:
        return cands, dict(z=z, stats=stats, zp=zp, snr=snr, wid=wid, sel=sel, windows=windows)
    return cands
