"""Oracle: Stage I re-evaluation and the automated Stage II cuts (Section 2.4), FP64.

Test infrastructure only: the product path never imports this module.

The paper names the steps without fixing their details; the readings here:

1. Re-evaluation in a local spectral window.  For a candidate of width w at
   channel k (boxcar support S = k - floor((w-1)/2) .. k + ceil((w-1)/2)),
   the guard half-width is the NMS exclusion half-width g = max(1, floor(w/2))
   and the off-line channels are the M = 64 channels on each side beyond the
   guard, O = [lo - g - M, lo - g) u (hi + g, hi + g + M], clipped to the
   coarse channel (lo, hi the ends of S).  On the MAD-standardised spectrum z
   of the candidate's pixel: b = median(z_O) (the small-scale baseline),
   sigma = 1.482602218505602 median(|z_O - b|), and
   SNR_re = sum_S (z - b) / (sigma sqrt(w)).  With fewer than 16 off-line
   channels or sigma = 0, sigma = 1 (the standardised noise model; b = 0 when
   O is empty).  The candidate is kept when SNR_re >= the Stage I cut.
2. The line image: for every pixel p of a (2h+1)^2 cutout centred on the
   candidate (h = 3), L_p = sum_S (z_p - b_p) / sqrt(w) with b_p the median
   of z_p over O.  Pixels outside the image or below the horizon are left out.
3. Gaussian fit (the centroid fit of Section 2.4): least squares of
   A exp(-(a dx^2 + 2 b dx dy + c dy^2) / 2), dx = col - x0, dy = row - y0,
   over the cutout, parameters (A, x0, y0, a, b, c), started at
   (L_centre, col, row, a_beam, b_beam, c_beam).  Covariance
   (J^T J)^-1 chi2_red with chi2_red = sum r^2 / (n - 6), so the 1-sigma
   centroid errors are rescaled by sqrt(chi2_red).  The library's
   least-squares routine finds the minimiser.
4. The synthesized beam: the same fit to the point-spread image (the dirty
   image of unit visibilities) around its centre pixel (N/2, N/2), started
   at (peak, N/2, N/2, 1, 0, 1).  FWHM = 2 sqrt(2 ln 2) (ac - b^2)^(-1/4),
   the geometric mean over the axes; the thermal astrometric error is
   FWHM / (2 SNR) with the Stage I SNR, reported beside the fit errors.
5. Extended morphology: the fitted area over the beam's,
   sqrt(det Q_beam / det Q_fit) with Q = [[a, b], [b, c]], above 2 rejects.
   A failed fit (non-finite, A <= 0, Q not positive definite, centroid more
   than h pixels from the candidate, fewer than 7 pixels) rejects too.
6. Images with abnormal noise: per channel, s = 1.482602218505602 MAD (the
   robust sigma) and sd = the standard deviation of the standardised
   in-horizon pixels.  A channel is flagged when sd > 1.5 or s is more than a
   factor 2 away from the median s over its coarse channel.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.optimize import least_squares

from .detect import MAD_TO_SIGMA

OFFLINE_HALF = 64
FIT_HALF = 3
MAX_AREA_RATIO = 2.0
MAX_NOISE_STD = 1.5
MAX_SIGMA_DEV = 2.0
MIN_OFFLINE = 16

REEVAL, EXTENDED, NOISY, FIT = 1, 2, 4, 8


def support(k: int, w: int):
    """(lo, hi) inclusive channel range of the width-w boxcar at channel k."""
    return k - (w - 1) // 2, k + (w - 1) - (w - 1) // 2


def offline_channels(k: int, w: int, c_lo: int, c_hi: int, m: int = OFFLINE_HALF) -> np.ndarray:
    """Off-line channels O for a candidate at channel k of width w; the coarse
    channel spans [c_lo, c_hi)."""
    lo, hi = support(k, w)
    g = max(1, w // 2)
    left = np.arange(max(c_lo, lo - g - m), max(c_lo, lo - g))
    right = np.arange(min(c_hi, hi + g + 1), min(c_hi, hi + g + m + 1))
    return np.concatenate([left, right]).astype(np.int64)


def reevaluate(z_spec: np.ndarray, k: int, w: int, c_lo: int, c_hi: int, m: int = OFFLINE_HALF):
    """(SNR_re, baseline, sigma, off-line count) on one pixel's z spectrum."""
    off = offline_channels(k, w, c_lo, c_hi, m)
    lo, hi = support(k, w)
    zo = z_spec[off].astype(np.float64)
    b = float(np.median(zo)) if zo.size else 0.0
    sig = MAD_TO_SIGMA * float(np.median(np.abs(zo - b))) if zo.size else 0.0
    if zo.size < MIN_OFFLINE or not sig > 0.0:
        sig = 1.0
    s = float(np.sum(z_spec[lo:hi + 1].astype(np.float64) - b))
    return s / (sig * math.sqrt(w)), b, sig, int(zo.size)


def line_image(z: np.ndarray, mask: np.ndarray, k: int, w: int, c_lo: int, c_hi: int, row: int, col: int,
               h: int = FIT_HALF, m: int = OFFLINE_HALF):
    """(L, valid): the (2h+1)^2 line image around (row, col) and its valid pixels."""
    n = z.shape[1]
    off = offline_channels(k, w, c_lo, c_hi, m)
    lo, hi = support(k, w)
    L = np.zeros((2 * h + 1, 2 * h + 1))
    valid = np.zeros((2 * h + 1, 2 * h + 1), bool)
    for dr in range(-h, h + 1):
        for dc in range(-h, h + 1):
            r, c = row + dr, col + dc
            if not (0 <= r < n and 0 <= c < n and mask[r, c]):
                continue
            zp = z[:, r, c].astype(np.float64)
            b = float(np.median(zp[off])) if off.size else 0.0
            L[dr + h, dc + h] = np.sum(zp[lo:hi + 1] - b) / math.sqrt(w)
            valid[dr + h, dc + h] = True
    return L, valid


def gauss(p, x, y):
    A, x0, y0, a, b, c = p
    dx, dy = x - x0, y - y0
    return A * np.exp(-0.5 * (a * dx * dx + 2.0 * b * dx * dy + c * dy * dy))


def gauss_jac(p, x, y):
    A, x0, y0, a, b, c = p
    dx, dy = x - x0, y - y0
    e = np.exp(-0.5 * (a * dx * dx + 2.0 * b * dx * dy + c * dy * dy))
    f = A * e
    return np.stack([e, f * (a * dx + b * dy), f * (b * dx + c * dy), -0.5 * f * dx * dx, -f * dx * dy,
                     -0.5 * f * dy * dy], axis=-1)


@dataclass
class Fit:
    ok: bool
    p: np.ndarray          # (A, x0, y0, a, b, c)
    cov: np.ndarray        # (J^T J)^-1 chi2_red
    chi2_red: float
    n: int


def fit_gaussian(img: np.ndarray, valid: np.ndarray, x: np.ndarray, y: np.ndarray, p0, centre, h: int) -> Fit:
    """Least-squares elliptical Gaussian over the valid pixels (x = col, y = row)."""
    xv, yv, dv = x[valid].astype(np.float64), y[valid].astype(np.float64), img[valid].astype(np.float64)
    n = dv.size
    p0 = np.asarray(p0, np.float64)
    if n < 7:
        return Fit(False, p0, np.full((6, 6), np.nan), math.nan, n)
    res = least_squares(lambda p: gauss(p, xv, yv) - dv, p0, jac=lambda p: gauss_jac(p, xv, yv), method="lm",
                        xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=20000)
    p = res.x
    r = gauss(p, xv, yv) - dv
    chi2 = float(r @ r) / (n - 6)
    J = gauss_jac(p, xv, yv)
    try:
        cov = np.linalg.inv(J.T @ J) * chi2
    except np.linalg.LinAlgError:
        cov = np.full((6, 6), np.nan)
    A, x0, y0, a, b, c = p
    ok = (np.all(np.isfinite(p)) and np.all(np.isfinite(cov)) and A > 0 and a > 0 and c > 0
          and a * c - b * b > 0 and abs(x0 - centre[0]) <= h and abs(y0 - centre[1]) <= h)
    return Fit(bool(ok), p, cov, chi2, n)


def beam_fit(psf: np.ndarray, h: int = FIT_HALF) -> Fit:
    """Gaussian fit to the point-spread image around (N/2, N/2)."""
    n = psf.shape[0]
    c0 = n // 2
    yy, xx = np.mgrid[c0 - h:c0 + h + 1, c0 - h:c0 + h + 1]
    inside = (yy >= 0) & (yy < n) & (xx >= 0) & (xx < n)
    img = np.zeros(xx.shape)
    img[inside] = psf[yy[inside], xx[inside]]
    return fit_gaussian(img, inside, xx, yy, (psf[c0, c0], c0, c0, 1.0, 0.0, 1.0), (c0, c0), h)


def fwhm(q) -> float:
    """Geometric-mean FWHM of a Gaussian with quadratic form q = (a, b, c)."""
    a, b, c = q
    return 2.0 * math.sqrt(2.0 * math.log(2.0)) * (a * c - b * b) ** -0.25


def noise_stats(cube: np.ndarray, stats: np.ndarray, mask: np.ndarray):
    """Per channel (robust sigma s, std of the standardised in-horizon pixels)."""
    out = np.zeros((cube.shape[0], 2))
    for f in range(cube.shape[0]):
        med, mad = stats[f]
        s = MAD_TO_SIGMA * mad
        if s > 0:
            zf = (cube[f][mask].astype(np.float64) - med) / s
            out[f] = s, float(np.sqrt(np.mean((zf - zf.mean()) ** 2)))
        else:
            out[f] = 0.0, 0.0
    return out


def noisy_channels(ns: np.ndarray, chan_bounds, max_std=MAX_NOISE_STD, max_dev=MAX_SIGMA_DEV) -> np.ndarray:
    flag = np.zeros(ns.shape[0], bool)
    for lo, hi in chan_bounds:
        ref = float(np.median(ns[lo:hi, 0]))
        s = ns[lo:hi, 0]
        flag[lo:hi] = (ns[lo:hi, 1] > max_std) | (s > max_dev * ref) | (s * max_dev < ref)
    return flag


@dataclass
class Vetted:
    keep: bool
    flags: int
    snr_re: float
    area_ratio: float
    col: float
    row: float
    sigma_col: float
    sigma_row: float
    chi2_red: float
    amp: float
    beam_fwhm: float
    sigma_therm: float
    noise_std: float


def vet(cube: np.ndarray, stats: np.ndarray, mask: np.ndarray, nfft_list, cands, cut: float, psfs,
        h: int = FIT_HALF, m: int = OFFLINE_HALF, max_area=MAX_AREA_RATIO, max_std=MAX_NOISE_STD,
        max_dev=MAX_SIGMA_DEV):
    """Re-evaluate and vet Stage I candidates (oracle.detect.Candidate records).

    cube [n_chan][N][N] images, stats [n_chan][2] (median, MAD), psfs one
    point-spread image per coarse channel.
    """
    from .detect import chan_bounds_of
    bounds = chan_bounds_of(nfft_list)
    z = np.zeros(cube.shape)
    for f in range(cube.shape[0]):
        med, mad = stats[f]
        if mad > 0:
            z[f][mask] = (cube[f][mask].astype(np.float64) - med) / (MAD_TO_SIGMA * mad)
    ns = noise_stats(cube, stats, mask)
    noisy = noisy_channels(ns, bounds, max_std, max_dev)
    beams = [beam_fit(p, h) for p in psfs]
    out = []
    for cd in cands:
        c_lo, c_hi = bounds[cd.coarse]
        snr_re, _, _, _ = reevaluate(z[:, cd.row, cd.col], cd.chan, cd.width, c_lo, c_hi, m)
        L, valid = line_image(z, mask, cd.chan, cd.width, c_lo, c_hi, cd.row, cd.col, h, m)
        yy, xx = np.mgrid[cd.row - h:cd.row + h + 1, cd.col - h:cd.col + h + 1]
        bm = beams[cd.coarse]
        fit = fit_gaussian(L, valid, xx, yy, (L[h, h], cd.col, cd.row, bm.p[3], bm.p[4], bm.p[5]),
                           (cd.col, cd.row), h)
        flags = 0
        if snr_re < cut:
            flags |= REEVAL
        if noisy[cd.chan]:
            flags |= NOISY
        det_b = bm.p[3] * bm.p[5] - bm.p[4] ** 2
        if fit.ok and bm.ok:
            det_f = fit.p[3] * fit.p[5] - fit.p[4] ** 2
            ratio = math.sqrt(det_b / det_f)
            if ratio > max_area:
                flags |= EXTENDED
        else:
            ratio = math.nan
            flags |= FIT
        bf = fwhm(bm.p[3:6]) if bm.ok else math.nan
        out.append(Vetted(flags == 0, flags, snr_re, ratio, fit.p[1], fit.p[2], math.sqrt(fit.cov[1, 1]),
                          math.sqrt(fit.cov[2, 2]), fit.chi2_red, fit.p[0], bf, bf / (2.0 * cd.snr),
                          ns[cd.chan, 1]))
    return out
