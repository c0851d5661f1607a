"""Pins for the re-evaluation and Stage II vetting oracle (Section 2.4)
against closed forms, exact recoveries and Monte Carlo error scaling."""
import math

import numpy as np
import pytest

from oracle import vetting as V
from oracle.detect import MAD_TO_SIGMA, Candidate, chan_bounds_of


def test_support_and_offline_channels_by_hand():
    assert V.support(100, 1) == (100, 100)
    assert V.support(100, 4) == (99, 102)        # same convention as the matched filter
    assert V.support(100, 5) == (98, 102)
    off = V.offline_channels(100, 5, 0, 1000)
    # g = 2: left 32..95, right 105..168
    assert off.tolist() == list(range(32, 96)) + list(range(105, 169))
    # clipped at the coarse channel [90, 130)
    off = V.offline_channels(100, 5, 90, 130)
    assert off.tolist() == list(range(90, 96)) + list(range(105, 130))
    # w = 1: g = 1 still guards the neighbours
    assert V.offline_channels(10, 1, 0, 30).tolist() == list(range(0, 9)) + list(range(12, 30))


@pytest.mark.parametrize("w", [1, 4, 7, 50])
def test_reevaluate_flat_baseline_closed_form(w):
    # z = c0 off the line, c0 + A on its support: b = c0, MAD = 0 -> sigma = 1,
    # SNR_re = A w / sqrt(w) = A sqrt(w)
    n, k, c0, A = 600, 300, 0.7, 2.5
    z = np.full(n, c0)
    lo, hi = V.support(k, w)
    z[lo:hi + 1] += A
    snr, b, sig, cnt = V.reevaluate(z, k, w, 0, n)
    assert cnt == 128 and b == c0 and sig == 1.0
    assert snr == pytest.approx(A * math.sqrt(w), rel=1e-12)


def test_reevaluate_noise_scale_closed_form():
    # off-line values alternate c0 +- d: median c0, MAD d, sigma = 1.4826 d
    n, k, w, c0, d, A = 400, 200, 3, -0.2, 0.8, 4.0
    j = np.arange(n)
    z = c0 + d * np.where(j % 2 == 0, 1.0, -1.0)
    lo, hi = V.support(k, w)
    z[lo:hi + 1] = c0 + A
    snr, b, sig, _ = V.reevaluate(z, k, w, 0, n)
    assert b == pytest.approx(c0, abs=1e-15)
    assert sig == pytest.approx(MAD_TO_SIGMA * d, rel=1e-12)
    assert snr == pytest.approx(A * w / (MAD_TO_SIGMA * d * math.sqrt(w)), rel=1e-12)


def test_reevaluate_too_few_offline_channels_uses_unit_sigma():
    z = np.arange(20, dtype=float)
    snr, b, sig, cnt = V.reevaluate(z, 10, 3, 5, 16)     # coarse channel [5, 16): 5..7 and 13..15
    assert cnt == 6 and sig == 1.0 and b == np.median([5, 6, 7, 13, 14, 15])
    assert snr == pytest.approx(sum(z[9:12] - b) / math.sqrt(3), rel=1e-12)


def _gauss_img(p, n):
    yy, xx = np.mgrid[0:n, 0:n]
    return V.gauss(p, xx, yy), xx, yy


def test_fit_recovers_a_noiseless_gaussian():
    p = np.array([5.0, 7.3, 6.8, 0.5, 0.1, 0.4])
    img, xx, yy = _gauss_img(p, 15)
    valid = np.ones_like(img, bool)
    f = V.fit_gaussian(img, valid, xx, yy, (img[7, 7], 7, 7, 1.0, 0.0, 1.0), (7, 7), 7)
    assert f.ok and np.allclose(f.p, p, rtol=1e-9, atol=1e-9)
    assert f.chi2_red < 1e-20


def test_fit_errors_match_monte_carlo_scatter():
    # Gaussian noise of sigma 0.4 (chi2_red ~ 0.16): only the chi2_red-scaled
    # covariance predicts the scatter of x0; the unscaled one is 2.5x too wide
    g = np.random.default_rng(12)
    p = np.array([6.0, 3.2, 2.9, 0.6, 0.05, 0.5])
    clean, xx, yy = _gauss_img(p, 7)
    valid = np.ones_like(clean, bool)
    xs, sx, ys, sy = [], [], [], []
    for _ in range(300):
        f = V.fit_gaussian(clean + 0.4 * g.normal(size=clean.shape), valid, xx, yy, (clean[3, 3], 3, 3, 1.0, 0.0, 1.0),
                           (3, 3), 3)
        assert f.ok
        xs.append(f.p[1]); ys.append(f.p[2])
        sx.append(math.sqrt(f.cov[1, 1])); sy.append(math.sqrt(f.cov[2, 2]))
        assert 0.04 < f.chi2_red < 0.4
    assert np.std(xs) == pytest.approx(np.median(sx), rel=0.15)
    assert np.std(ys) == pytest.approx(np.median(sy), rel=0.15)
    assert abs(np.mean(xs) - p[1]) < 4 * np.std(xs) / math.sqrt(300)


def test_fwhm_of_a_circular_gaussian():
    s = 1.7
    assert V.fwhm((1 / s ** 2, 0.0, 1 / s ** 2)) == pytest.approx(2 * math.sqrt(2 * math.log(2)) * s, rel=1e-14)
    # an elliptical one: the geometric mean of the axes
    s1, s2 = 1.2, 3.0
    assert V.fwhm((1 / s1 ** 2, 0.0, 1 / s2 ** 2)) == pytest.approx(2.354820045 * math.sqrt(s1 * s2), rel=1e-9)


def test_beam_fit_of_a_gaussian_psf():
    n = 32
    p = np.array([1.0, n // 2, n // 2, 1 / 1.5 ** 2, 0.0, 1 / 2.0 ** 2])
    psf, _, _ = _gauss_img(p, n)
    f = V.beam_fit(psf)
    assert f.ok and np.allclose(f.p, p, atol=1e-9)


def test_noise_statistics_and_flags():
    g = np.random.default_rng(13)
    n, nc = 48, 12
    mask = np.ones((n, n), bool)
    cube = g.normal(size=(nc, n, n))
    cube[3] *= 3.0                                   # robust sigma a factor 3 off
    t = g.random((n, n)) < 0.05
    cube[7][t] = 25.0 * np.sign(g.normal(size=t.sum()))   # heavy tails: std >> robust sigma
    stats = np.array([[np.median(c), np.median(np.abs(c - np.median(c)))] for c in cube])
    ns = V.noise_stats(cube, stats, mask)
    assert np.allclose(ns[[0, 1, 2]][:, 1], 1.0, atol=0.1)
    assert ns[3, 0] == pytest.approx(3 * np.median(ns[[0, 1, 2, 4]][:, 0]), rel=0.15)
    flags = V.noisy_channels(ns, chan_bounds_of([nc]))
    assert flags.tolist() == [i in (3, 7) for i in range(nc)]
    # a dead image (MAD = 0) is flagged too
    cube[5] = 1.0
    stats[5] = 1.0, 0.0
    assert V.noisy_channels(V.noise_stats(cube, stats, mask), chan_bounds_of([nc]))[5]


def _psf(n, s=1.3):
    p = np.array([1.0, n // 2, n // 2, 1 / s ** 2, 0.0, 1 / s ** 2])
    return _gauss_img(p, n)[0]


def _cube_with_lines(seed=14):
    g = np.random.default_rng(seed)
    n, nc = 40, 300
    cube = g.normal(size=(nc, n, n))
    lines = [  # (row, col, k, w, amplitude per channel, sigma px)
        (10, 12, 80, 3, 6.0, 1.3),       # compact: the beam
        (25, 28, 150, 5, 4.0, 3.5),      # extended: ~2.7x the beam's width
        (30, 9, 220, 1, 2.2, 1.3),       # weak: fails the re-evaluation
    ]
    yy, xx = np.mgrid[0:n, 0:n]
    for r, c, k, w, amp, s in lines:
        lo, hi = V.support(k, w)
        blob = amp * np.exp(-0.5 * ((xx - c) ** 2 + (yy - r) ** 2) / s ** 2)
        cube[lo:hi + 1] += blob
    return cube, lines


def test_vet_end_to_end_on_a_synthetic_cube():
    cube, lines = _cube_with_lines()
    nc, n = cube.shape[0], cube.shape[1]
    mask = np.ones((n, n), bool)
    stats = np.array([[np.median(c), np.median(np.abs(c - np.median(c)))] for c in cube])
    cands = [Candidate(0, k, k, r, c, w, 8.0) for r, c, k, w, _, _ in lines]
    res = V.vet(cube, stats, mask, [nc], cands, 5.0, [_psf(n)])
    compact, ext, weak = res
    assert compact.keep and compact.flags == 0
    assert abs(compact.col - 12) < 4 * compact.sigma_col and abs(compact.row - 10) < 4 * compact.sigma_row
    assert compact.beam_fwhm == pytest.approx(2.354820045 * 1.3, rel=1e-6)
    assert compact.sigma_therm == pytest.approx(compact.beam_fwhm / 16.0)
    assert 0.5 < compact.area_ratio < 1.5
    assert ext.flags & V.EXTENDED and not ext.keep and ext.area_ratio > 4
    assert weak.flags & V.REEVAL and weak.snr_re < 5.0
    # the compact line's SNR_re is its injected boxcar SNR within noise
    assert compact.snr_re == pytest.approx(6.0 * 3 / math.sqrt(3) / 1.0, rel=0.35)
