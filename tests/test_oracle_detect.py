"""Pins for the Stage I detection oracle (Section 2.4)."""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import ndtri, erfc

import synth
from oracle import detect as D

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_mad_constant():
    assert D.MAD_TO_SIGMA == pytest.approx(1.0 / ndtri(0.75), rel=1e-15)


def test_channel_stats_brute_force():
    g = np.random.default_rng(1)
    for n in (7, 8, 33):
        x = g.normal(size=(1, n))
        mask = np.ones((1, n), bool)
        s = sorted(x[0].tolist())
        med = s[n // 2] if n % 2 else 0.5 * (s[n // 2 - 1] + s[n // 2])
        dev = sorted(abs(v - med) for v in x[0])
        mad = dev[n // 2] if n % 2 else 0.5 * (dev[n // 2 - 1] + dev[n // 2])
        assert D.channel_stats(x, mask) == (pytest.approx(med, abs=0), pytest.approx(mad, abs=0))


def test_mad_gives_unit_sigma_on_noise():
    g = np.random.default_rng(2)
    cube = g.normal(3.0, 7.0, size=(4, 128, 128))
    mask = np.ones((128, 128), bool)
    z, stats = D.standardise(cube, mask)
    for f in range(4):
        assert abs(z[f].std() - 1.0) < 0.02           # sampling error ~ 1 / sqrt(2 * 16384)
        assert abs(stats[f, 1] * D.MAD_TO_SIGMA - 7.0) < 0.15


def test_window_rule():
    # smallest odd W with W df > 5 kHz
    assert D.window_channels(24_000 / 8192) == 1707
    assert D.window_channels(24_000 / 256) == 55
    assert D.window_channels(10.0) == 501               # 500 * 10 Hz is not "over" 5 kHz
    g = json.load(open(os.path.join(GOLD, "paper_numbers.json")))
    w = D.window_channels(g["fine_channel_hz_search"], g["running_median_window_over_hz"])
    assert w * g["fine_channel_hz_search"] > g["running_median_window_over_hz"] > g["widest_line_hz"]


def test_running_median_brute_force():
    g = np.random.default_rng(3)
    for n, w in ((40, 7), (12, 9), (5, 11), (30, 1)):
        x = g.normal(size=(3, n))
        got = D.running_median(x, w)
        h = w // 2
        for r in range(3):
            for k in range(n):
                win = sorted(x[r, max(0, k - h): min(n, k + h + 1)].tolist())
                m = len(win)
                ref = win[m // 2] if m % 2 else 0.5 * (win[m // 2 - 1] + win[m // 2])
                assert got[r, k] == ref


def test_width_set():
    g = json.load(open(os.path.join(GOLD, "paper_numbers.json")))
    w = D.WIDTHS
    assert len(w) == 29 and len(set(w)) == 29 and list(w) == sorted(w)
    assert w[0] == g["boxcar_width_min_channels"] and w[-1] == g["boxcar_width_max_channels"]
    assert list(w[:10]) == list(range(1, 11))          # single-channel spacing at small widths


def test_matched_filter_vs_convolve():
    g = np.random.default_rng(4)
    n = 300
    zp = g.normal(size=(n, 2, 3))
    widths = (1, 2, 5, 8, 50, 100)
    snr, wid = D.matched_filter(zp, [(0, n)], widths)
    best = np.full((n, 2, 3), -np.inf)
    bw = np.zeros((n, 2, 3), int)
    for w in widths:
        a = (w - 1) // 2
        for r in range(2):
            for c in range(3):
                full = np.convolve(zp[:, r, c], np.ones(w), mode="valid") / math.sqrt(w)
                # valid output j covers channels j .. j + w - 1, centred at k = j + a
                for j, v in enumerate(full):
                    if v > best[j + a, r, c]:
                        best[j + a, r, c], bw[j + a, r, c] = v, w
    assert np.allclose(snr, best, rtol=1e-12, atol=1e-12) and np.array_equal(wid, bw)


def test_matched_filter_respects_coarse_edges():
    zp = np.zeros((20, 1, 1))
    zp[9, 0, 0] = 5.0      # last channel of coarse 0
    zp[10, 0, 0] = 5.0     # first channel of coarse 1
    snr, wid = D.matched_filter(zp, [(0, 10), (10, 20)], (1, 2))
    # width 2 at channel 9 would span 9..10 across the boundary: not evaluated
    assert wid[9, 0, 0] == 1 and snr[9, 0, 0] == 5.0


def test_log_p_closed_form():
    s = np.array([0.0, 1.0, 3.0, 10.0, 30.0])
    assert np.allclose(D.log_p(s), np.log(0.5 * erfc(s / math.sqrt(2))), rtol=1e-12)
    # far tail: ln Q(s) ~ -s^2/2 - ln(s sqrt(2 pi)) + ln(1 - 1/s^2 + 3/s^4)
    s = 60.0
    ref = -s * s / 2 - math.log(s * math.sqrt(2 * math.pi)) + math.log(1 - 1 / s ** 2 + 3 / s ** 4)
    assert D.log_p(s) == pytest.approx(ref, rel=1e-9)


def test_bh_published_example():
    g = json.load(open(os.path.join(GOLD, "bh_example.json")))
    p = np.array(g["p_values"])
    k = D.bh_threshold(np.log(np.sort(p)), p.size, g["alpha"])
    assert k == g["n_rejected"]
    assert int((p <= g["alpha"] / p.size).sum()) == g["n_rejected_bonferroni"]


def test_bh_brute_force_and_noise_fdr():
    g = np.random.default_rng(5)
    for _ in range(20):
        p = np.concatenate([g.uniform(size=200), g.uniform(0, 1e-4, size=g.integers(0, 10))])
        m, alpha = p.size, 0.05
        ps = sorted(p.tolist())
        ref = 0
        for i in range(1, m + 1):
            if ps[i - 1] <= i * alpha / m:
                ref = i
        assert D.bh_threshold(np.log(np.sort(p)), m, alpha) == ref
    # noise only: P(any rejection) = alpha for independent tests, so over many
    # seeds the mean number of false discoveries stays near or below alpha
    fd = [D.select(g.normal(size=(8, 16, 16)), np.ones((16, 16), bool), "bh", 0.05).sum() > 0
          for _ in range(400)]
    assert np.mean(fd) < 0.05 + 3 * math.sqrt(0.05 * 0.95 / 400)


def test_nms_half_width_rule_and_brute_force():
    # half-width max(1, floor(w / 2)): w = 1, 2, 3 -> 1; w = 4 -> 2; w = 100 -> 50
    n = 40
    snr = np.zeros((n, 1, 1))
    wid = np.ones((n, 1, 1), int)
    sel = np.zeros((n, 1, 1), bool)
    for f, s, w in ((10, 9.0, 4), (12, 8.0, 1), (13, 7.5, 1), (20, 6.0, 1), (21, 6.0, 1), (30, 5.0, 100)):
        snr[f], wid[f], sel[f] = s, w, True
    cands = D.nms(sel, snr, wid, [(0, n)])
    got = [(c.chan, c.width) for c in cands]
    # 10 (w4, hw2) kills 12; 13 survives (3 away); 20 beats 21 on the tie (lower channel);
    # 30 is outside every accepted region
    assert got == [(10, 4), (13, 1), (20, 1), (30, 100)]


def test_nms_random_vs_brute_force():
    g = np.random.default_rng(6)
    n = 64
    for _ in range(30):
        snr = g.normal(size=(n, 1, 1)).round(1)
        wid = g.choice(D.WIDTHS, size=(n, 1, 1))
        sel = g.uniform(size=(n, 1, 1)) < 0.3
        got = {c.chan for c in D.nms(sel, snr, wid, [(0, n)])}
        live = [f for f in range(n) if sel[f, 0, 0]]
        acc = []
        while live:
            best = max(live, key=lambda f: (snr[f, 0, 0], -f))
            acc.append(best)
            hw = max(1, wid[best, 0, 0] // 2)
            live = [f for f in live if f != best and abs(f - best) > hw]
        assert got == set(acc)


@pytest.fixture(scope="module")
def tiny_pipeline():
    from oracle import upchan as U, xengine as X, imaging as I
    cfg = synth.make_config("tiny", cell_dircos=0.005)
    vol = synth.generate(cfg)
    pos = synth.antenna_positions(cfg)
    specs, ss, qs = U.upchan_all(vol, cfg.nfft)
    q = np.concatenate(qs)
    vis = X.correlate(q, cfg.n_ant)
    freqs = synth.fine_freqs_hz(cfg.nfft)
    imgs, ng, nd = I.dirty_images(vis, pos, freqs, cfg.image_size, cfg.cell)
    return cfg, imgs, ng, nd


def test_injected_tone_detected(tiny_pipeline):
    cfg, imgs, ng, nd = tiny_pipeline
    assert nd.max() == 0                               # this cell fits every baseline
    from oracle import imaging as I
    mask = I.horizon_mask(cfg.image_size, cfg.cell)
    cands = D.detect(imgs, mask, cfg.nfft)
    t = cfg.tones[0]
    chan = sum(cfg.nfft[: t.coarse]) + t.fine
    hit = [c for c in cands if c.chan == chan and c.row == t.row and c.col == t.col]
    assert hit and hit[0].width == 1
    # the tone is the brightest candidate, its PSF sidelobes aside
    assert max(cands, key=lambda c: c.snr).chan == chan
