"""GPU parity: the drift-rate search (ovro_drift_search) against the oracle on
synthetic sub-integration cubes with drifting tones, and end to end through
sub-integration slicing, correlation, imaging and Stage I's filters."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import drift as DR, imaging as OI

pytestmark = pytest.mark.gpu


def _cube(seed, T, nfft, n, tones):
    g = np.random.default_rng(seed)
    z = g.normal(size=(T, sum(nfft), n, n))
    tab = DR.shift_table(T)
    for f0, d0, r, c, a in tones:
        for t in range(T):
            z[t, f0 + (tab[abs(d0), t] if d0 >= 0 else -tab[abs(d0), t]), r, c] += a
    return z.astype(np.float32)


@pytest.mark.parametrize("T", [2, 4, 8, 16])
def test_maps_and_candidates_against_oracle(lib, T):
    n, nfft = 32, [96, 64]
    cell = 2.0 / n
    a = 12.0 / math.sqrt(T) + 1.0                      # path SNR a sqrt(T) >= 13
    tones = [(30, T - 1, 10, 12, a), (70, -(T // 2), 20, 9, a + 1), (100, 0, 16, 16, a + 2),
             (158, -(T - 1), 5, 15, a + 0.5)]
    z = _cube(T, T, nfft, n, tones)
    freqs = synth.fine_freqs_hz(nfft)
    cands, drifts, snr, drm = lib.drift_search(torch.from_numpy(z).cuda(), cell, nfft, freqs, 5.0, want_maps=True)
    mask = OI.horizon_mask(n, cell)
    rs, rd, rc, rdr = DR.drift_search(z.astype(np.float64), mask, nfft, 5.0)
    gs, gd = snr.cpu().numpy(), drm.cpu().numpy()
    assert np.all(np.isneginf(gs[:, ~mask])) and np.all(gd[:, ~mask] == 0)
    assert np.allclose(gs[:, mask], rs[:, mask], rtol=0, atol=2e-5 * max(1.0, np.abs(rs[:, mask]).max()))
    # drifts equal except where another drift's SNR is within rounding of the best
    diff = gd != rd
    if diff.any():
        for f, r, c in zip(*np.nonzero(diff)):
            assert abs(gs[f, r, c] - rs[f, r, c]) < 1e-4
    got = sorted((int(x["chan"]), int(x["row"]), int(x["col"]), int(d)) for x, d in zip(cands, drifts))
    assert got == sorted((x.chan, x.row, x.col, int(d)) for x, d in zip(rc, rdr))
    for f0, d0, r, c, _ in tones:
        assert any(int(x["chan"]) == f0 and x["row"] == r and x["col"] == c and d == d0 for x, d in zip(cands, drifts))
    assert all(x["width"] == abs(d) + 1 for x, d in zip(cands, drifts))


def test_spectra_slice(lib):
    g = torch.Generator(device="cuda").manual_seed(1)
    for n_in in (704, 6):
        q = torch.randint(-127, 128, (7, 29, n_in, 2), generator=g, device="cuda", dtype=torch.int16).to(torch.int8)
        s = lib.spectra_slice(q, 7, 29, n_in, 9, 11)
        assert torch.equal(s, q[:, 9:20])


def test_drifting_tone_end_to_end(lib):
    # a tone drifting ~6 fine channels over the integration: 8 sub-integrations
    # imaged separately, filtered by Stage I, searched over drift: found at its
    # start channel and pixel with its drift, as the oracle finds it on the same cubes
    cfg = synth.make_config("tiny", cell_dircos=0.005, n_tones=0, n_time=128 * 256)
    N = cfg.nfft[0]
    df = 24000.0 / N                                  # fine-channel width, Hz
    t_int = cfg.n_time / 24000.0                      # integration, s
    n_bl = cfg.n_ant * (cfg.n_ant - 1) // 2
    amp = synth.tone_amplitude(60.0, N, cfg.n_time // N, n_bl)
    cfg.tones = [synth.Tone(0, 100, 30, 34, amp, 0.0, 6.0 * df / t_int, 60.0)]
    volt = torch.from_numpy(synth.generate(cfg)).cuda()
    pos = synth.antenna_positions(cfg)
    freqs = synth.fine_freqs_hz(cfg.nfft)
    q, _ = lib.upchan(volt, cfg.nfft)
    T, K = 8, cfg.n_spec[0]
    kt = K // T
    zps = []
    n_chan = cfg.n_chan_total
    for t in range(T):
        vis = torch.empty((n_chan, lib.n_baselines(cfg.n_ant), 4, 2), dtype=torch.int32, device="cuda")
        qoff = c0 = 0
        for n, k in zip(cfg.nfft, cfg.n_spec):
            m = n * k * cfg.n_input * 2
            sub = lib.spectra_slice(q[qoff:qoff + m], n, k, cfg.n_input, t * kt, kt)
            lib.correlate(sub, cfg.n_ant, n, kt, out=vis[c0:c0 + n])
            qoff += m
            c0 += n
        img = lib.grid_image(vis, pos, freqs, cfg.image_size, cfg.cell)
        st = lib.detect_stats(img, cfg.cell)
        zp, _, _ = lib.detect_filter(img, st, cfg.cell, cfg.nfft, want_zp=True)
        zps.append(zp)
    zsub = torch.stack(zps)
    cands, drifts = lib.drift_search(zsub, cfg.cell, cfg.nfft, freqs, 8.0)
    hit = [(int(c["chan"]), int(d), float(c["snr"])) for c, d in zip(cands, drifts)
           if c["row"] == 30 and c["col"] == 34]
    assert hit, "drifting tone not found"
    chan, d, s = max(hit, key=lambda h: h[2])
    assert abs(chan - 100) <= 1 and abs(d - 6) <= 1, hit
    mask = OI.horizon_mask(cfg.image_size, cfg.cell)
    _, _, rc, rdr = DR.drift_search(zsub.cpu().numpy().astype(np.float64), mask, cfg.nfft, 8.0)
    assert sorted((c.chan, c.row, c.col, dd) for c, dd in zip(rc, rdr)) == \
        sorted((int(c["chan"]), int(c["row"]), int(c["col"]), int(dd)) for c, dd in zip(cands, drifts))


@pytest.mark.parametrize("T,alpha", [(4, 0.01), (8, 0.05)])
def test_bh_mode_against_oracle(lib, T, alpha):
    # Benjamini-Hochberg over the map of maxima over drifts, m = in-horizon
    # pixels x channels, decided bin by bin on the GPU: the oracle's selection
    n, nfft = 32, [96, 64]
    cell = 2.0 / n
    a = 12.0 / math.sqrt(T) + 1.0
    tones = [(30, T - 1, 10, 12, a), (70, -(T // 2), 20, 9, a + 1), (100, 0, 16, 16, a + 2)]
    z = _cube(T + 100, T, nfft, n, tones)
    freqs = synth.fine_freqs_hz(nfft)
    prm = lib.detect_params(alpha=alpha)
    cands, drifts = lib.drift_search(torch.from_numpy(z).cuda(), cell, nfft, freqs, params=prm)
    mask = OI.horizon_mask(n, cell)
    _, _, rc, rdr = DR.drift_search(z.astype(np.float64), mask, nfft, mode="bh", alpha=alpha)
    assert len(rc) > 0
    got = sorted((int(x["chan"]), int(x["row"]), int(x["col"]), int(d)) for x, d in zip(cands, drifts))
    assert got == sorted((x.chan, x.row, x.col, int(d)) for x, d in zip(rc, rdr))
