"""GPU parity: FP64 uvw (bit-exact), gridding + 2D FFT dirty images (1e-5)."""
import numpy as np
import pytest
import torch

import synth
from oracle import imaging as OI, xengine as OX

pytestmark = pytest.mark.gpu


def _oracle_p(pos, freqs, n, cell):
    a, b = np.triu_indices(pos.shape[0], 1)
    s = OI.cells_per_metre(freqs, n, cell)[:, None]
    pu = np.rint((pos[a, 0] - pos[b, 0])[None, :] * s * OI.OVERSAMPLE)
    pv = np.rint((pos[a, 1] - pos[b, 1])[None, :] * s * OI.OVERSAMPLE)
    lim = 2.0 ** 30
    return np.clip(pu, -lim, lim).astype(np.int64), np.clip(pv, -lim, lim).astype(np.int64)


@pytest.mark.parametrize("name,n", [("tiny", 64), ("full", 256)])
def test_uvw_bit_exact(lib, name, n):
    cfg = synth.make_config(name)
    pos = synth.antenna_positions(cfg)
    freqs = synth.fine_freqs_hz(cfg.nfft)[::7]
    pu, pv = lib.uvw(pos, freqs, n, 2.0 / n)
    ru, rv = _oracle_p(pos, freqs, OI.PAD * n, 2.0 / n)
    assert np.array_equal(pu.cpu().numpy(), ru) and np.array_equal(pv.cpu().numpy(), rv)


def _vis_random(g, n_chan, n_ant):
    return g.integers(-2 ** 20, 2 ** 20, (n_chan, OX.n_baselines(n_ant), 4, 2)).astype(np.int32)


@pytest.mark.parametrize("n,cell,n_ant", [(64, 2.0 / 64, 16), (64, 0.005, 16), (32, 0.01, 5),
                                          (128, 2.0 / 128, 40), (256, 2.0 / 256, 60)])
def test_images_vs_oracle(lib, n, cell, n_ant):
    g = np.random.default_rng(n + n_ant)
    cfg = synth.Config("t", n_ant, 1, [16], 16, n, 11, core_radius_m=200.0)
    pos = synth.antenna_positions(cfg)
    n_chan = 6
    freqs = 60e6 + np.arange(n_chan) * 1234.5
    vis = _vis_random(g, n_chan, n_ant)
    img, cnt = lib.grid_image(torch.from_numpy(vis).cuda(), pos, freqs, n, cell, want_counts=True)
    ref, ng, nd = OI.dirty_images(vis, pos, freqs, n, cell)
    got = img.cpu().numpy()
    assert np.array_equal(cnt.cpu().numpy(), ng)
    scale = np.abs(ref).max(axis=(1, 2), keepdims=True)
    err = (np.abs(got - ref) / np.maximum(scale, 1e-30)).max()
    assert err <= 1e-5, err


def test_point_source_peak(lib):
    cfg = synth.make_config("tiny", cell_dircos=0.005)
    pos = synth.antenna_positions(cfg)
    n, cell, nu = 64, 0.005, 60e6
    r0, c0 = 40, 21
    l0, m0 = (c0 - n // 2) * cell, (r0 - n // 2) * cell
    a, b = np.triu_indices(cfg.n_ant)
    lam = OI.C_LIGHT / nu
    ph = -2 * np.pi * ((pos[a, 0] - pos[b, 0]) * l0 + (pos[a, 1] - pos[b, 1]) * m0) / lam
    amp = 2 ** 20
    vis = np.zeros((1, a.size, 4, 2), np.int32)
    for p in (0, 3):
        vis[0, :, p, 0] = np.rint(amp * np.cos(ph))
        vis[0, :, p, 1] = np.rint(amp * np.sin(ph))
    img = lib.grid_image(torch.from_numpy(vis).cuda(), pos, [nu], n, cell).cpu().numpy()[0] / amp
    assert np.unravel_index(np.argmax(img), img.shape) == (r0, c0)
    assert abs(img[r0, c0] - 1.0) < 2e-3


def test_pipeline_images_full_size_sample(lib):
    # the full 352-antenna array at 256^2 all-sky: channels sampled against the oracle
    cfg = synth.make_config("full")
    pos = synth.antenna_positions(cfg)
    freqs = synth.fine_freqs_hz(cfg.nfft)
    g = np.random.default_rng(3)
    n_chan = 96
    vis = _vis_random(g, n_chan, cfg.n_ant)
    img = lib.grid_image(torch.from_numpy(vis).cuda(), pos, freqs[:n_chan], 256, 2.0 / 256).cpu().numpy()
    chans = [0, 63, 64, 95]
    ref, ng, nd = OI.dirty_images(vis, pos, freqs, 256, 2.0 / 256, channels=chans)
    scale = np.abs(ref).max(axis=(1, 2), keepdims=True)
    assert (np.abs(img[chans] - ref) / scale).max() <= 1e-5


def _straddling_cut(pos, freqs, n, cell):
    """A uv range over the baselines that are on the grid: the lower cut between
    channels 2 and 3 of the kept baseline a third of the way up in length, the
    upper one past four fifths of them."""
    a, b, _ = OI._cross_pairs(pos.shape[0])
    s = OI.cells_per_metre(freqs[0], OI.PAD * n, cell)
    on = (np.abs(pos[a, 0] - pos[b, 0]) * s < OI.PAD * n / 2 - 5) & (np.abs(pos[a, 1] - pos[b, 1]) * s < OI.PAD * n / 2 - 5)
    lam = OI.uv_length_wavelengths(pos, a, b, freqs[0])[on]
    srt = np.sort(lam)
    L = srt[srt.size // 3] / (freqs[0] / OI.C_LIGHT)
    return L * (0.5 * (freqs[2] + freqs[3]) / OI.C_LIGHT), float(srt[(4 * srt.size) // 5]) * 1.00001


@pytest.mark.parametrize("n,n_ant,mode", [(64, 16, "both"), (64, 16, "gains"), (128, 40, "cut"), (256, 60, "both")])
def test_calibration_and_uv_range_vs_oracle(lib, n, n_ant, mode):
    # per-channel, per-input complex corrections and a baseline-length cut; the
    # lower cut sits between channels 2 and 3 of one baseline, so that baseline
    # is dropped in channels 0-2 and kept in 3-5 (decided per channel on the device)
    g = np.random.default_rng(17 * n + n_ant)
    cfg = synth.Config("t", n_ant, 1, [16], 16, n, 11, core_radius_m=200.0)
    pos = synth.antenna_positions(cfg)
    n_chan, cell = 6, 2.0 / n
    freqs = 60e6 + np.arange(n_chan) * 1234.5
    vis = _vis_random(g, n_chan, n_ant)
    gains = None
    if mode in ("both", "gains"):
        gains = ((1.0 + 0.3 * g.normal(size=(n_chan, 2 * n_ant))) *
                 np.exp(1j * g.uniform(-np.pi, np.pi, (n_chan, 2 * n_ant)))).astype(np.complex64)
    uv = None
    if mode in ("both", "cut"):
        uv = _straddling_cut(pos, freqs, n, cell)
    dg = None if gains is None else torch.from_numpy(gains).cuda()
    img, cnt = lib.grid_image(torch.from_numpy(vis).cuda(), pos, freqs, n, cell, want_counts=True, gains=dg,
                              uv_range=uv)
    ref, ng, nd = OI.dirty_images(vis, pos, freqs, n, cell,
                                  gains=None if gains is None else gains.astype(np.complex128), uv_range=uv)
    assert np.array_equal(cnt.cpu().numpy(), ng), (cnt.cpu().numpy(), ng)
    if uv is not None:
        assert ng[2] == ng[3] - 2                    # the straddling baseline enters at channel 3
    got = img.cpu().numpy()
    scale = np.abs(ref).max(axis=(1, 2), keepdims=True)
    err = (np.abs(got - ref) / np.maximum(scale, 1e-30)).max()
    assert err <= 1e-5, err
