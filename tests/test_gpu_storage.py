"""GPU: 16-bit storage of the half-transformed uv grid (BF16; FP16 with a
power-of-two scale per row) against the FP64 oracle images; FP32 arithmetic
throughout.  The errors are stated per result (L-inf and L2 relative to the
image, and the peak position of a point source)."""
import numpy as np
import pytest
import torch

import synth
from oracle import imaging as OI, xengine as OX

pytestmark = pytest.mark.gpu

# bounds on ||err||_inf / max|I| (measured errors are printed; the 16-bit
# storage rounds each value to 2^-9 (BF16) or 2^-12 of its row maximum (FP16))
TOL = {0: 1e-5, 1: 1.5e-2, 2: 2e-3}
NAMES = {0: "fp32", 1: "bf16", 2: "fp16"}


def _errs(got, ref):
    scale = np.abs(ref).max(axis=(1, 2), keepdims=True)
    linf = (np.abs(got - ref) / scale).max()
    l2 = np.sqrt(((got - ref) ** 2).sum()) / np.sqrt((ref ** 2).sum())
    return float(linf), float(l2)


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("n,n_ant", [(32, 12), (64, 16), (256, 60)])
def test_storage_vs_oracle(lib, storage, n, n_ant):
    g = np.random.default_rng(7 * n + storage)
    cfg = synth.Config("t", n_ant, 1, [16], 16, n, 11, core_radius_m=200.0)
    pos = synth.antenna_positions(cfg)
    freqs = 60e6 + np.arange(5) * 977.0
    vis = g.integers(-2 ** 20, 2 ** 20, (5, OX.n_baselines(n_ant), 4, 2)).astype(np.int32)
    dv = torch.from_numpy(vis).cuda()
    got = lib.grid_image(dv, pos, freqs, n, 2.0 / n, storage=storage).cpu().numpy()
    ref, _, _ = OI.dirty_images(vis, pos, freqs, n, 2.0 / n)
    linf, l2 = _errs(got, ref)
    print(f"{NAMES[storage]} N={n}: Linf {linf:.2e} L2 {l2:.2e}")
    assert linf <= TOL[storage] and l2 <= TOL[storage]


def test_c4_1024_sampled(lib):
    # 352-antenna array, 1024^2 all-sky images (G = 2048): point source at a
    # pixel centre on top of random visibilities, channels sampled against the oracle
    cfg = synth.make_config("precision")
    pos = synth.antenna_positions(cfg)
    n = cfg.image_size
    cell = cfg.cell
    freqs = synth.fine_freqs_hz(cfg.nfft)[1000:1008]
    a, b = np.triu_indices(cfg.n_ant)
    r0, c0 = 612, 401
    l0, m0 = (c0 - n // 2) * cell, (r0 - n // 2) * cell
    g = np.random.default_rng(4)
    vis = g.integers(-2 ** 14, 2 ** 14, (freqs.size, a.size, 4, 2)).astype(np.int64)
    for f, nu in enumerate(freqs):
        ph = -2 * np.pi * ((pos[a, 0] - pos[b, 0]) * l0 + (pos[a, 1] - pos[b, 1]) * m0) * nu / OI.C_LIGHT
        for p in (0, 3):
            vis[f, :, p, 0] += np.rint(2 ** 18 * np.cos(ph)).astype(np.int64)
            vis[f, :, p, 1] += np.rint(2 ** 18 * np.sin(ph)).astype(np.int64)
    vis = vis.astype(np.int32)
    dv = torch.from_numpy(vis).cuda()
    chans = [0, 7]
    ref, _, _ = OI.dirty_images(vis, pos, freqs, n, cell, channels=chans)
    for storage in (0, 1, 2):
        got = lib.grid_image(dv, pos, freqs, n, cell, storage=storage).cpu().numpy()
        linf, l2 = _errs(got[chans], ref)
        peaks = [np.unravel_index(np.argmax(im), im.shape) for im in got]
        print(f"c4 1024^2 {NAMES[storage]}: Linf {linf:.2e} L2 {l2:.2e} peaks {set(peaks)}")
        assert linf <= TOL[storage] and l2 <= TOL[storage]
        assert all(pk == (r0, c0) for pk in peaks)
