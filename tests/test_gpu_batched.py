"""GPU, the batched workload at full size: 352 antennas, 32 coarse channels
with seeded fine-channel counts N in {1024, 4096, 16384} (K = 234 / 58 / 14
spectra in 10 s), 256^2 images, 20 drifting tones, through the captured and
autotuned pipeline (one graph launch per integration), against the same
integration streamed coarse channel by coarse channel through the public
stage calls, against the oracle on sampled outputs (one coarse channel of
each N: spectra of two inputs, visibilities, an image, the MAD statistics,
one pixel spectrum's z' and SNR), and with every injected tone found."""
import numpy as np
import pytest
import torch

import synth
from synth import workloads as W
from oracle import detect as OD, imaging as OI, upchan as OU, xengine as OX

pytestmark = pytest.mark.gpu


def _key(c):
    return (int(c["chan"]), int(c["row"]), int(c["col"]))


@pytest.fixture(scope="module")
def batched(lib):
    cfg = synth.make_config("batched")
    volt_h = synth.generate_parallel(cfg)
    pos = synth.antenna_positions(cfg)
    freqs = synth.fine_freqs_hz(cfg.nfft)
    volt = torch.from_numpy(volt_h).cuda()
    centres = [synth.coarse_centre_hz(c) for c in range(cfg.n_coarse)]
    N = cfg.image_size
    lib.tune_clear()
    pl = lib.Pipeline(cfg.n_ant, cfg.nfft, centres, cfg.n_time, pos, N, cfg.cell, use_graph=True)
    # noise images of K spectra are sums of K squared beam magnitudes (a
    # skewed, Gamma(K)-like law): at K = 14 the Gaussian p-values pass about one
    # test in eight thousand, some 8 million candidates here
    cap = 1 << 24
    lib.autotune(True)
    try:
        tuned = pl.run(volt, max_out=cap)
    finally:
        lib.autotune(False)
    got = pl.run(volt, max_out=cap)
    assert pl.stats()[1]
    assert lib.correlate_status() == 0
    pl.close()
    del pl
    torch.cuda.empty_cache()
    # one coarse channel of each N is sampled against the oracle
    sample = {}
    for c, n in enumerate(cfg.nfft):
        sample.setdefault(n, c)
    img = torch.empty((cfg.n_chan_total, N, N), dtype=torch.float32, device="cuda")
    keep = {}
    c0 = 0
    for c, (n, k) in enumerate(zip(cfg.nfft, cfg.n_spec)):
        want = sample.get(n) == c
        q, f32 = lib.upchan(volt[c:c + 1].contiguous(), [n], want_f32=want)
        vis = lib.correlate(q, cfg.n_ant, n, k, lib.XENG_TC)
        lib.grid_image(vis, pos, freqs[c0:c0 + n], N, cfg.cell, out=img[c0:c0 + n])
        if want:
            ch = n // 3
            keep[c] = dict(q=q.view(n, k, cfg.n_input, 2)[ch].cpu().numpy(), f32=f32.view(n, k, cfg.n_input, 2),
                           vis=vis[ch].cpu().numpy(), chan=c0 + ch, fine=ch, c0=c0)
        del q, f32, vis
        c0 += n
    torch.cuda.synchronize()
    stage = lib.detect(img, cfg.cell, cfg.nfft, freqs, max_out=cap)
    yield dict(cfg=cfg, volt=volt_h, pos=pos, freqs=freqs, img=img, tuned=tuned, got=got, stage=stage, keep=keep)
    lib.tune_clear()


def test_pipeline_equals_streamed_stage_calls(batched):
    stage = {_key(c): (int(c["width"]), float(c["snr"])) for c in batched["stage"]}
    for run in (batched["tuned"], batched["got"]):
        got = {_key(c): (int(c["width"]), float(c["snr"])) for c in run}
        assert got.keys() == stage.keys()
        for k, (w, s) in got.items():
            assert w == stage[k][0] and abs(s - stage[k][1]) <= 1e-6 * abs(s), k


def test_every_tone_found(batched):
    cfg = batched["cfg"]
    found = {_key(c) for c in batched["got"]}
    chan0 = np.concatenate([[0], np.cumsum(cfg.nfft)])
    T = cfg.n_time / W.F_COARSE_HZ
    for t in cfg.tones:
        df = W.F_COARSE_HZ / cfg.nfft[t.coarse]
        span = int(np.ceil(t.drift_hz_s * T / df))
        chans = range(chan0[t.coarse] + t.fine - 2, chan0[t.coarse] + t.fine + span + 3)
        assert any((ch, t.row + dr, t.col + dc) in found for ch in chans for dr in (-1, 0, 1) for dc in (-1, 0, 1)), t


def test_sampled_spectra_and_visibilities(batched):
    cfg = batched["cfg"]
    for c, s in batched["keep"].items():
        n, k = cfg.nfft[c], cfg.n_spec[c]
        inputs = [5, 600]
        X = OU.upchannelize(batched["volt"][c][:, inputs], n)                 # [N][inputs][K]
        fh = s["f32"][:, :, inputs].cpu().numpy().astype(np.float64)
        got = (fh[..., 0] + 1j * fh[..., 1]).transpose(0, 2, 1)
        for i in range(len(inputs)):
            assert np.abs(got[:, i] - X[:, i]).max() <= 1e-5 * np.abs(X[:, i]).max(), (c, n)
        ref = OX.correlate(s["q"][None].transpose(0, 2, 1, 3), cfg.n_ant)[0]
        assert np.array_equal(s["vis"], ref), (c, n)


def test_sampled_images_and_statistics(lib, batched):
    cfg = batched["cfg"]
    mask = OI.horizon_mask(cfg.image_size, cfg.cell)
    for c, s in batched["keep"].items():
        ch = s["chan"]
        ref, _, _ = OI.dirty_images(s["vis"][None], batched["pos"], batched["freqs"][ch:ch + 1], cfg.image_size,
                                    cfg.cell)
        got = batched["img"][ch].cpu().numpy()
        assert np.abs(got - ref[0]).max() <= 1e-5 * np.abs(ref[0]).max(), c
        n = cfg.nfft[c]
        blk = batched["img"][s["c0"]:s["c0"] + n]
        st = lib.detect_stats(blk, cfg.cell).cpu().numpy()
        for f in range(0, n, max(1, n // 64)):
            med, mad = OD.channel_stats(blk[f].cpu().numpy(), mask)
            assert st[f, 0] == med and st[f, 1] == mad, (c, f)


def test_sampled_pixel_spectrum(lib, batched):
    # one in-horizon pixel through the high-pass and boxcars of each sampled
    # coarse channel (its own window: 215, 855 or 3415 channels)
    cfg = batched["cfg"]
    r, col = cfg.image_size // 2 + 17, cfg.image_size // 2 - 40
    for c, s in batched["keep"].items():
        n = cfg.nfft[c]
        blk = batched["img"][s["c0"]:s["c0"] + n].contiguous()
        st = lib.detect_stats(blk, cfg.cell)
        zp, snr, _ = lib.detect_filter(blk, st, cfg.cell, [n], want_zp=True)
        stats = st.cpu().numpy()
        x = blk[:, r, col].cpu().numpy().astype(np.float64)
        z = np.where(stats[:, 1] > 0, (x - stats[:, 0]) / (OD.MAD_TO_SIGMA * np.where(stats[:, 1] > 0, stats[:, 1], 1)),
                     0.0)
        zpo = OD.highpass(z[:, None], [(0, n)], [OD.window_channels(24000.0 / n)])
        so, _ = OD.matched_filter(zpo, [(0, n)])
        assert np.abs(zp[:, r, col].cpu().numpy() - zpo[:, 0]).max() < 1e-5 * max(1.0, np.abs(zpo).max()), c
        assert np.abs(snr[:, r, col].cpu().numpy() - so[:, 0]).max() < 2e-4, c
