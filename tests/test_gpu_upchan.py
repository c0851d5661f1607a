"""GPU parity: unpack + FFT upchannelizer + requantisation against the oracle."""
import numpy as np
import pytest
import torch

import synth
from oracle import upchan as OU

pytestmark = pytest.mark.gpu


def _run(lib, volt, nfft, scales=None):
    d = torch.from_numpy(volt).cuda()
    q, f = lib.upchan(d, nfft, scales=scales, want_f32=True)
    torch.cuda.synchronize()
    return q.cpu().numpy(), f.cpu().numpy()


def _blocks(arr, nfft, n_time, n_input, last):
    out, off = [], 0
    for n in nfft:
        k = n_time // n
        m = n * k * n_input * last
        out.append(arr[off:off + m].reshape(n, k, n_input, last))
        off += m
    return out


def _check_coarse(volt_c, n, qb, fb, scale=None):
    """qb int8 [N][K][in][2], fb float [N][K][in][2] from the GPU for one coarse channel."""
    X = OU.upchannelize(volt_c, n)                               # [N][in][K]
    K = X.shape[2]
    Xg = (fb[..., 0] + 1j * fb[..., 1]).transpose(0, 2, 1)        # [N][in][K]
    # FP32 spectra within 1e-5 of the FP64 oracle, per (input, spectrum)
    den = np.maximum(np.abs(X).max(axis=0), 1e-30)
    rel = np.abs(Xg - X).max(axis=0) / den
    assert rel.max() <= 1e-5, rel.max()
    s = OU.requant_scale(OU.power(volt_c, n), n, K * n) if scale is None else np.asarray(scale)
    # int8: exact against the oracle requantising the GPU's FP32 spectra in FP32
    ref32 = OU.requantize(Xg.astype(np.complex64), s, np.float32)        # [N][in][K][2]
    got = qb.transpose(0, 2, 1, 3)
    assert np.array_equal(got, ref32)
    # against the oracle's own FP64 spectra only rounding ties may differ
    ref64 = OU.requantize(X, s)
    bad = got != ref64
    if bad.any():
        sx = np.stack([X.real, X.imag], -1) * np.asarray(s)[None, :, None, None]
        frac = np.abs(np.abs(sx - np.floor(sx)) - 0.5)
        assert (frac[bad] < 1e-4).all()


def test_tiny_config(lib):
    cfg = synth.make_config("tiny")
    volt = synth.generate(cfg)
    q, f = _run(lib, volt, cfg.nfft)
    qb = _blocks(q, cfg.nfft, cfg.n_time, cfg.n_input, 2)
    fb = _blocks(f, cfg.nfft, cfg.n_time, cfg.n_input, 2)
    for c in range(cfg.n_coarse):
        _check_coarse(volt[c], cfg.nfft[c], qb[c], fb[c])


@pytest.mark.parametrize("nfft", [[2, 4, 8, 16], [32, 64, 128, 512], [1024, 2048, 4096, 8192], [16384]])
def test_all_lengths_and_ragged_inputs(lib, nfft):
    # 6 inputs (3 antennas: not a multiple of 4), leftover samples, mixed N
    g = np.random.default_rng(len(nfft) * 100 + nfft[0])
    n_time = 2 * max(nfft) + 5
    volt = g.integers(0, 256, (len(nfft), n_time, 6), dtype=np.uint8)
    q, f = _run(lib, volt, nfft)
    qb = _blocks(q, nfft, n_time, 6, 2)
    fb = _blocks(f, nfft, n_time, 6, 2)
    for c, n in enumerate(nfft):
        _check_coarse(volt[c], n, qb[c], fb[c])


def test_pure_tone_one_channel(lib):
    # x[n] = i^n (a + ib): every fine channel but (N/4 + N/2) mod N is zero
    n, a, b = 4096, 5, -3
    rot = [(a, b), (-b, a), (-a, -b), (b, -a)]
    re = np.array([rot[t % 4][0] for t in range(2 * n)], np.int8)[:, None].repeat(16, 1)
    im = np.array([rot[t % 4][1] for t in range(2 * n)], np.int8)[:, None].repeat(16, 1)
    volt = synth.pack_nibbles(re, im)[None]
    q, f = _run(lib, volt, [n])
    fb = f.reshape(n, 2, 16, 2)
    mag = np.hypot(fb[..., 0], fb[..., 1])
    kp = (n // 4 + n // 2) % n
    assert np.allclose(mag[kp], n * np.hypot(a, b), rtol=1e-5)
    assert np.delete(mag, kp, axis=0).max() < 1e-5 * n * np.hypot(a, b)


def test_user_scales_and_full_size_sample(lib):
    cfg = synth.make_config("full")
    volt = synth.generate(cfg)
    n = cfg.nfft[0]
    sc = np.full((1, cfg.n_input), 0.01)
    d = torch.from_numpy(volt).cuda()
    q, f = lib.upchan(d, cfg.nfft, want_f32=True)
    qs, _ = lib.upchan(d, cfg.nfft, scales=sc)
    torch.cuda.synchronize()
    K = cfg.n_spec[0]
    qb = q.view(n, K, cfg.n_input, 2)
    fb = f.view(n, K, cfg.n_input, 2)
    qsb = qs.view(n, K, cfg.n_input, 2)
    # sampled inputs at full size, each checked over all fine channels and spectra
    for i in (0, 1, 351, 352, 703):
        sub = volt[0][:, [i]]
        _check_coarse(sub, n, qb[:, :, [i]].cpu().numpy(), fb[:, :, [i]].cpu().numpy())
        Xg = fb[:, :, i].cpu().numpy()
        ref = np.clip(np.rint(np.float32(0.01) * Xg), -127, 127).astype(np.int8)
        assert np.array_equal(qsb[:, :, i].cpu().numpy(), ref)


# ------------------------------------------------ 3,5-smooth lengths, PFB, channel windows
def _split(arr, nfft, n_time, n_input, n_taps=1, count=0):
    out, off = [], 0
    for n in nfft:
        k = n_time // n - n_taps + 1
        c = count or n
        m = c * k * n_input * 2
        out.append(arr[off:off + m].reshape(c, k, n_input, 2))
        off += m
    assert off == arr.size
    return out


def _check_spectra(X, qb, fb, s):
    """X oracle [C][in][K] complex; qb / fb GPU [C][K][in][2]; s the oracle's scales."""
    Xg = (fb[..., 0] + 1j * fb[..., 1]).transpose(0, 2, 1)
    den = np.maximum(np.abs(X).max(axis=0), 1e-30)
    rel = np.abs(Xg - X).max(axis=0) / den
    assert rel.max() <= 1e-5, rel.max()
    ref32 = OU.requantize(Xg.astype(np.complex64), s, np.float32)
    assert np.array_equal(qb.transpose(0, 2, 1, 3), ref32)


@pytest.mark.parametrize("nfft,n_input", [
    ([2400], 704 // 16),                       # the paper's factor, 44 inputs
    ([2400, 6, 10, 12], 6),                    # ragged inputs, mixed lengths in one call
    ([30, 96, 360, 480, 1000], 33),
    ([4800, 7680, 256], 5),                    # four-pass plans, mixed with a power of two
    ([4374], 3),                               # 2 x 3^7: radices 6 and 3
])
def test_mixed_radix_lengths(lib, nfft, n_input):
    g = np.random.default_rng(sum(nfft) + n_input)
    n_time = 3 * max(nfft) + 7
    volt = g.integers(0, 256, (len(nfft), n_time, n_input), dtype=np.uint8)
    q, f = _run(lib, volt, nfft)
    qb = _split(q, nfft, n_time, n_input)
    fb = _split(f, nfft, n_time, n_input)
    specs, ss, _ = OU.upchan_all(volt, nfft)
    for c in range(len(nfft)):
        _check_spectra(specs[c], qb[c], fb[c], ss[c])


def test_2400_pure_tone(lib):
    n, a, b = 2400, -4, 7
    rot = [(a, b), (-b, a), (-a, -b), (b, -a)]
    t = np.arange(2 * n)
    re = np.array([rot[(3 * x) % 4][0] for x in t], np.int8)[:, None].repeat(8, 1)
    im = np.array([rot[(3 * x) % 4][1] for x in t], np.int8)[:, None].repeat(8, 1)
    volt = synth.pack_nibbles(re, im)[None]
    _, f = _run(lib, volt, [n])
    fb = f.reshape(n, 2, 8, 2)
    mag = np.hypot(fb[..., 0], fb[..., 1])
    kp = (3 * n // 4 + n // 2) % n
    assert np.allclose(mag[kp], n * np.hypot(a, b), rtol=1e-5)
    assert np.delete(mag, kp, axis=0).max() < 1e-5 * n * np.hypot(a, b)


def _run_opts(lib, volt, nfft, taps=None, window=None, scales=None):
    d = torch.from_numpy(volt).cuda()
    tt = None if taps is None else [torch.from_numpy(np.ascontiguousarray(h, np.float32)).cuda() for h in taps]
    q, f = lib.upchan(d, nfft, scales=scales, want_f32=True, taps=tt, window=window)
    torch.cuda.synchronize()
    return q.cpu().numpy(), f.cpu().numpy()


@pytest.mark.parametrize("nfft,n_taps,n_input", [([2400], 4, 12), ([96, 60], 3, 7), ([1024], 2, 16), ([6], 5, 2)])
def test_pfb_against_oracle(lib, nfft, n_taps, n_input):
    g = np.random.default_rng(n_taps * 1000 + n_input)
    n_time = (n_taps + 2) * max(nfft) + 3
    volt = g.integers(0, 256, (len(nfft), n_time, n_input), dtype=np.uint8)
    taps = [synth.pfb_prototype(n, n_taps) if c == 0 else g.normal(size=n * n_taps).astype(np.float32)
            for c, n in enumerate(nfft)]
    q, f = _run_opts(lib, volt, nfft, taps=taps)
    qb = _split(q, nfft, n_time, n_input, n_taps)
    fb = _split(f, nfft, n_time, n_input, n_taps)
    specs, ss, _ = OU.upchan_all(volt, nfft, taps=[h.astype(np.float64) for h in taps])
    for c in range(len(nfft)):
        assert specs[c].shape[2] == n_time // nfft[c] - n_taps + 1
        _check_spectra(specs[c], qb[c], fb[c], ss[c])


@pytest.mark.parametrize("nfft,window", [([2400, 2400], (900, 300)), ([4096], (3796, 300)), ([240], (0, 1))])
def test_channel_window(lib, nfft, window):
    g = np.random.default_rng(window[0] + len(nfft))
    n_time = 2 * max(nfft) + 1
    volt = g.integers(0, 256, (len(nfft), n_time, 10), dtype=np.uint8)
    q, f = _run_opts(lib, volt, nfft, window=window)
    qa, fa = _run(lib, volt, nfft)
    lo, cnt = window
    qb = _split(q, nfft, n_time, 10, 1, cnt)
    fb = _split(f, nfft, n_time, 10, 1, cnt)
    qfull = _split(qa, nfft, n_time, 10)
    ffull = _split(fa, nfft, n_time, 10)
    specs, ss, _ = OU.upchan_all(volt, nfft, window=window)
    for c in range(len(nfft)):
        _check_spectra(specs[c], qb[c], fb[c], ss[c])
        if nfft[c] & (nfft[c] - 1):
            # both calls ran the mixed-radix kernel: a window is the same rows of
            # the whole spectrum, bit for bit (a windowed power of two runs the
            # mixed-radix kernel, the whole one the radix-16 kernel: oracle only)
            assert np.array_equal(qb[c], qfull[c][lo:lo + cnt])
            assert np.array_equal(fb[c], ffull[c][lo:lo + cnt])


def test_window_batches_correlate_like_the_whole(lib):
    # Section 2.1: 300-fine-channel batches cross-correlated one after another give
    # the visibilities of correlating all 2400 channels at once
    n_ant, n, k = 8, 2400, 3
    g = np.random.default_rng(5)
    volt = g.integers(0, 256, (1, n * k, 2 * n_ant), dtype=np.uint8)
    d = torch.from_numpy(volt).cuda()
    q_all, _ = lib.upchan(d, [n])
    v_all = lib.correlate(q_all, n_ant, n, k)
    for b in range(n // 300):
        qb, _ = lib.upchan(d, [n], window=(300 * b, 300))
        vb = lib.correlate(qb, n_ant, 300, k)
        assert torch.equal(vb, v_all[300 * b:300 * (b + 1)])


def test_full_size_2400_sample(lib):
    # the paper's search setting: 352 antennas, N = 2400 (9.9 Hz), 30 s -> K = 300;
    # every fine channel and spectrum of sampled inputs against the oracle
    cfg = synth.make_config("full")
    n, n_time = 2400, 720_000
    g = np.random.default_rng(6)
    volt = g.integers(0, 256, (1, n_time, cfg.n_input), dtype=np.uint8)
    d = torch.from_numpy(volt).cuda()
    q, f = lib.upchan(d, [n], want_f32=True)
    torch.cuda.synchronize()
    K = n_time // n
    qb = q.view(n, K, cfg.n_input, 2)
    fb = f.view(n, K, cfg.n_input, 2)
    for i in (0, 5, 351, 700, 703):
        sub = volt[0][:, [i]]
        specs, ss, _ = OU.upchan_all(sub[None], [n])
        _check_spectra(specs[0], qb[:, :, [i]].cpu().numpy(), fb[:, :, [i]].cpu().numpy(), ss[0])


def test_option_errors(lib):
    d = torch.zeros((1, 4800, 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(lib.OvroError):
        lib.upchan(d, [2400], window=(2200, 300))          # past N
    with pytest.raises(lib.OvroError):
        lib.upchan(d, [2400], taps=[torch.ones(3 * 2400, device="cuda")])   # K = 0
    with pytest.raises(lib.OvroError):
        lib.upchan(d, [2401])                               # odd length
    with pytest.raises(lib.OvroError):
        lib.upchan(d, [14])                                 # 2 x 7
