"""Pins for the upchannelizer oracle (Section 2.1) against closed forms."""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import upchan as U

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _bytes_from(re, im):
    return synth.pack_nibbles(np.asarray(re, np.int8), np.asarray(im, np.int8))


def test_unpack_all_nibbles():
    # every (re, im) pair in [-8, 7]^2 survives pack -> unpack, and a few bytes by hand
    re, im = np.meshgrid(np.arange(-8, 8), np.arange(-8, 8), indexing="ij")
    b = _bytes_from(re.ravel(), im.ravel())
    r2, i2 = U.unpack(b)
    assert np.array_equal(r2, re.ravel()) and np.array_equal(i2, im.ravel())
    r, i = U.unpack(np.array([0x00, 0x7F, 0x80, 0xF1, 0x17, 0x88], np.uint8))
    assert r.tolist() == [0, 7, -8, -1, 1, -8]
    assert i.tolist() == [0, -1, 0, 1, 7, -8]


def _rotating_tone(n_time, n_input, k0_quarter, a, b):
    """x[n] = i^(k n) (a + i b): exact integer tone at baseband bin k N/4."""
    rot = [(a, b), (-b, a), (-a, -b), (b, -a)]
    re = np.empty((n_time, n_input), np.int8)
    im = np.empty((n_time, n_input), np.int8)
    for n in range(n_time):
        r, i = rot[(k0_quarter * n) % 4]
        re[n, :] = r
        im[n, :] = i
    return _bytes_from(re, im)


@pytest.mark.parametrize("nfft", [4, 8, 256, 8192])
@pytest.mark.parametrize("quarter", [0, 1, 2, 3])
def test_pure_tone_lands_in_one_channel(nfft, quarter):
    # a tone at baseband bin q N / 4 lands in exactly one fine channel,
    # fftshifted index (q N/4 + N/2) mod N, with value N (a + i b) and power N^2 |a+ib|^2
    a, b = 3, -5
    k = 2
    v = _rotating_tone(k * nfft, 2, quarter, a, b)
    X = U.upchannelize(v, nfft)                      # [N][input][K]
    kp = (quarter * nfft // 4 + nfft // 2) % nfft
    expect = np.zeros(nfft, complex)
    expect[kp] = nfft * (a + 1j * b)
    for i in range(2):
        for s in range(k):
            assert np.max(np.abs(X[:, i, s] - expect)) < 1e-9 * nfft
    assert abs(np.abs(X[kp, 0, 0]) ** 2 - nfft ** 2 * (a * a + b * b)) < 1e-6 * nfft ** 2


def test_parseval_exact_rhs():
    g = np.random.default_rng(1)
    nfft, k, ni = 512, 3, 5
    re = g.integers(-7, 8, (k * nfft, ni))
    im = g.integers(-7, 8, (k * nfft, ni))
    X = U.upchannelize(_bytes_from(re, im), nfft)
    lhs = (np.abs(X) ** 2).sum(axis=0)               # [input][K]
    rhs = nfft * (re ** 2 + im ** 2).reshape(k, nfft, ni).sum(axis=1).T   # exact ints
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=0)


def test_impulse_gives_flat_spectrum():
    nfft = 64
    re = np.zeros((nfft, 1), int)
    im = np.zeros((nfft, 1), int)
    re[17, 0], im[17, 0] = 5, -2
    X = U.upchannelize(_bytes_from(re, im), nfft)
    assert np.allclose(np.abs(X[:, 0, 0]), math.hypot(5, 2), rtol=1e-13)


def test_small_n_integer_dft():
    # N = 2 and N = 4 have integer twiddles; write out the DFT by hand
    x = [(3, 1), (-2, 4), (7, -7), (-8, 0)]
    re = np.array([[p[0]] for p in x])
    im = np.array([[p[1]] for p in x])
    z = [complex(*p) for p in x]
    X2 = U.upchannelize(_bytes_from(re, im), 2)      # two spectra of N = 2
    for s in range(2):
        x0, x1 = z[2 * s], z[2 * s + 1]
        assert X2[:, 0, s].tolist() == [x0 - x1, x0 + x1]       # fftshift: [bin 1, bin 0]
    X4 = U.upchannelize(_bytes_from(re, im), 4)[:, 0, 0]
    d = [sum(z[n] * (1j) ** (-k * n) for n in range(4)) for k in range(4)]
    assert np.allclose(X4, [d[2], d[3], d[0], d[1]], atol=1e-12)


def test_leftover_samples_dropped():
    g = np.random.default_rng(2)
    nfft = 16
    v = g.integers(0, 256, (3 * nfft + 7, 4), dtype=np.uint8)
    v2 = v.copy()
    v2[3 * nfft:] = g.integers(0, 256, (7, 4), dtype=np.uint8)
    assert np.array_equal(U.upchannelize(v, nfft), U.upchannelize(v2, nfft))
    assert np.array_equal(U.power(v, nfft), U.power(v2, nfft))


def test_scale_closed_form_and_level():
    # constant (1, 0) samples: P = 1, s = 8 sqrt(2) / sqrt(N)
    nfft = 1024
    v = _bytes_from(np.ones((nfft, 1), int), np.zeros((nfft, 1), int))
    s = U.requant_scale(U.power(v, nfft), nfft, nfft)
    assert s[0] == pytest.approx(8 * math.sqrt(2) / math.sqrt(nfft), rel=1e-15)
    # Gaussian voltages requantise to about 8 levels rms per component
    cfg = synth.make_config("tiny", n_tones=0)
    vol = synth.generate(cfg)
    specs, ss, qs = U.upchan_all(vol, cfg.nfft)
    rms = np.sqrt((qs[0].astype(float) ** 2).mean())
    assert 7.7 < rms < 8.3


def test_requantize_rounding_and_clip():
    X = np.array([0.5, 1.5, 2.5, -0.5, -1.5, 300.0, -300.0, 126.5, -127.5]) + 0j
    q = U.requantize(X[None, None, :], np.ones(1))[0, 0, :, 0]
    assert q.tolist() == [0, 2, 2, 0, -2, 127, -127, 126, -127]
    # the FP32 decision multiplies in single precision: with s = 0.7, x = 45 the FP32
    # product is exactly 31.5 (rint -> 32, half to even) while FP64 gives
    # 31.499999999999996 (rint -> 31)
    x = np.array([45.0])
    q32 = U.requantize(x[None, None, :].astype(np.complex64), np.array([0.7]), np.float32)
    q64 = U.requantize(x[None, None, :].astype(np.complex128), np.array([0.7]), np.float64)
    assert np.float32(0.7) * np.float32(45.0) == np.float32(31.5)
    assert q32[0, 0, 0, 0] == 32 and q64[0, 0, 0, 0] == 31


def test_paper_channel_widths():
    # Section 2.1: 23.9 kHz / 2400 -> ~9.9 Hz; / 32 -> ~750 Hz; 300 channels ~ 3 kHz;
    # Abstract / Section 2.2: > 3e6 images over 50-86 MHz
    g = json.load(open(os.path.join(GOLD, "paper_numbers.json")))
    df = g["coarse_channel_hz"] / g["upchan_factor_search"]
    assert abs(df - g["fine_channel_hz_search"]) < 0.1
    assert abs(g["coarse_channel_hz"] / g["upchan_factor_gw"] - g["fine_channel_hz_gw"]) < 5
    assert abs(g["fine_channels_per_batch"] * df - g["batch_bandwidth_hz"]) < 50
    n_img = (g["band_hi_hz"] - g["band_lo_hz"]) / df
    assert n_img > g["images_per_epoch_at_least"]
    # the same rule the fine-channel axis uses: channel k' at nu_c + (k' - N/2) f_c / N
    f = synth.fine_freqs_hz([2400])
    assert f[1] - f[0] == pytest.approx(24_000.0 / 2400, rel=1e-9)
    assert f[1200] == synth.coarse_centre_hz(0)


# ---------------------------------------------------------------- N = 2400 and other 3,5-smooth N
def _direct_dft(z):
    """X_k = sum_n z_n exp(-2 pi i k n / N) as a matrix product, the phase taken
    from the exact integer (k n) mod N."""
    n = z.shape[0]
    kn = np.outer(np.arange(n), np.arange(n)) % n
    return np.exp(-2j * np.pi * kn / n) @ z


@pytest.mark.parametrize("nfft", [6, 10, 12, 30, 60, 96, 360, 2400])
def test_mixed_radix_matches_direct_dft(nfft):
    # the library FFT of a 2^a 3^b 5^c length against the DFT summed directly
    g = np.random.default_rng(nfft)
    re = g.integers(-8, 8, (2 * nfft + 3, 2))
    im = g.integers(-8, 8, (2 * nfft + 3, 2))
    X = U.upchannelize(_bytes_from(re, im), nfft)                       # [N][in][K]
    z = (re + 1j * im)[: 2 * nfft].reshape(2, nfft, 2)
    for s in range(2):
        for i in range(2):
            d = np.fft.fftshift(_direct_dft(z[s, :, i]))
            assert np.max(np.abs(X[:, i, s] - d)) < 1e-9 * nfft * 8


@pytest.mark.parametrize("nfft", [12, 2400])
@pytest.mark.parametrize("quarter", [0, 1, 3])
def test_2400_pure_tone(nfft, quarter):
    a, b = -7, 2
    v = _rotating_tone(2 * nfft, 1, quarter, a, b)
    X = U.upchannelize(v, nfft)
    kp = (quarter * nfft // 4 + nfft // 2) % nfft
    assert abs(X[kp, 0, 0] - nfft * (a + 1j * b)) < 1e-9 * nfft
    assert np.delete(np.abs(X[:, 0, :]), kp, axis=0).max() < 1e-9 * nfft


def test_2400_parseval():
    g = np.random.default_rng(7)
    nfft, k = 2400, 2
    re = g.integers(-8, 8, (k * nfft, 3))
    im = g.integers(-8, 8, (k * nfft, 3))
    X = U.upchannelize(_bytes_from(re, im), nfft)
    lhs = (np.abs(X) ** 2).sum(axis=0)
    rhs = nfft * (re ** 2 + im ** 2).reshape(k, nfft, 3).sum(axis=1).T
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=0)


# ---------------------------------------------------------------- polyphase filter bank option
def test_pfb_one_tap_of_ones_is_the_block_fft():
    g = np.random.default_rng(8)
    nfft = 60
    v = g.integers(0, 256, (5 * nfft + 11, 3), dtype=np.uint8)
    assert np.array_equal(U.pfb_upchannelize(v, nfft, np.ones(nfft)), U.upchannelize(v, nfft))


@pytest.mark.parametrize("nfft,n_tap", [(12, 3), (2400, 4)])
def test_pfb_constant_taps_on_a_tone(nfft, n_tap):
    # N a multiple of 4: every block of i^n (a + ib) is the same, so constant taps c
    # give X = c P N (a + ib) in the tone's channel and nothing elsewhere
    a, b, c = 4, -3, 0.375
    blocks = n_tap + 2
    v = _rotating_tone(blocks * nfft + 5, 1, 1, a, b)
    X = U.pfb_upchannelize(v, nfft, np.full(n_tap * nfft, c))
    assert X.shape == (nfft, 1, blocks - n_tap + 1)
    kp = (nfft // 4 + nfft // 2) % nfft
    assert np.allclose(X[kp, 0, :], c * n_tap * nfft * (a + 1j * b), rtol=1e-12)
    assert np.delete(np.abs(X[:, 0, :]), kp, axis=0).max() < 1e-9 * nfft


def test_pfb_impulse_response():
    # one non-zero sample at block b0, offset n0: spectrum s sees it through tap
    # p = b0 - s (if 0 <= p < P) with weight h[p][n0], so |X_k| = |h[p][n0]| |x| for all k
    nfft, n_tap, blocks = 30, 3, 6
    h = np.random.default_rng(9).normal(size=n_tap * nfft)
    re = np.zeros((blocks * nfft, 1), int)
    im = np.zeros((blocks * nfft, 1), int)
    b0, n0 = 3, 17
    re[b0 * nfft + n0, 0], im[b0 * nfft + n0, 0] = -6, 5
    X = U.pfb_upchannelize(_bytes_from(re, im), nfft, h)
    for s in range(blocks - n_tap + 1):
        p = b0 - s
        w = abs(h[p * nfft + n0]) if 0 <= p < n_tap else 0.0
        assert np.allclose(np.abs(X[:, 0, s]), w * math.hypot(6, 5), rtol=1e-12, atol=1e-12)
        if w:
            # phase: exp(-2 pi i k n0 / N) times sign(h) (-6 + 5i), k the unshifted bin
            k = (np.arange(nfft) - nfft // 2) % nfft
            ref = h[p * nfft + n0] * (-6 + 5j) * np.exp(-2j * np.pi * k * n0 / nfft)
            assert np.allclose(X[:, 0, s], ref, atol=1e-12)


def test_pfb_brute_force_small():
    # N = 6, P = 2 written out as sums over taps and samples, no FFT
    g = np.random.default_rng(10)
    nfft, n_tap = 6, 2
    re = g.integers(-8, 8, (4 * nfft, 2))
    im = g.integers(-8, 8, (4 * nfft, 2))
    h = g.normal(size=n_tap * nfft)
    X = U.pfb_upchannelize(_bytes_from(re, im), nfft, h)
    z = re + 1j * im
    for s in range(3):
        for i in range(2):
            for kp in range(nfft):
                k = (kp - nfft // 2) % nfft
                acc = 0j
                for n in range(nfft):
                    y = sum(h[p * nfft + n] * z[(s + p) * nfft + n, i] for p in range(n_tap))
                    acc += y * complex(math.cos(2 * math.pi * k * n / nfft), -math.sin(2 * math.pi * k * n / nfft))
                assert abs(X[kp, i, s] - acc) < 1e-10


def test_pfb_scale_and_level():
    # constant (1, 0) samples: mean power 1, s = 8 sqrt(2) / sqrt(sum h^2)
    nfft, n_tap = 2400, 4
    h = synth.pfb_prototype(nfft, n_tap).astype(np.float64)
    v = _bytes_from(np.ones((6 * nfft, 1), int), np.zeros((6 * nfft, 1), int))
    _, ss, _ = U.upchan_all(v[None], [nfft], taps=[h])
    assert ss[0][0] == pytest.approx(8 * math.sqrt(2) / math.sqrt((h * h).sum()), rel=1e-15)
    # white Gaussian voltages through the prototype requantise to ~8 levels rms
    cfg = synth.make_config("tiny", n_tones=0)
    vol = synth.generate(cfg)[:, :, :8]
    hp = [synth.pfb_prototype(n, 4) for n in cfg.nfft]
    specs, _, qs = U.upchan_all(vol, cfg.nfft, taps=hp)
    assert specs[0].shape[2] == cfg.n_time // cfg.nfft[0] - 3
    rms = np.sqrt((qs[0].astype(float) ** 2).mean())
    assert 7.6 < rms < 8.4


def test_pfb_too_few_blocks_gives_no_spectra():
    v = np.zeros((3 * 12, 2), np.uint8)
    assert U.pfb_upchannelize(v, 12, np.ones(4 * 12)).shape == (12, 2, 0)


def test_channel_window_is_a_slice():
    g = np.random.default_rng(11)
    v = g.integers(0, 256, (2, 2 * 2400, 4), dtype=np.uint8)
    full = U.upchan_all(v, [2400, 2400])
    win = U.upchan_all(v, [2400, 2400], window=(900, 300))
    for c in range(2):
        assert np.array_equal(win[0][c], full[0][c][900:1200])
        assert np.array_equal(win[1][c], full[1][c])
        assert np.array_equal(win[2][c], full[2][c][900:1200])
