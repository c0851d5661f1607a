"""Oracle: unpack + FFT upchannelizer + 8-bit requantisation (Section 2.1).

Section 2.1 raises the spectral resolution with an FFT over the time samples
of each coarse channel.  Readings where it is silent: non-overlapping blocks of N samples, rectangular window, unnormalised
forward transform X_k = sum_n x_n exp(-2 pi i k n / N), fftshift so fine
channel k' = (k + N/2) mod N runs upward in frequency; leftover samples after
K = floor(n_time / N) blocks are dropped.

The correlator takes 8-bit complex input (xGPU, Section 2.1), so spectra are
requantised: q = clamp(rint(s X), -127, 127) per component, with one scale per
(coarse channel, input) s = 8 sqrt(2) / sqrt(N P), P the mean sample power
(an exact integer sum divided by the number of samples used).

N is any even length: the paper's search uses N = 2400 = 2^5 3 5^2 (Section
2.1); the FFT here is the library transform, which is a plain DFT of that
length.  Two further options of Section 2.1's upchannelizer:

* fine-channel batches: the paper cross-correlates 300 fine channels at a time;
  a window [lo, lo + count) of the fftshifted fine-channel axis selects one;
* a polyphase filter bank (the F-engine's channeliser, Section 2.1) in place
  of the bare block FFT: P taps h[p][n] (a prototype filter of P N
  coefficients, read row by row), y_n(s) = sum_p h[p][n] x[(s + p) N + n],
  X(s) = FFT(y(s)), K = floor(n_time / N) - P + 1 spectra.  P = 1, h = 1 is
  the plain FFT.  The requantisation scale becomes 8 sqrt(2) /
  sqrt(P_mean sum h^2), since E|X_k|^2 = P_mean sum_{p,n} h[p][n]^2 for white
  input; sum h^2 = N for the plain FFT.

Test infrastructure only: the product path never imports this module.
"""
from __future__ import annotations

import numpy as np


def unpack(volt: np.ndarray):
    """4+4-bit two's complement bytes -> (re, im) int64; re is the high nibble."""
    v = volt.astype(np.int64)
    hi = v >> 4
    lo = v & 0xF
    re = np.where(hi >= 8, hi - 16, hi)
    im = np.where(lo >= 8, lo - 16, lo)
    return re, im


def n_spectra(n_time: int, nfft: int) -> int:
    return n_time // nfft


def power(volt_coarse: np.ndarray, nfft: int) -> np.ndarray:
    """Exact int64 sum over the used samples of |x|^2, per input.  [n_input]"""
    k = n_spectra(volt_coarse.shape[0], nfft)
    re, im = unpack(volt_coarse[: k * nfft])
    return (re * re + im * im).sum(axis=0)


def requant_scale(pwr: np.ndarray, nfft: int, n_used: int, sum_h2=None) -> np.ndarray:
    """s = 8 sqrt(2) / sqrt(W * P), P = pwr / n_used, in FP64; s = 0 where P = 0.

    W = N for the plain FFT, W = sum of the squared filter taps for a PFB.
    """
    pbar = pwr.astype(np.float64) / float(n_used)
    w = float(nfft) if sum_h2 is None else float(sum_h2)
    s = np.zeros_like(pbar)
    nz = pbar > 0
    s[nz] = (8.0 * np.sqrt(2.0)) / np.sqrt(w * pbar[nz])
    return s


def upchannelize(volt_coarse: np.ndarray, nfft: int) -> np.ndarray:
    """FP64 fine-channel spectra of one coarse channel.

    volt_coarse: uint8 [n_time][n_input].  Returns complex128 [N][n_input][K]
    (fine channel, input, spectrum), fftshifted along the fine-channel axis.
    """
    k = n_spectra(volt_coarse.shape[0], nfft)
    re, im = unpack(volt_coarse[: k * nfft])
    x = (re + 1j * im).reshape(k, nfft, -1)              # [K][N][input]
    X = np.fft.fft(x, axis=1)                             # e^{-2 pi i k n / N}, unnormalised
    X = np.fft.fftshift(X, axes=1)
    return np.ascontiguousarray(X.transpose(1, 2, 0))     # [N][input][K]


def pfb_upchannelize(volt_coarse: np.ndarray, nfft: int, taps: np.ndarray) -> np.ndarray:
    """FP64 polyphase-filter-bank spectra of one coarse channel.

    taps: P N coefficients, h[p][n] = taps[p N + n].  Block b holds samples
    [b N, (b + 1) N); spectrum s weights blocks s .. s + P - 1:
    y_n(s) = sum_p h[p][n] x[(s + p) N + n], then the unnormalised FFT of y(s),
    fftshifted.  Returns complex128 [N][n_input][K], K = floor(n_time / N) - P + 1.
    """
    h = np.asarray(taps, dtype=np.float64).reshape(-1, nfft)          # [P][N]
    n_tap = h.shape[0]
    blocks = n_spectra(volt_coarse.shape[0], nfft)
    k = blocks - n_tap + 1
    n_input = volt_coarse.shape[1]
    if k <= 0:
        return np.zeros((nfft, n_input, 0), complex)
    re, im = unpack(volt_coarse[: blocks * nfft])
    x = (re + 1j * im).reshape(blocks, nfft, n_input)                   # [block][N][input]
    y = np.zeros((k, nfft, n_input), complex)
    for p in range(n_tap):
        y += h[p][None, :, None] * x[p:p + k]
    X = np.fft.fftshift(np.fft.fft(y, axis=1), axes=1)
    return np.ascontiguousarray(X.transpose(1, 2, 0))


def requantize(X: np.ndarray, s: np.ndarray, precision=np.float64):
    """q = clamp(rint(s X), -127, 127), round half to even, per component.

    ``precision`` is the arithmetic the rounding decision is taken in:
    float64 for the oracle's own spectra, float32 to requantise FP32 spectra
    exactly as a single-precision kernel does (s rounded to FP32, one FP32
    multiply, rint).  Returns int8 [..., 2] with (re, im) pairs.
    """
    sc = np.asarray(s, dtype=np.float64).astype(precision)[None, :, None]
    re = np.asarray(X.real).astype(precision)
    im = np.asarray(X.imag).astype(precision)
    qr = np.clip(np.rint(re * sc), -127, 127)
    qi = np.clip(np.rint(im * sc), -127, 127)
    return np.stack([qr, qi], axis=-1).astype(np.int8)


def upchan_all(volt: np.ndarray, nfft_list, scales=None, taps=None, window=None):
    """Whole upchannelizer for [n_coarse][n_time][n_input] voltages.

    taps: None (plain FFT) or one PFB coefficient array per coarse channel.
    window: None or (lo, count), the fftshifted fine channels kept.
    Returns (spectra per coarse channel, scales per coarse channel, int8 per
    coarse channel) with the layouts of ``upchannelize`` and ``requantize``.
    The scale uses the power of every whole block, floor(n_time / N) N samples.
    """
    specs, ss, qs = [], [], []
    for c, n in enumerate(nfft_list):
        blocks = n_spectra(volt[c].shape[0], n)
        if taps is None:
            X = upchannelize(volt[c], n)
            h2 = None
        else:
            h = np.asarray(taps[c], dtype=np.float64)
            X = pfb_upchannelize(volt[c], n, h)
            h2 = float((h * h).sum())
        if scales is None:
            s = requant_scale(power(volt[c], n), n, blocks * n, h2)
        else:
            s = np.asarray(scales[c], dtype=np.float64)
        if window is not None:
            lo, cnt = window
            X = X[lo:lo + cnt]
        specs.append(X)
        ss.append(s)
        qs.append(requantize(X, s))
    return specs, ss, qs
