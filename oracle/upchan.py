"""Oracle: unpack + FFT upchannelizer + 8-bit requantisation (Section 2.1).

The paper upchannelizes "by applying a fast Fourier transform to the time
samples within each coarse channel" (Section 2.1).  Readings where it is
silent: non-overlapping blocks of N samples, rectangular window, unnormalised
forward transform X_k = sum_n x_n exp(-2 pi i k n / N), fftshift so fine
channel k' = (k + N/2) mod N runs upward in frequency; leftover samples after
K = floor(n_time / N) blocks are dropped.

The correlator takes 8-bit complex input (xGPU, Section 2.1), so spectra are
requantised: q = clamp(rint(s X), -127, 127) per component, with one scale per
(coarse channel, input) s = 8 sqrt(2) / sqrt(N P), P the mean sample power
(an exact integer sum divided by the number of samples used).
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


def requant_scale(pwr: np.ndarray, nfft: int, n_used: int) -> np.ndarray:
    """s = 8 sqrt(2) / sqrt(N * P), P = pwr / n_used, in FP64; s = 0 where P = 0."""
    pbar = pwr.astype(np.float64) / float(n_used)
    s = np.zeros_like(pbar)
    nz = pbar > 0
    s[nz] = (8.0 * np.sqrt(2.0)) / np.sqrt(float(nfft) * pbar[nz])
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


def upchan_all(volt: np.ndarray, nfft_list, scales=None):
    """Whole upchannelizer for [n_coarse][n_time][n_input] voltages.

    Returns (spectra per coarse channel, scales per coarse channel, int8 per
    coarse channel) with the layouts of ``upchannelize`` and ``requantize``.
    """
    specs, ss, qs = [], [], []
    for c, n in enumerate(nfft_list):
        X = upchannelize(volt[c], n)
        if scales is None:
            s = requant_scale(power(volt[c], n), n, X.shape[2] * n)
        else:
            s = np.asarray(scales[c], dtype=np.float64)
        specs.append(X)
        ss.append(s)
        qs.append(requantize(X, s))
    return specs, ss, qs
