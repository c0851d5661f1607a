"""Oracle: drift-rate search over sub-integration images, FP64.

Test infrastructure only: the product path never imports this module.

The paper's search applies no drift correction and names a drift search as
future work (Section 2.3.4, Doppler drift, and Section 4: drifts of up to
tens of Hz over 30 s for transmitters on close-in planets).  The readings here:

1. Sub-integrations: the K spectra of an integration are split into
   T = 2^k equal consecutive chunks (K_t = floor(K / T) spectra each; the
   leftover spectra are dropped).  Each chunk is correlated and imaged on
   its own and run through Stage I's standardisation and high-pass, giving
   z'_t[f][row][col] for t < T (unit-variance noise in every chunk).
2. Drift paths are the digital lines of the Taylor tree: over n = 2^j rows a
   path of total drift d in [0, n) is shift(d, 1, 0) = 0 and, for n > 1,
   shift(d, n, t) = shift(floor(d/2), n/2, t) for t < n/2 and
   ceil(d/2) + shift(floor(d/2), n/2, t - n/2) otherwise.  Every path starts
   at shift 0 and ends at shift d and never steps by more than one channel.
3. For start channel f of a coarse channel [c_lo, c_hi), drift d >= 0 sums
   z'_t[f + shift(d, T, t)] over t and drift -d sums z'_t[f - shift(d, T, t)];
   a sum counts only when its whole path lies inside the coarse channel
   (f + d < c_hi, resp. f - d >= c_lo).  SNR = sum / sqrt(T).
4. Per (pixel, channel) the search keeps the largest SNR over the 2T - 1
   drifts, visited in the order 0, +1, -1, +2, -2, ...; a later drift
   replaces the kept one only when strictly larger.
5. Candidates: Benjamini-Hochberg on p = Q(SNR) over every in-horizon
   (pixel, channel), m = in-horizon pixels x channels (the maximum over drifts
   taken like Stage I's maximum over widths, with no correction for the
   trials), or a fixed threshold SNR >= n_sigma; then Stage I's greedy
   non-maximum suppression along frequency per pixel with the line's width
   in the integrated spectrum, |d| + 1 channels, as its width
   (half-width max(1, floor((|d| + 1) / 2))).
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np

from . import detect as OD


def shift(d: int, n: int, t: int) -> int:
    """Channel offset at row t of the Taylor path of total drift d over n rows."""
    if n == 1:
        return 0
    h = n // 2
    if t < h:
        return shift(d // 2, h, t)
    return (d - d // 2) + shift(d // 2, h, t - h)


@lru_cache(maxsize=None)
def shift_table(n: int) -> np.ndarray:
    """[d][t] offsets for d, t < n."""
    return np.array([[shift(d, n, t) for t in range(n)] for d in range(n)], dtype=np.int64)


def drift_order(n: int):
    """Signed drifts in visiting order: 0, +1, -1, ..., +(n-1), -(n-1)."""
    out = [0]
    for d in range(1, n):
        out += [d, -d]
    return out


def drift_sums(zsub: np.ndarray, c_lo: int, c_hi: int):
    """SNR[drift index][f][...] (NaN where the path leaves the coarse channel)
    for the coarse channel [c_lo, c_hi); zsub [T][n_chan][...]."""
    T = zsub.shape[0]
    tab = shift_table(T)
    order = drift_order(T)
    nc = c_hi - c_lo
    out = np.full((len(order), nc) + zsub.shape[2:], np.nan)
    for i, sd in enumerate(order):
        d = abs(sd)
        for f in range(c_lo, c_hi):
            end = f + d if sd >= 0 else f - d
            if not (c_lo <= end < c_hi):
                continue
            acc = np.zeros(zsub.shape[2:])
            for t in range(T):
                ch = f + tab[d, t] if sd >= 0 else f - tab[d, t]
                acc = acc + zsub[t, ch].astype(np.float64)
            out[i, f - c_lo] = acc / math.sqrt(T)
    return out, order


def drift_search(zsub: np.ndarray, mask: np.ndarray, nfft_list, n_sigma: float = 10.0, mode: str = "fixed",
                 alpha: float = 0.01):
    """(snr [n_chan][N][N], drift [n_chan][N][N], candidates, drifts).

    Pixels below the horizon hold snr = -inf, drift 0.  Candidates are
    oracle.detect.Candidate records whose width is |d| + 1, with the signed
    drift in a parallel list.
    """
    T, n_chan = zsub.shape[0], zsub.shape[1]
    snr = np.full((n_chan,) + zsub.shape[2:], -np.inf)
    dr = np.zeros((n_chan,) + zsub.shape[2:], np.int64)
    for lo, hi in OD.chan_bounds_of(nfft_list):
        s, order = drift_sums(zsub, lo, hi)
        best = np.full(s.shape[1:], -np.inf)
        bd = np.zeros(s.shape[1:], np.int64)
        for i, sd in enumerate(order):
            v = s[i]
            better = ~np.isnan(v) & (v > best)
            best[better] = v[better]
            bd[better] = sd
        snr[lo:hi] = best
        dr[lo:hi] = bd
    snr[:, ~mask] = -np.inf
    dr[:, ~mask] = 0
    sel = OD.select(snr, mask, mode, alpha, n_sigma)
    cands = OD.nms(sel, snr, np.abs(dr) + 1, OD.chan_bounds_of(nfft_list))
    drifts = [int(dr[c.chan, c.row, c.col]) for c in cands]
    return snr, dr, cands, drifts


def subint_bounds(n_spec: int, n_sub: int):
    """[(s0, count)] of the T chunks of K spectra."""
    k = n_spec // n_sub
    return [(t * k, k) for t in range(n_sub)]
