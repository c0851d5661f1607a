"""Oracle: X-engine cross-correlation in exact int64 (Section 2.1).

Per fine channel the correlator forms, for every antenna pair and every
polarisation product, the integrated product of the 8-bit fine-channel
voltages (the xGPU correlation of Section 2.1):

    V_{ij}^{pq} = sum_{s < K} q_{ip}(s) conj(q_{jq}(s)),   i <= j (autos kept)

Inputs are numbered input = 2 * antenna + pol.  Output layout
[channel][baseline][pol product][re, im], baseline index of (a, b), a <= b,
row-major over the upper triangle: bl = a n - a (a - 1) / 2 + (b - a);
pol product p = 2 * p_a + p_b (XX, XY, YX, YY).
"""
from __future__ import annotations

import numpy as np


def n_baselines(n_ant: int) -> int:
    return n_ant * (n_ant + 1) // 2


def baseline_index(a: int, b: int, n_ant: int) -> int:
    return a * n_ant - a * (a - 1) // 2 + (b - a)


def baseline_pairs(n_ant: int):
    """(a, b) arrays for every baseline index, a <= b."""
    a, b = np.triu_indices(n_ant)
    return a, b


def full_matrix(q: np.ndarray):
    """Full Hermitian correlation matrix of one channel, int64.

    q: int8 [n_input][K][2].  Returns (Re, Im) int64 [n_input][n_input] with
    V[i, j] = sum_s q_i(s) conj(q_j(s)).
    """
    r = q[..., 0].astype(np.int64)
    m = q[..., 1].astype(np.int64)
    vre = r @ r.T + m @ m.T
    vim = m @ r.T - r @ m.T
    return vre, vim


def pack(vre: np.ndarray, vim: np.ndarray, n_ant: int) -> np.ndarray:
    """Full input-by-input matrix -> [baseline][pol product][2] int64."""
    a, b = baseline_pairs(n_ant)
    out = np.empty((a.size, 4, 2), dtype=np.int64)
    for pa in range(2):
        for pb in range(2):
            i = 2 * a + pa
            j = 2 * b + pb
            out[:, 2 * pa + pb, 0] = vre[i, j]
            out[:, 2 * pa + pb, 1] = vim[i, j]
    return out


def correlate(q: np.ndarray, n_ant: int, channels=None) -> np.ndarray:
    """q: int8 [n_chan][n_input][K][2] -> int64 [n_sel][n_bl][4][2]."""
    chans = range(q.shape[0]) if channels is None else channels
    out = [pack(*full_matrix(q[c]), n_ant) for c in chans]
    return np.stack(out) if out else np.zeros((0, n_baselines(n_ant), 4, 2), np.int64)
