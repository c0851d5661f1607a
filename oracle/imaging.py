"""Oracle: FP64 uvw, prolate-spheroidal gridding and dirty imaging (Section 2.2).

The paper images every fine channel over the visible hemisphere on a
512 x 512 grid with 0.25 degree pixels (Section 2.2, WSClean, dirty images
are the search product).  Readings where the paper is silent:

* Stokes I = (XX + YY) / 2, autocorrelations excluded, natural weights.
* The uv grid is padded by 2, as imagers such as WSClean pad theirs: it has
  G = 2N cells a side, du = 1 / (G * cell), and the image is the central
  N x N of the G x G transform.  Without padding the horizon of an all-sky
  image sits where the kernel's transform has fallen to ~2e-4, and dividing
  by it amplifies round-off and aliasing there by ~5000.
* uv in grid cells: u = (x_a - x_b) * s_nu with s_nu = nu / (c * du); one
  FP64 multiply per coordinate.  Zenith phase centre with a planar array, so
  w = 0.
* Each visibility V at (u, v) and its mirror conj(V) at (-u, -v) is
  convolved onto the grid with a separable 7 x 7 prolate-spheroidal kernel
  C(x) = psi_0(c, x / 3.5) / psi_0(c, 0), c = 7 pi / 2, tabulated at Q = 1024
  samples per cell.  The position is rounded to the table once:
  p = rint(u Q); centre cell c0 = p / Q rounded half away from zero (so a
  visibility at -p has centre -c0 and its footprint is the exact point
  reflection); the tap at cell c0 + t takes table sample t Q - (p - c0 Q).
* A baseline whose footprint (or its mirror's) leaves the G x G grid is
  dropped and counted.
* Image I(r, c) = Re sum_grid G exp(+2 pi i (u l + v m)) / (sum w * C^(r) C^(c)),
  with pixel (r, c) <-> l = (c - N/2) cell, m = (r - N/2) cell and grid
  correction C^(d) = (1/Q) sum_m C(m/Q) cos(2 pi m d / (Q G)), the Fourier
  transform of the tabulated kernel.  sum w counts gridded visibilities,
  mirrors included.  Pixels with l^2 + m^2 >= 1 (below the horizon) are 0.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import legendre as npleg

C_LIGHT = 299_792_458.0
PAD = 2
SUPPORT = 7
OVERSAMPLE = 1024
PSWF_C = math.pi * SUPPORT / 2.0


# --------------------------------------------------------------------------------------
# Prolate spheroidal wave function psi_0(c, eta), Legendre-series eigenproblem
# (Bouwkamp's method): L psi = chi psi with L = -d/de (1 - e^2) d/de + c^2 e^2,
# psi = sum_k d_k P_k(e) over even k; psi_0 is the eigenvector of smallest chi.
# --------------------------------------------------------------------------------------
def pswf_legendre_coeffs(c: float = PSWF_C, n_terms: int = 60) -> np.ndarray:
    ks = np.arange(0, 2 * n_terms, 2, dtype=np.float64)
    M = np.zeros((n_terms, n_terms))
    for j, k in enumerate(ks):
        beta = (2 * k * k + 2 * k - 1) / ((2 * k - 1) * (2 * k + 3))
        M[j, j] = k * (k + 1) + c * c * beta
        if j + 1 < n_terms:                      # coefficient of P_k from d_{k+2} P_{k+2}
            k2 = k + 2
            M[j, j + 1] = c * c * k2 * (k2 - 1) / ((2 * k2 - 1) * (2 * k2 + 1))
        if j >= 1:                               # coefficient of P_k from d_{k-2} P_{k-2}
            km = k - 2
            M[j, j - 1] = c * c * (km + 1) * (km + 2) / ((2 * km + 1) * (2 * km + 3))
    w, v = np.linalg.eig(M)
    i = int(np.argmin(w.real))
    d = v[:, i].real
    full = np.zeros(2 * n_terms)
    full[0::2] = d
    if npleg.legval(0.0, full) < 0:
        full = -full
    return full


def pswf_psi0(eta, c: float = PSWF_C) -> np.ndarray:
    """psi_0(c, eta) normalised to psi_0(c, 0) = 1."""
    coef = pswf_legendre_coeffs(c)
    return npleg.legval(np.asarray(eta, dtype=np.float64), coef) / npleg.legval(0.0, coef)


def kernel_table(support: int = SUPPORT, q: int = OVERSAMPLE, c: float = PSWF_C) -> np.ndarray:
    """C(m / Q) for m = -support Q / 2 .. +support Q / 2 (support * Q + 1 samples)."""
    half = support * q // 2
    m = np.arange(-half, half + 1, dtype=np.float64)
    return pswf_psi0(m / q / (support / 2.0), c)


def grid_correction(table: np.ndarray, n: int, q: int = OVERSAMPLE, g: int = 0) -> np.ndarray:
    """C^(d) for pixel offsets d = -N/2 .. N/2 - 1 on a G-cell grid (default G = PAD N)."""
    g = g or PAD * n
    half = (table.size - 1) // 2
    m = np.arange(-half, half + 1, dtype=np.float64)
    d = np.arange(-n // 2, n // 2, dtype=np.float64)
    return (table[None, :] * np.cos(2 * np.pi * np.outer(d, m) / (q * g))).sum(axis=1) / q


# --------------------------------------------------------------------------------------
# uvw and gridding
# --------------------------------------------------------------------------------------
def cells_per_metre(nu_hz, g: int, cell: float):
    """s_nu = nu / (c * du), du = 1 / (G cell): grid cells per metre of baseline."""
    du = 1.0 / (g * cell)
    return np.asarray(nu_hz, dtype=np.float64) / (C_LIGHT * du)


def stokes_i(vis_chan: np.ndarray) -> np.ndarray:
    """(XX + YY) / 2 per baseline, complex128; vis_chan is [n_bl][4][2] int."""
    xx = vis_chan[:, 0, 0] + 1j * vis_chan[:, 0, 1]
    yy = vis_chan[:, 3, 0] + 1j * vis_chan[:, 3, 1]
    return (xx.astype(np.complex128) + yy) / 2.0


def _cross_pairs(n_ant: int):
    a, b = np.triu_indices(n_ant)
    keep = a != b
    idx = np.nonzero(keep)[0]
    return a[keep], b[keep], idx


def _taps(p: np.ndarray, n: int, q: int):
    """Centre cell, table offset and in-grid flag for rounded positions p (1/Q cells)."""
    c0 = np.sign(p) * ((np.abs(p) + q // 2) // q)
    off = p - c0 * q
    half = SUPPORT // 2
    inside = (n // 2 + c0 - half >= 0) & (n // 2 + c0 + half <= n - 1)
    return c0, off, inside


def uv_length_wavelengths(pos, a, b, nu_hz):
    """Baseline length in wavelengths, L * (nu / c) with L = sqrt(dx^2 + dy^2)
    (planar array, zenith phase centre)."""
    dx = pos[a, 0] - pos[b, 0]
    dy = pos[a, 1] - pos[b, 1]
    return np.sqrt(dx * dx + dy * dy) * (float(nu_hz) / C_LIGHT)


def grid_channel(vis_chan, pos, nu_hz, n, cell, table, q=OVERSAMPLE, gains_chan=None, uv_range=None):
    """FP64 uv grid G[kv][ku] (n = G cells a side) of one channel, plus the number
    of gridded visibilities (mirrors included) and of dropped baselines.

    gains_chan: optional complex [2 n_ant] corrections applied per polarisation
    before Stokes I; uv_range: optional (uv_min, uv_max) in wavelengths, keeping
    baselines with uv_min <= length < uv_max (the baseline cuts of the near-field
    test, Section 2.5.1); baselines outside it are dropped like baselines off the grid."""
    n_ant = pos.shape[0]
    a, b, idx = _cross_pairs(n_ant)
    if gains_chan is None:
        vi = stokes_i(vis_chan)[idx]
    else:
        g = np.asarray(gains_chan, dtype=np.complex128)
        xx = vis_chan[idx, 0, 0] + 1j * vis_chan[idx, 0, 1].astype(np.float64)
        yy = vis_chan[idx, 3, 0] + 1j * vis_chan[idx, 3, 1].astype(np.float64)
        vi = (g[2 * a] * np.conj(g[2 * b]) * xx + g[2 * a + 1] * np.conj(g[2 * b + 1]) * yy) / 2.0
    s = cells_per_metre(nu_hz, n, cell)
    u = (pos[a, 0] - pos[b, 0]) * s
    v = (pos[a, 1] - pos[b, 1]) * s
    pu = np.rint(u * q).astype(np.int64)
    pv = np.rint(v * q).astype(np.int64)
    keep = np.ones(a.size, dtype=bool)
    if uv_range is not None:
        lam = uv_length_wavelengths(pos, a, b, nu_hz)
        lo, hi = uv_range
        keep &= (lam >= lo) & (lam < hi)
    sides = []
    for sign in (1, -1):
        cu, ou, iu = _taps(sign * pu, n, q)
        cv, ov, iv = _taps(sign * pv, n, q)
        keep &= iu & iv
        sides.append((sign, cu, ou, cv, ov))
    G = np.zeros((n, n), dtype=np.complex128)
    half_tab = (table.size - 1) // 2
    half = SUPPORT // 2
    for sign, cu, ou, cv, ov in sides:
        val = vi if sign > 0 else np.conj(vi)
        cu, ou, cv, ov, val = cu[keep], ou[keep], cv[keep], ov[keep], val[keep]
        for tv in range(-half, half + 1):
            wv = table[half_tab + tv * q - ov]
            kv = n // 2 + cv + tv
            for tu in range(-half, half + 1):
                wu = table[half_tab + tu * q - ou]
                ku = n // 2 + cu + tu
                np.add.at(G, (kv, ku), wv * wu * val)
    n_grid = 2 * int(keep.sum())
    return G, n_grid, int((~keep).sum())


def horizon_mask(n: int, cell: float) -> np.ndarray:
    """True for pixels above the horizon, l^2 + m^2 < 1."""
    d = (np.arange(n) - n // 2) * cell
    return (d[None, :] ** 2 + d[:, None] ** 2) < 1.0


def image_from_grid(G, n_grid, n, cell, corr):
    """Dirty N x N image from an FP64 G x G grid: exp(+) transform with centred
    axes, central N x N kept."""
    g = G.shape[0]
    raw = np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(G))) * (g * g)
    o = g // 2 - n // 2
    img = raw[o:o + n, o:o + n].real / (max(n_grid, 1) * np.outer(corr, corr))
    img[~horizon_mask(n, cell)] = 0.0
    return img


def dirty_images(vis, pos, freqs_hz, n, cell, channels=None, gains=None, uv_range=None):
    """vis: [n_chan][n_bl][4][2] int -> FP64 images [n_sel][N][N] and stats.
    gains: optional complex [n_chan][2 n_ant] corrections; uv_range: optional
    (uv_min, uv_max) in wavelengths (see grid_channel)."""
    table = kernel_table()
    corr = grid_correction(table, n)
    chans = range(vis.shape[0]) if channels is None else channels
    imgs, ngrid, ndrop = [], [], []
    for c in chans:
        G, ng, nd = grid_channel(vis[c], pos, freqs_hz[c], PAD * n, cell, table,
                                 gains_chan=None if gains is None else gains[c], uv_range=uv_range)
        imgs.append(image_from_grid(G, ng, n, cell, corr))
        ngrid.append(ng)
        ndrop.append(nd)
    return np.stack(imgs), np.array(ngrid), np.array(ndrop)


def dft_image(vis_chan, pos, nu_hz, n, cell, baselines=None):
    """Direct (ungridded) dirty image: sum_b 2 Re[V_b exp(+2 pi i (u l + v m))] / sum w.

    u, v in wavelengths.  ``baselines`` selects cross baselines by their index
    among the cross pairs (default all).
    """
    a, b, idx = _cross_pairs(pos.shape[0])
    vi = stokes_i(vis_chan)[idx]
    if baselines is not None:
        a, b, vi = a[baselines], b[baselines], vi[baselines]
    lam = C_LIGHT / nu_hz
    u = (pos[a, 0] - pos[b, 0]) / lam
    v = (pos[a, 1] - pos[b, 1]) / lam
    d = (np.arange(n) - n // 2) * cell
    ph_l = np.exp(2j * np.pi * np.outer(u, d))     # [bl][col]
    ph_m = np.exp(2j * np.pi * np.outer(v, d))     # [bl][row]
    img = 2.0 * np.einsum("b,br,bc->rc", vi, ph_m, ph_l).real / max(2 * vi.size, 1)
    img[~horizon_mask(n, cell)] = 0.0
    return img
