"""Pins for the imaging oracle (Section 2.2): the PSWF kernel against scipy and
its integral eigen-relation, grid correction against the closed form, a point
source at a pixel centre, and brute-force DFT imaging on tiny arrays."""
import math

import numpy as np
import pytest
from scipy.special import pro_ang1

import synth
from oracle import imaging as I
from oracle import xengine as X


def test_pswf_matches_scipy():
    eta = np.linspace(-0.999, 0.999, 41)      # scipy's pro_ang1 returns nan at |eta| = 1
    ref = np.array([pro_ang1(0, 0, I.PSWF_C, e)[0] for e in eta]) / pro_ang1(0, 0, I.PSWF_C, 0.0)[0]
    assert np.max(np.abs(I.pswf_psi0(eta) - ref)) < 1e-10


def _lambda0():
    x, w = np.polynomial.legendre.leggauss(200)
    return float(np.sum(w * I.pswf_psi0(x)))      # integral of psi_0 = lambda_0 psi_0(0)


def test_pswf_eigen_relation():
    # int_{-1}^{1} psi_0(x) exp(i c x eta) dx = lambda_0 psi_0(eta)
    x, w = np.polynomial.legendre.leggauss(200)
    psi = I.pswf_psi0(x)
    lam = _lambda0()
    for eta in np.linspace(-1, 1, 11):
        lhs = np.sum(w * psi * np.exp(1j * I.PSWF_C * x * eta))
        assert abs(lhs - lam * I.pswf_psi0(eta)) < 1e-12


def test_kernel_table_shape_and_symmetry():
    t = I.kernel_table()
    assert t.size == I.SUPPORT * I.OVERSAMPLE + 1
    assert t[t.size // 2] == 1.0 and np.allclose(t, t[::-1], atol=1e-15)
    assert t.min() > 0 and np.all(np.diff(t[: t.size // 2 + 1]) > 0)


@pytest.mark.parametrize("n", [64, 256, 1024])
def test_grid_correction_closed_form(n):
    # FT of C(x) = psi_0(x / 3.5) over [-3.5, 3.5] at frequency d / G is
    # 3.5 lambda_0 psi_0(2 d / G); the tabulated sum matches to the Riemann-sum error
    for g in (n, 2 * n):
        corr = I.grid_correction(I.kernel_table(), n, g=g)
        d = np.arange(-n // 2, n // 2)
        ref = 3.5 * _lambda0() * I.pswf_psi0(2 * d / g)
        assert np.max(np.abs(corr - ref)) < 1e-6


def test_uv_cells_closed_form():
    # a baseline of B metres at wavelength lam spans B / lam wavelengths = (B / lam) N cell cells
    nu = 60e6
    lam = I.C_LIGHT / nu
    g, cell = 512, 2.0 / 256
    s = I.cells_per_metre(nu, g, cell)
    assert 123.0 * s == pytest.approx(123.0 / lam * g * cell, rel=1e-14)


def _point_source_vis(pos, nu, l0, m0):
    """Noise-free unit point source: V_ab = exp(-2 pi i (u l0 + v m0)), XX = YY."""
    n_ant = pos.shape[0]
    a, b = X.baseline_pairs(n_ant)
    lam = I.C_LIGHT / nu
    ph = -2 * np.pi * ((pos[a, 0] - pos[b, 0]) * l0 + (pos[a, 1] - pos[b, 1]) * m0) / lam
    v = np.exp(1j * ph)
    vis = np.zeros((a.size, 4, 2))
    for p in (0, 3):
        vis[:, p, 0], vis[:, p, 1] = v.real, v.imag
    return vis


def _small_array(n_ant=12, radius=60.0, seed=3):
    cfg = synth.Config("t", n_ant, 1, [8], 8, 64, seed, core_radius_m=radius)
    return synth.antenna_positions(cfg)


@pytest.mark.parametrize("n,cell", [(64, 0.02), (64, 2.0 / 64)])
def test_point_source_peak_at_pixel(n, cell):
    pos = _small_array()
    nu = 60e6
    r0, c0 = n // 2 + 5, n // 2 - 9
    l0, m0 = (c0 - n // 2) * cell, (r0 - n // 2) * cell
    vis = _point_source_vis(pos, nu, l0, m0)
    img, ng, nd = I.dirty_images(vis[None], pos, np.array([nu]), n, cell)
    img = img[0]
    assert np.unravel_index(np.argmax(img), img.shape) == (r0, c0)
    assert ng[0] > 0
    assert abs(img[r0, c0] - 1.0) < 2e-3


def test_gridded_matches_direct_dft():
    # brute-force DFT imaging of the same (kept) baselines agrees with the
    # gridded image to the kernel's aliasing level inside |l|, |m| < 0.5 of the field
    pos = _small_array(10, 50.0, 9)
    n, cell, nu = 64, 0.02, 60e6
    g = np.random.default_rng(4)
    nbl = X.n_baselines(pos.shape[0])
    vis = g.normal(size=(nbl, 4, 2)) * 100
    img, ng, nd = I.dirty_images(vis[None], pos, np.array([nu]), n, cell)
    assert nd[0] == 0
    ref = I.dft_image(vis, pos, nu, n, cell)
    # with the 2x padded grid the kernel's aliasing stays small over the whole image
    err = np.max(np.abs(img[0] - ref))
    assert err < 1e-3 * np.max(np.abs(ref))


def test_hermitian_grid_gives_real_image():
    pos = _small_array()
    n, cell, nu = 32, 0.03, 60e6
    vis = np.random.default_rng(8).normal(size=(X.n_baselines(pos.shape[0]), 4, 2))
    G, ng, nd = I.grid_channel(vis, pos, nu, n, cell, I.kernel_table())
    # with the mirror at (-u, -v) the grid is Hermitian about the centre cell
    flip = np.roll(G[::-1, ::-1], 1, axis=(0, 1))
    assert np.allclose(G, np.conj(flip), atol=1e-12)
    raw = np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(G)))
    assert np.max(np.abs(raw.imag)) < 1e-12 * np.max(np.abs(raw.real))


def test_mirror_footprint_is_point_reflection():
    # centre cells round half away from zero, so the tap set of -p is the reflection
    # of the tap set of p, ties (p = Q/2 mod Q) included
    q, n = I.OVERSAMPLE, 64
    p = np.array([0, 1, q // 2, -q // 2, 3 * q // 2, 5 * q + q // 2, 7 * q - 3, -(9 * q + q // 2)])
    c0, off, _ = I._taps(p, n, q)
    c1, off1, _ = I._taps(-p, n, q)
    assert np.array_equal(c1, -c0) and np.array_equal(off1, -off)
    assert np.all(np.abs(off) <= q // 2)


def test_baselines_off_grid_are_dropped():
    # an east-west pair whose footprint just fits / just does not fit a G = 32 grid
    n, cell, nu = 32, 2.0 / 32, 60e6
    s = I.cells_per_metre(nu, n, cell)
    limit = (n // 2 - 4 + 0.49) / s        # centre cell G/2 - 4 from the middle: taps reach cell 1
    for dx, kept in ((limit * 0.98, True), ((n // 2 - 2) / s, False)):
        pos = np.array([[0.0, 0, 0], [dx, 0, 0]])
        vis = np.ones((3, 4, 2))
        G, ng, nd = I.grid_channel(vis, pos, nu, n, cell, I.kernel_table())
        assert (ng == 2) == kept and (nd == 0) == kept


def test_horizon_mask():
    m = I.horizon_mask(64, 2.0 / 64)
    assert m[32, 32] and not m[0, 0] and not m[32, 0]
    assert abs(m.sum() / 64 ** 2 - math.pi / 4) < 0.02


# ---- calibration corrections and uv-range selection (Sections 2.2, 2.5.1)
def _rand_vis(g, pos, n_chan=1, scale=100.0):
    return g.normal(size=(n_chan, X.n_baselines(pos.shape[0]), 4, 2)) * scale


def test_unit_gains_and_open_uv_range_change_nothing():
    pos = _small_array(10, 50.0, 9)
    n, cell, nu = 64, 0.02, np.array([60e6])
    vis = _rand_vis(np.random.default_rng(1), pos)
    ref, ng, nd = I.dirty_images(vis, pos, nu, n, cell)
    ones = np.ones((1, 2 * pos.shape[0]), np.complex128)
    got, ng2, nd2 = I.dirty_images(vis, pos, nu, n, cell, gains=ones, uv_range=(0.0, np.inf))
    assert np.array_equal(got, ref) and np.array_equal(ng, ng2) and np.array_equal(nd, nd2)


def test_common_gain_scales_image_by_its_power():
    # V' = g conj(g) V = |g|^2 V for every baseline
    pos = _small_array(10, 50.0, 9)
    n, cell, nu = 64, 0.02, np.array([60e6])
    vis = _rand_vis(np.random.default_rng(2), pos)
    gval = 0.6 - 1.3j
    ref, _, _ = I.dirty_images(vis, pos, nu, n, cell)
    got, _, _ = I.dirty_images(vis, pos, nu, n, cell, gains=np.full((1, 2 * pos.shape[0]), gval))
    assert np.allclose(got, abs(gval) ** 2 * ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_gains_act_per_polarisation():
    # corrections of 2 on every X input and 1 on every Y input: I' = (4 XX + YY) / 2,
    # the image of the visibilities with XX scaled by 4
    pos = _small_array(10, 50.0, 9)
    n, cell, nu = 64, 0.02, np.array([60e6])
    vis = _rand_vis(np.random.default_rng(3), pos)
    gains = np.ones((1, 2 * pos.shape[0]), np.complex128)
    gains[0, 0::2] = 2.0
    got, _, _ = I.dirty_images(vis, pos, nu, n, cell, gains=gains)
    v4 = vis.copy()
    v4[:, :, 0, :] *= 4.0
    ref, _, _ = I.dirty_images(v4, pos, nu, n, cell)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_phase_gains_move_a_source_to_its_pixel():
    # a source at the phase centre with corrections c_i = exp(-2 pi i (x_i l0 + y_i m0) / lambda)
    # has V'_ab = exp(-2 pi i (u l0 + v m0)): the image peaks at (l0, m0) with value 1
    pos = _small_array()
    n, cell, nu = 64, 0.02, 60e6
    r0, c0 = n // 2 + 7, n // 2 - 4
    l0, m0 = (c0 - n // 2) * cell, (r0 - n // 2) * cell
    vis = _point_source_vis(pos, nu, 0.0, 0.0)[None]
    lam = I.C_LIGHT / nu
    ph = np.exp(-2j * np.pi * (pos[:, 0] * l0 + pos[:, 1] * m0) / lam)
    gains = np.repeat(ph, 2)[None]                       # inputs 2a (X) and 2a+1 (Y)
    img, _, _ = I.dirty_images(vis, pos, np.array([nu]), n, cell, gains=gains)
    assert np.unravel_index(np.argmax(img[0]), img[0].shape) == (r0, c0)
    assert abs(img[0][r0, c0] - 1.0) < 2e-3


def test_uv_length_closed_form():
    pos = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    nu = I.C_LIGHT / 2.5                                 # lambda = 2.5 m: 5 m = 2 wavelengths
    assert I.uv_length_wavelengths(pos, np.array([0]), np.array([1]), nu)[0] == pytest.approx(2.0, rel=1e-15)


def test_uv_range_keeps_exactly_the_selected_baselines():
    # the cut image equals brute-force DFT imaging of the baselines whose length
    # lies in [uv_min, uv_max), and the counts follow
    pos = _small_array(10, 50.0, 9)
    n, cell, nu = 64, 0.02, 60e6
    vis = _rand_vis(np.random.default_rng(5), pos)
    a, b, idx = I._cross_pairs(pos.shape[0])
    lam = I.uv_length_wavelengths(pos, a, b, nu)
    srt = np.sort(lam)
    lo, hi = (srt[10] + srt[11]) / 2, (srt[30] + srt[31]) / 2          # between baseline lengths
    sel = np.nonzero((lam >= lo) & (lam < hi))[0]
    assert sel.size == 20
    img, ng, nd = I.dirty_images(vis, pos, np.array([nu]), n, cell, uv_range=(lo, hi))
    assert ng[0] == 2 * sel.size and nd[0] == a.size - sel.size
    ref = I.dft_image(vis[0], pos, nu, n, cell, baselines=sel)
    assert np.max(np.abs(img[0] - ref)) < 1e-3 * np.max(np.abs(ref))
    # an empty range grids nothing
    img0, ng0, _ = I.dirty_images(vis, pos, np.array([nu]), n, cell, uv_range=(hi, lo))
    assert ng0[0] == 0 and not img0.any()
