"""Pins for the X-engine oracle (Section 2.1): brute force, Hermitian symmetry,
autocorrelation = summed power, unit-modulus phase-only visibilities."""
import numpy as np

from oracle import xengine as X


def _rand_q(g, n_in, k, lim=127):
    return g.integers(-lim, lim + 1, (n_in, k, 2)).astype(np.int8)


def test_brute_force_tiny():
    g = np.random.default_rng(5)
    n_ant, k = 3, 4
    q = _rand_q(g, 2 * n_ant, k)
    got = X.correlate(q[None], n_ant)[0]
    bl = 0
    for a in range(n_ant):
        for b in range(a, n_ant):
            for pa in range(2):
                for pb in range(2):
                    acc = 0
                    for s in range(k):
                        zi = complex(int(q[2 * a + pa, s, 0]), int(q[2 * a + pa, s, 1]))
                        zj = complex(int(q[2 * b + pb, s, 0]), int(q[2 * b + pb, s, 1]))
                        acc += zi * zj.conjugate()
                    assert got[bl, 2 * pa + pb].tolist() == [int(acc.real), int(acc.imag)]
            bl += 1
    assert bl == X.n_baselines(n_ant)


def test_baseline_index_enumeration():
    n = 7
    k = 0
    for a in range(n):
        for b in range(a, n):
            assert X.baseline_index(a, b, n) == k
            k += 1
    a, b = X.baseline_pairs(n)
    assert all(X.baseline_index(int(x), int(y), n) == i for i, (x, y) in enumerate(zip(a, b)))


def test_hermitian_and_autos():
    g = np.random.default_rng(6)
    q = _rand_q(g, 10, 29)
    vre, vim = X.full_matrix(q)
    assert np.array_equal(vre, vre.T) and np.array_equal(vim, -vim.T)
    p = (q.astype(np.int64) ** 2).sum(axis=(1, 2))
    assert np.array_equal(np.diag(vre), p) and not np.diag(vim).any()


def test_unit_modulus_point_source():
    # q_i(s) = i^{m_i} z(s): V_ij = i^{m_i - m_j} sum |z|^2, so V_ij / sqrt(V_ii V_jj)
    # is exactly a unit-modulus quarter-turn phase
    g = np.random.default_rng(7)
    k, n_in = 17, 8
    z = g.integers(-100, 101, (k, 2))
    m = g.integers(0, 4, n_in)
    q = np.empty((n_in, k, 2), np.int64)
    for i in range(n_in):
        zr, zi = z[:, 0], z[:, 1]
        for _ in range(m[i]):
            zr, zi = -zi, zr
        q[i, :, 0], q[i, :, 1] = zr, zi
    vre, vim = X.full_matrix(q.astype(np.int8))
    pw = int((z ** 2).sum())
    for i in range(n_in):
        for j in range(n_in):
            ph = (1j) ** int(m[i] - m[j])
            assert vre[i, j] == round(pw * ph.real) and vim[i, j] == round(pw * ph.imag)
            assert vre[i, j] ** 2 + vim[i, j] ** 2 == vre[i, i] * vre[j, j]


def test_worst_case_fits_int32():
    # -128 everywhere: |V| <= 2 * 128^2 * K, below 2^31 up to K ~ 65,000; below 2^24 up to K = 511
    k = 511
    q = np.full((2, k, 2), -128, np.int8)
    vre, vim = X.full_matrix(q)
    assert np.abs(vre).max() == 2 * 128 * 128 * k < 2 ** 24
