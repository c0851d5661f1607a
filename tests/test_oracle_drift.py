"""Pins for the drift-rate search oracle: Taylor paths by hand and by their
properties, the brute-force path sums against an independently written
staged Taylor tree, drifting tones on and off the paths, edges and NMS."""
import math

import numpy as np
import pytest

from oracle import detect as OD, drift as DR


def test_paths_by_hand():
    assert DR.shift_table(4).tolist() == [[0, 0, 0, 0], [0, 0, 1, 1], [0, 1, 1, 2], [0, 1, 2, 3]]
    assert DR.shift_table(2).tolist() == [[0, 0], [0, 1]]
    assert DR.drift_order(3) == [0, 1, -1, 2, -2]


@pytest.mark.parametrize("T", [2, 4, 8, 16, 32])
def test_path_properties(T):
    tab = DR.shift_table(T)
    for d in range(T):
        row = tab[d]
        assert row[0] == 0 and row[-1] == d                 # starts at 0, ends at the drift
        assert set(np.diff(row)) <= {0, 1}                   # unit steps at most
        line = d * np.arange(T) / max(T - 1, 1)
        assert np.max(np.abs(row - line)) <= 1.0             # near the straight line
    # distinct drifts are distinct paths
    assert len({tuple(r) for r in tab}) == T


def _staged_tree(x):
    """Classic Taylor tree on rows x[t][f] (zero beyond the end): blocks of
    2, 4, ... rows, each row pair (top d', bottom d') of a block merged into
    drifts 2d' and 2d'+1; returns S[d][f] with rows kept in drift order."""
    T, F = x.shape
    pad = np.concatenate([x, np.zeros((T, T))], axis=1)
    blocks = [pad[t:t + 1] for t in range(T)]                  # each: [drifts][F + T]
    n = 1
    while n < T:
        nxt = []
        for b in range(0, len(blocks), 2):
            top, bot = blocks[b], blocks[b + 1]
            S = np.zeros((2 * n, F + T))
            for d in range(2 * n):
                dp, up = d // 2, d - d // 2
                S[d, : F + T - up] = top[dp, : F + T - up] + bot[dp, up:]
            nxt.append(S)
        blocks = nxt
        n *= 2
    return blocks[0][:, :F]


@pytest.mark.parametrize("T", [2, 4, 8, 16])
def test_brute_force_sums_equal_the_staged_tree(T):
    g = np.random.default_rng(T)
    F = 40
    x = g.normal(size=(T, F))
    s, order = DR.drift_sums(x[:, :, None], 0, F)
    tree = _staged_tree(x)
    for i, sd in enumerate(order):
        if sd < 0:
            continue
        ok = ~np.isnan(s[i, :, 0])
        assert np.allclose(s[i, ok, 0] * math.sqrt(T), tree[sd, ok], rtol=1e-12, atol=1e-12)
        assert ok.sum() == F - sd                          # valid while f + d < F
    # negative drifts are the mirror image
    rev, order2 = DR.drift_sums(x[:, ::-1, None], 0, F)
    for i, sd in enumerate(order):
        if sd > 0:
            j = order2.index(-sd)
            a, b = s[j, :, 0], rev[i, ::-1, 0]
            assert np.array_equal(np.isnan(a), np.isnan(b))
            assert np.allclose(a[~np.isnan(a)], b[~np.isnan(b)], rtol=1e-12)


@pytest.mark.parametrize("T,d0", [(8, 5), (8, -3), (16, 11), (4, 0)])
def test_tone_on_a_path(T, d0):
    # amplitude A on the path of drift d0 from channel f0, unit noise elsewhere
    # scaled down: the search finds (f0, d0) with SNR = A sqrt(T)
    g = np.random.default_rng(abs(d0) + T)
    F, n, f0, A = 64, 6, 30, 5.0
    z = 1e-3 * g.normal(size=(T, F, n, n))
    tab = DR.shift_table(T)
    for t in range(T):
        ch = f0 + (tab[abs(d0), t] if d0 >= 0 else -tab[abs(d0), t])
        z[t, ch, 2, 3] += A
    mask = np.ones((n, n), bool)
    snr, dr, cands, drifts = DR.drift_search(z, mask, [F], 8.0)
    assert dr[f0, 2, 3] == d0
    assert snr[f0, 2, 3] == pytest.approx(A * math.sqrt(T), rel=1e-3)
    assert [(c.chan, c.row, c.col, c.width) for c in cands] == [(f0, 2, 3, abs(d0) + 1)] and drifts == [d0]


def test_straight_tone_found_near_its_drift():
    # a tone drifting 9.6 channels over T = 16 sub-integrations (a straight
    # line, not a Taylor path): the best drift is within one of it
    T, F, f0, A = 16, 80, 20, 3.0
    z = np.zeros((T, F, 1, 1))
    for t in range(T):
        z[t, f0 + int(round(9.6 * t / (T - 1))), 0, 0] = A
    snr, dr, _, _ = DR.drift_search(z, np.ones((1, 1), bool), [F], 1.0)
    assert abs(dr[f0, 0, 0] - 9.6) <= 1.0
    assert snr[f0, 0, 0] >= A * (T - 3) / math.sqrt(T)


def test_edges_zero_drift_and_mask():
    T, F = 4, 10
    g = np.random.default_rng(3)
    z = g.normal(size=(T, 2 * F, 3, 3))
    s, order = DR.drift_sums(z, F, 2 * F)
    # drift 0 is the plain sum over sub-integrations
    assert np.allclose(s[0], z[:, F:].sum(axis=0) / 2.0)
    # at the last channel only drift 0 and the negative drifts are valid
    valid = [sd for i, sd in enumerate(order) if not np.isnan(s[i, F - 1, 0, 0])]
    assert valid == [0, -1, -2, -3]
    assert [sd for i, sd in enumerate(order) if not np.isnan(s[i, 0, 0, 0])] == [0, 1, 2, 3]
    mask = np.ones((3, 3), bool)
    mask[0, 0] = False
    snr, dr, _, _ = DR.drift_search(z, mask, [F, F], 50.0)
    assert np.all(np.isneginf(snr[:, 0, 0])) and np.all(dr[:, 0, 0] == 0)


def test_nms_suppresses_along_the_drifting_line():
    # two strong adjacent starts on one pixel: the weaker lies within the
    # stronger's half-width max(1, (|d|+1)//2) and is suppressed
    T, F = 8, 60
    z = np.zeros((T, F, 1, 1))
    tab = DR.shift_table(T)
    for t in range(T):
        z[t, 20 + tab[6, t], 0, 0] += 4.0
        z[t, 22 + tab[6, t], 0, 0] += 3.0
    _, _, cands, drifts = DR.drift_search(z, np.ones((1, 1), bool), [F], 5.0)
    assert [c.chan for c in cands] == [20] and drifts == [6] and cands[0].width == 7


def test_subint_bounds():
    assert DR.subint_bounds(29, 4) == [(0, 7), (7, 7), (14, 7), (21, 7)]


def test_bh_mode_is_stage_one_selection_on_the_drift_map():
    # the drift search's BH step is Stage I's selection applied to the map of
    # maxima over drifts: same p-values, m = in-horizon pixels x channels
    from oracle import detect as OD
    T, F, n = 8, 48, 8
    g = np.random.default_rng(21)
    z = g.normal(size=(T, F, n, n))
    tab = DR.shift_table(T)
    for t in range(T):
        z[t, 20 + tab[5, t], 3, 4] += 3.0
    mask = np.ones((n, n), bool)
    mask[0, 0] = False
    snr, dr, cands, drifts = DR.drift_search(z, mask, [F], mode="bh", alpha=0.05)
    sel = OD.select(snr, mask, "bh", 0.05)
    lp = OD.log_p(snr[:, mask].ravel())
    order = np.argsort(lp, kind="stable")
    k = OD.bh_threshold(lp[order], mask.sum() * F, 0.05)
    assert k > 0 and sel.sum() == k
    assert (3, 4) in {(c.row, c.col) for c in cands}
    assert all(sel[c.chan, c.row, c.col] for c in cands)
    # fixed mode keeps its meaning
    _, _, c10, _ = DR.drift_search(z, mask, [F], 10.0)
    assert all(c.snr >= 10.0 for c in c10)
