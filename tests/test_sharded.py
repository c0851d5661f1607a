"""The sharded Benjamini-Hochberg threshold on CPU: world_size-2 gloo ranks,
each holding one shard's SNR values, agree on the cut the oracle's
Benjamini-Hochberg step-up finds over the union of all values."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import detect as OD


def _shard(rank, n=120_000, df=3.0):
    g = np.random.default_rng(1000 + rank)
    return np.abs(g.standard_t(df, size=n)).astype(np.float32) * np.float32(1.3)


def _keys(v):
    u = v.view(np.uint32)
    return (np.where(u >> 31, ~u, u | np.uint32(0x80000000)) >> 16).astype(np.int64)


def _hist(v, key0, nb):
    k = _keys(v) - key0
    k = k[k >= 0]
    return np.bincount(np.minimum(k, nb - 1), minlength=nb).astype(np.uint64)


def _bin_values(v, key0, nb):
    k = _keys(v) - key0

    def f(b):
        return v[(k == b) | ((b == nb - 1) & (k > b))]
    return f


def _oracle_cut(values, alpha):
    lp = OD.log_p(values.astype(np.float64))
    order = np.argsort(lp, kind="stable")
    k = OD.bh_threshold(lp[order], values.size, alpha)
    return k, (values.astype(np.float64)[order][k - 1] if k else None)


def _worker(rank, world, port, alpha, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2606_04304_gb300 import ovro, sharded
        prm = ovro.detect_params(alpha=alpha)
        key0, nb = ovro.bh_layout(prm)
        v = _shard(rank)
        trace = []
        cut = sharded.global_cut(_hist(v, key0, nb), key0, v.size, prm, _bin_values(v, key0, nb), trace=trace)
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.array([np.nan if cut is None else cut, 2 in trace], np.float64))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("alpha", [0.05, 0.2])
def test_two_rank_cut_matches_oracle(tmp_path, alpha):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), alpha, str(tmp_path)), nprocs=world, join=True)
    res = [np.load(tmp_path / f"r{r}.npy") for r in range(world)]
    assert res[0][0] == res[1][0] or (np.isnan(res[0][0]) and np.isnan(res[1][0]))
    allv = np.concatenate([_shard(r) for r in range(world)])
    k, ref_cut = _oracle_cut(allv, alpha)
    cut = res[0][0]
    assert res[0][1] == 1 and res[1][1] == 1     # an open bin was resolved from both ranks' values
    if k == 0:
        assert np.isnan(cut)
    else:
        # the same rejected set: exactly the k largest values
        assert int((allv >= np.float32(cut)).sum()) == k
        assert np.float32(cut) == np.float32(ref_cut)


def test_single_shard_and_fixed_mode():
    from paper_2606_04304_gb300 import ovro, sharded
    prm = ovro.detect_params(alpha=0.1)
    key0, nb = ovro.bh_layout(prm)
    v = np.concatenate([_shard(0), _shard(1)])
    trace = []
    cut = sharded.global_cut(_hist(v, key0, nb), key0, v.size, prm, _bin_values(v, key0, nb), trace=trace)
    k, ref_cut = _oracle_cut(v, 0.1)
    assert k > 0 and int((v >= np.float32(cut)).sum()) == k
    # the library's key is the one the test bins with
    for x in (0.3, 2.33, 5.0, 17.25, 63.9):
        assert ovro.snr_bin_key(x) == int(_keys(np.array([x], np.float32))[0])
    fixed = ovro.detect_params(mode=ovro.DETECT_FIXED, nsigma=7.5)
    assert sharded.global_cut(np.zeros(nb, np.uint64), key0, 10, fixed, lambda b: None) == 7.5


def test_gaussian_noise_small_family_rejects_nothing():
    from paper_2606_04304_gb300 import ovro, sharded
    prm = ovro.detect_params(alpha=0.01)
    key0, nb = ovro.bh_layout(prm)
    v = np.abs(np.random.default_rng(3).normal(size=5000)).astype(np.float32)
    k, _ = _oracle_cut(v, 0.01)
    cut = sharded.global_cut(_hist(v, key0, nb), key0, v.size, prm, _bin_values(v, key0, nb))
    assert k == 0 and cut is None
