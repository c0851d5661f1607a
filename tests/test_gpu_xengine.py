"""GPU parity: X-engine, tensor-core and FP32 paths, bit-exact against the int64 oracle."""
import numpy as np
import pytest
import torch

import synth
from oracle import xengine as OX

pytestmark = pytest.mark.gpu


def _q(g, n_chan, k, n_input, lim=127):
    return g.integers(-lim, lim + 1, (n_chan, k, n_input, 2)).astype(np.int8)


def _oracle(q, n_ant, chans):
    # oracle layout [chan][input][K][2]
    return OX.correlate(q.transpose(0, 2, 1, 3), n_ant, chans)


@pytest.mark.parametrize("n_ant,k", [(1, 1), (2, 5), (3, 29), (16, 64), (17, 29), (64, 32), (65, 33),
                                     (130, 7), (200, 29), (384, 29), (383, 17), (352, 299)])
def test_random_exact(lib, n_ant, k):
    g = np.random.default_rng(n_ant * 1000 + k)
    n_chan = 5
    q = _q(g, n_chan, k, 2 * n_ant)
    d = torch.from_numpy(q).cuda()
    tc = lib.correlate(d, n_ant, n_chan, k, lib.XENG_TC).cpu().numpy()
    fp = lib.correlate(d, n_ant, n_chan, k, lib.XENG_FP32).cpu().numpy()
    assert lib.correlate_status() == 0
    ref = _oracle(q, n_ant, range(n_chan))
    assert np.array_equal(tc, ref)
    assert np.array_equal(fp, ref)


@pytest.mark.parametrize("k", [29, 260, 511])
def test_worst_case_magnitudes(lib, k):
    # -128 and 127 everywhere, input 0 all -128: partial sums reach 2 * 128^2 * K,
    # below 2^24 up to K = 511, the largest K the call accepts
    n_ant, n_chan = 24, 2
    g = np.random.default_rng(k)
    q = (g.integers(0, 2, (n_chan, k, 2 * n_ant, 2)) * 255 - 128).astype(np.int8)
    q[:, :, 0, :] = -128
    d = torch.from_numpy(q).cuda()
    tc = lib.correlate(d, n_ant, n_chan, k, lib.XENG_TC).cpu().numpy()
    fp = lib.correlate(d, n_ant, n_chan, k, lib.XENG_FP32).cpu().numpy()
    ref = _oracle(q, n_ant, range(n_chan))
    assert np.array_equal(tc, ref) and np.array_equal(fp, ref)
    assert np.abs(ref).max() == 2 * 128 * 128 * k


@pytest.mark.parametrize("mode", ["tc", "fp32"])
def test_accumulation_bound_rejected(lib, mode):
    # K = 512 could reach 2^24 with -128 inputs: refused before any launch
    n_ant, n_chan, k = 4, 1, 512
    d = torch.zeros((n_chan, k, 2 * n_ant, 2), dtype=torch.int8, device="cuda")
    md = lib.XENG_TC if mode == "tc" else lib.XENG_FP32
    with pytest.raises(lib.OvroError) as e:
        lib.correlate(d, n_ant, n_chan, k, md)
    assert e.value.status == lib.ERR_OVERFLOW


def test_full_array_sampled_channels(lib):
    # 352 antennas, K = 29, 8192 channels: sampled channels against the oracle,
    # every channel TC == FP32
    cfg = synth.make_config("full")
    g = np.random.default_rng(7)
    n_chan, k, n_ant = 8192, 29, 352
    q = np.clip(np.rint(g.normal(0, 8, (n_chan, k, 2 * n_ant, 2))), -127, 127).astype(np.int8)
    d = torch.from_numpy(q).cuda()
    tc = lib.correlate(d, n_ant, n_chan, k, lib.XENG_TC)
    fp = lib.correlate(d, n_ant, n_chan, k, lib.XENG_FP32)
    assert lib.correlate_status() == 0
    assert torch.equal(tc, fp)
    chans = [0, 1, 4095, 8191]
    ref = _oracle(q, n_ant, chans)
    assert np.array_equal(tc[chans].cpu().numpy(), ref)
    del cfg


def test_hermitian_autos_from_pipeline(lib):
    cfg = synth.make_config("tiny")
    volt = synth.generate(cfg)
    d = torch.from_numpy(volt).cuda()
    q, _ = lib.upchan(d, cfg.nfft)
    K = cfg.n_spec[0]
    vis = lib.correlate(q, cfg.n_ant, cfg.n_chan_total, K, lib.XENG_TC).cpu().numpy()
    qh = q.cpu().numpy().reshape(cfg.n_chan_total, K, cfg.n_input, 2).astype(np.int64)
    # autos: XX and YY real and equal to the summed power; XY = conj(YX)
    for a in range(cfg.n_ant):
        bl = OX.baseline_index(a, a, cfg.n_ant)
        px = (qh[:, :, 2 * a] ** 2).sum(axis=(1, 2))
        py = (qh[:, :, 2 * a + 1] ** 2).sum(axis=(1, 2))
        assert np.array_equal(vis[:, bl, 0, 0], px) and not vis[:, bl, 0, 1].any()
        assert np.array_equal(vis[:, bl, 3, 0], py) and not vis[:, bl, 3, 1].any()
        assert np.array_equal(vis[:, bl, 1, 0], vis[:, bl, 2, 0])
        assert np.array_equal(vis[:, bl, 1, 1], -vis[:, bl, 2, 1])
