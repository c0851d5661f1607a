"""The seeded input generator: determinism, level distribution, layouts."""
import numpy as np
from scipy.special import ndtr

import synth
from synth import workloads as W


def test_noise_thresholds_from_normal_cdf():
    ref = [int(round(ndtr((k + 0.5) / W.SIGMA_LEVELS) * 2 ** 32)) for k in range(-7, 7)]
    assert W.NOISE_THRESHOLDS_U32.tolist() == ref


def test_deterministic_and_sliceable():
    cfg = synth.make_config("tiny", n_tones=0)
    a = synth.generate(cfg)
    b = synth.generate(cfg, coarse=[1])
    assert np.array_equal(a[1], b[0])
    assert np.array_equal(a, synth.generate(cfg))


def test_layouts_and_counts():
    cfg = synth.make_config("full")
    assert cfg.n_input == 704 and cfg.n_spec == [29] and cfg.n_chan_total == 8192
    pos = synth.antenna_positions(cfg)
    r = np.hypot(pos[:, 0], pos[:, 1])
    assert (r[:251] <= 200).all() and ((r[251:] > 200) & (r[251:] <= 1500)).all()
    assert not pos[:, 2].any()
    f = synth.fine_freqs_hz([8192])
    assert f.size == 8192 and f[4096] == synth.coarse_centre_hz(0)


def test_batched_mix():
    cfg = synth.make_config("batched")
    assert len(cfg.nfft) == 32 and set(cfg.nfft) <= {1024, 4096, 16384}
    assert len(cfg.tones) == 20


def test_parallel_generation_is_identical():
    cfg = synth.make_config("tiny")
    assert np.array_equal(synth.generate_parallel(cfg, workers=2), synth.generate(cfg))
