"""The C-ABI library loads, exports every symbol include/ovro.h declares, and
rejects invalid arguments on the host (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ovro.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ovro_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def ov():
    from paper_2606_04304_gb300 import build
    build.build()
    from paper_2606_04304_gb300 import ovro
    return ovro


def test_exports_every_declared_symbol(ov):
    names = _declared()
    assert len(names) >= 15
    lib = ctypes.CDLL(ov.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(ov):
    lib = ov.lib()
    assert lib.ovro_status_string(0) == b"OVRO_OK"
    assert lib.ovro_status_string(-7) == b"OVRO_ERR_CAPACITY"
    assert lib.ovro_version() >> 16 == 1


def test_host_validation_without_gpu(ov):
    lib = ov.lib()
    # null pointers / bad sizes are rejected before any CUDA call
    assert lib.ovro_correlate(None, 4, 1, 1, 0, None, None) == -1
    assert lib.ovro_correlate(ctypes.c_void_p(16), 4, 1, 521, 0, ctypes.c_void_p(16), None) == -6
    assert lib.ovro_correlate(ctypes.c_void_p(16), 4, 1, 1, 7, ctypes.c_void_p(16), None) == -1
    assert lib.ovro_correlate(ctypes.c_void_p(16), 5000, 1, 1, 0, ctypes.c_void_p(16), None) == -2
    nf = (ctypes.c_int32 * 1)(1002)          # 2 x 3 x 167: no mixed-radix plan
    assert lib.ovro_upchan(ctypes.c_void_p(16), 4, 1, 4096, nf, None, ctypes.c_void_p(16), None,
                           None, 0, None) == -2
    nf[0] = 2400                                # planned; then the missing workspace is refused
    assert lib.ovro_upchan(ctypes.c_void_p(16), 4, 1, 4800, nf, None, ctypes.c_void_p(16), None,
                           None, 0, None) == -5
    nf[0] = 1024
    assert lib.ovro_upchan(ctypes.c_void_p(16), 4, 1, 4096, nf, None, ctypes.c_void_p(16), None,
                           None, 0, None) == -5
    assert lib.ovro_upchan_workspace_size(704, 1) > 0
    assert lib.ovro_grid_image_workspace_size(352, 8192, 256, 0) > 0
    assert lib.ovro_grid_image_workspace_size(352, 8192, 300, 0) == 0


def test_upchan_options_validation_without_gpu(ov):
    lib = ov.lib()
    nf = (ctypes.c_int32 * 2)(2400, 4096)
    v, q = ctypes.c_void_p(16), ctypes.c_void_p(16)

    def call(opt, n_time=3 * 4096):
        return lib.ovro_upchan_ex(v, 4, 2, n_time, nf, None, ctypes.byref(opt), q, None, None, 0, None)

    O = ov._UpchanOptions
    assert call(O(0, None, 0, 0)) == -1                 # n_taps < 1
    assert call(O(2, None, 0, 0)) == -1                 # taps needed for P > 1
    assert call(O(1, None, -1, 0)) == -1                # chan_lo < 0
    assert call(O(1, None, 0, -3)) == -1                # chan_count < 0
    assert call(O(1, None, 2200, 300)) == -1            # window past N = 2400
    taps = (ctypes.c_void_p * 2)(16, None)
    assert call(O(2, ctypes.cast(taps, ctypes.c_void_p), 0, 0)) == -1     # a NULL taps pointer
    taps = (ctypes.c_void_p * 2)(16, 16)
    assert call(O(4, ctypes.cast(taps, ctypes.c_void_p), 0, 0)) == -2     # K = 3 - 4 + 1 = 0 for N = 4096
    assert call(O(1, None, 2100, 300)) == -5            # valid: only the workspace is missing


def test_default_widths(ov):
    from oracle.detect import WIDTHS
    assert ov.default_widths().tolist() == list(WIDTHS)


def _pipeline_cfg(ov, nfft, n_ant=8, **kw):
    import numpy as np
    keep = dict(nf=np.asarray(nfft, np.int32), hz=60e6 + 24e3 * np.arange(len(nfft), dtype=np.float64),
                ant=np.zeros((n_ant, 3)))
    cfg = ov.PipelineConfig(n_ant, len(nfft), keep["nf"].ctypes.data, keep["hz"].ctypes.data, kw.get("n_time", 4096),
                            keep["ant"].ctypes.data, kw.get("image_size", 32), kw.get("cell", 2.0 / 32),
                            kw.get("xeng", ov.XENG_TC), ov.detect_params(), 1)
    return cfg, keep


def test_pipeline_host_planning(ov):
    import numpy as np
    import synth
    lib = ov.lib()
    cfg, keep = _pipeline_cfg(ov, [256, 64, 1024])
    h = ctypes.c_void_p()
    assert lib.ovro_pipeline_create(ctypes.byref(cfg), ctypes.byref(h)) == 0
    try:
        assert lib.ovro_pipeline_workspace_size(h) > 0
        n = lib.ovro_pipeline_channels(h, None)
        assert n == 256 + 64 + 1024
        f = np.zeros(n)
        lib.ovro_pipeline_channels(h, f.ctypes.data_as(ctypes.c_void_p))
        # fine channel k of coarse c at nu_c + (k - N/2) f_c / N, as the synthetic generator
        assert np.array_equal(f, synth.fine_freqs_hz([256, 64, 1024]))
        out, n_out = (ov.Candidate * 1)(), ctypes.c_int(7)
        # not bound: refused before any device access
        assert lib.ovro_pipeline_run(h, ctypes.c_void_p(16), out, 1, ctypes.byref(n_out), None) == -5
        assert n_out.value == 0
        k, g = ctypes.c_longlong(-1), ctypes.c_int(-1)
        assert lib.ovro_pipeline_stats(h, ctypes.byref(k), ctypes.byref(g)) == 0 and g.value == 0
    finally:
        lib.ovro_pipeline_destroy(h)


def test_pipeline_rejects_bad_configs(ov):
    lib = ov.lib()
    h = ctypes.c_void_p()
    assert lib.ovro_pipeline_create(None, ctypes.byref(h)) == -1
    for kw, nfft, want in ((dict(n_time=100), [256], -1),       # fewer samples than one spectrum
                           (dict(xeng=7), [256], -1),
                           (dict(cell=0.0), [256], -1),
                           (dict(image_size=48), [256], -2),   # not a power of two
                           (dict(), [0], -1)):
        cfg, keep = _pipeline_cfg(ov, nfft, **kw)
        assert lib.ovro_pipeline_create(ctypes.byref(cfg), ctypes.byref(h)) == want, (kw, nfft)


def test_tuner_cache_roundtrip(ov, tmp_path):
    ov.tune_clear()
    assert ov.tune_count() == 0 and ov.tune_get("k_rank/sm152/1/2") is None
    ov.tune_set("k_rank/sm152/1/2", 4)
    ov.tune_set("grid_batch/sm152/352/8192/256", 16)
    p = tmp_path / "tune.txt"
    ov.tune_save(p)
    ov.tune_clear()
    ov.tune_load(p)
    assert ov.tune_count() == 2
    assert ov.tune_get("k_rank/sm152/1/2") == 4 and ov.tune_get("grid_batch/sm152/352/8192/256") == 16
    (tmp_path / "bad.txt").write_text("k 1 2 x\nk2 notanumber\n")
    with pytest.raises(ov.OvroError):
        ov.tune_load(tmp_path / "bad.txt")
    ov.tune_clear()
