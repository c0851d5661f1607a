"""ovro_upchan_noalloc: the upchannelizer for callers that cannot allocate
device memory (a plugin whose host owns the device heap, a real-time loop that
must not trigger an allocation).  Its scratch is a fixed array inside the
library, so it takes no workspace.  Checked through the C ABI against
ovro_upchan with a caller-allocated workspace, on two calls in a row."""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _fn(ov):
    fn = ov.lib().ovro_upchan_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return fn


def _noalloc(ov, volt, nfft, total):
    lib = ov.lib()
    fn = _fn(ov)
    nf = np.ascontiguousarray(nfft, dtype=np.int32)
    q = torch.empty(total, dtype=torch.int8, device="cuda")
    f = torch.empty(total, dtype=torch.float32, device="cuda")
    n_coarse, n_time, n_input = volt.shape
    st = fn(ctypes.c_void_p(volt.data_ptr()), n_input, n_coarse, n_time,
            nf.ctypes.data_as(ctypes.c_void_p), None, ctypes.c_void_p(q.data_ptr()),
            ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.ovro_last_error()
    return q, f


def test_noalloc_matches_workspace_entry_point(lib):
    cfg = synth.make_config("tiny")
    volt_a = torch.from_numpy(synth.generate(cfg)).cuda()
    volt_b = torch.from_numpy(synth.generate(synth.make_config("tiny", seed=99))).cuda()
    total = lib.fine_elements(cfg.nfft, cfg.n_time, cfg.n_input)
    for volt in (volt_a, volt_b):             # two calls in a row share the scratch array
        q_ref, f_ref = lib.upchan(volt, cfg.nfft, want_f32=True)
        q, f = _noalloc(lib, volt, cfg.nfft, total)
        torch.cuda.synchronize()
        assert torch.equal(q, q_ref)          # int8 spectra: bit-exact
        assert torch.equal(f, f_ref)          # same kernels, same FP32 spectra


def test_noalloc_rejects_oversized_call(lib):
    fn = _fn(lib)
    nf = (ctypes.c_int32 * 1)(1024)
    # 46,000 inputs x 1 coarse channel needs more than the fixed 1 MiB of scratch;
    # no device buffers are passed: the size check comes first, and were it ever
    # skipped the upchannelizer would refuse the null pointers without launching
    st = fn(None, 46000, 1, 4096, nf, None, None, None, None)
    assert st == -7
    assert b"scratch" in lib.lib().ovro_last_error()
