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
    nf = (ctypes.c_int32 * 1)(1000)
    assert lib.ovro_upchan(ctypes.c_void_p(16), 4, 1, 4096, nf, None, ctypes.c_void_p(16), None,
                           None, 0, None) == -2
    nf[0] = 1024
    assert lib.ovro_upchan(ctypes.c_void_p(16), 4, 1, 4096, nf, None, ctypes.c_void_p(16), None,
                           None, 0, None) == -5
    assert lib.ovro_upchan_workspace_size(704, 1) > 0
    assert lib.ovro_grid_image_workspace_size(352, 8192, 256, 0) > 0
    assert lib.ovro_grid_image_workspace_size(352, 8192, 300, 0) == 0


def test_default_widths(ov):
    from oracle.detect import WIDTHS
    assert ov.default_widths().tolist() == list(WIDTHS)
