"""Thin Python binding of the C ABI in include/ovro.h (argument marshalling only).

PyTorch supplies device memory and the current CUDA stream; every step of the
computation runs in libovro.so.  Importing this module loads the library and
raises immediately if it has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libovro.so")

OVRO_OK = 0
(ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_CUDA, ERR_TIMEOUT, ERR_WORKSPACE, ERR_OVERFLOW,
 ERR_CAPACITY) = -1, -2, -3, -4, -5, -6, -7
XENG_TC, XENG_FP32 = 0, 1
STORE_FP32, STORE_BF16, STORE_FP16 = 0, 1, 2
DETECT_BH, DETECT_FIXED = 0, 1


class OvroError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        msg = _lib.ovro_status_string(status).decode()
        last = _lib.ovro_last_error().decode()
        super().__init__(f"{fn} -> {msg}" + (f" ({last})" if last else ""))


class DetectParams(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("alpha", ctypes.c_double), ("nsigma", ctypes.c_double),
                ("highpass_hz", ctypes.c_double), ("coarse_bw_hz", ctypes.c_double)]


class Candidate(ctypes.Structure):
    _fields_ = [("coarse", ctypes.c_int32), ("fine", ctypes.c_int32), ("chan", ctypes.c_int32),
                ("row", ctypes.c_int32), ("col", ctypes.c_int32), ("width", ctypes.c_int32),
                ("snr", ctypes.c_float), ("score", ctypes.c_float), ("freq_hz", ctypes.c_double),
                ("log10_p", ctypes.c_double)]


CANDIDATE_DTYPE = np.dtype([("coarse", "<i4"), ("fine", "<i4"), ("chan", "<i4"), ("row", "<i4"),
                            ("col", "<i4"), ("width", "<i4"), ("snr", "<f4"), ("score", "<f4"),
                            ("freq_hz", "<f8"), ("log10_p", "<f8")])


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(the library has no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, L, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    sig = {
        "ovro_status_string": (ctypes.c_char_p, [I]),
        "ovro_last_error": (ctypes.c_char_p, []),
        "ovro_version": (I, []),
        "ovro_launch_count": (ctypes.c_ulonglong, []),
        "ovro_profile": (I, [I]),
        "ovro_profile_query": (I, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
        "ovro_upchan_workspace_size": (S, [I, I]),
        "ovro_upchan": (I, [P, I, I, L, P, P, P, P, P, S, P]),
        "ovro_upchan_ex": (I, [P, I, I, L, P, P, P, P, P, P, S, P]),
        "ovro_correlate": (I, [P, I, I, I, I, P, P]),
        "ovro_correlate_status": (I, [P]),
        "ovro_grid_image_workspace_size": (S, [I, I, I, I]),
        "ovro_grid_image": (I, [P, I, P, P, I, I, D, I, P, P, P, S, P]),
        "ovro_uvw": (I, [P, I, P, I, I, D, P, P, P, S, P]),
        "ovro_grid_image_ex": (I, [P, I, P, P, I, I, D, P, P, P, P, S, P]),
        "ovro_default_widths": (I, [P]),
        "ovro_detect_workspace_size": (S, [I, I, I, P]),
        "ovro_detect": (I, [P, I, I, D, I, P, P, P, P, P, I, P, P, S, P]),
        "ovro_scorer_detect_workspace_size": (S, [I, I, I, I]),
        "ovro_detect_stats": (I, [P, I, I, D, P, P, S, P]),
        "ovro_detect_filter": (I, [P, P, I, I, D, I, P, P, P, P, P, P, S, P]),
        "ovro_scorer_n_params": (I, []),
        "ovro_scorer_workspace_size": (S, [I, I]),
        "ovro_scorer_cutouts": (I, [P, I, I, I, P, P, I, P, P, S, P]),
        "ovro_scorer_forward": (I, [P, P, I, P, P, S, P]),
        "ovro_scorer_grad": (I, [P, I, P, P, I, P, P, P, S, P]),
        "ovro_scorer_adam": (I, [P, P, P, P, I, ctypes.c_float, P, P]),
        "ovro_scorer_to_bf16": (I, [P, P, P]),
        "ovro_pipeline_create": (I, [P, P]),
        "ovro_pipeline_workspace_size": (S, [P]),
        "ovro_pipeline_bind": (I, [P, P, S, P]),
        "ovro_pipeline_run": (I, [P, P, P, I, P, P]),
        "ovro_pipeline_channels": (I, [P, P]),
        "ovro_pipeline_stats": (I, [P, P, P]),
        "ovro_pipeline_destroy": (None, [P]),
        "ovro_pipeline_gridded": (I, [P, P, P]),
        "ovro_search_create": (I, [I, I, D, I, P, P, P, S, P, P]),
        "ovro_search_reset": (I, [P, P]),
        "ovro_search_add": (I, [P, I, P, P]),
        "ovro_search_layout": (I, [P, P, P, P]),
        "ovro_search_histogram": (I, [P, P, I, P]),
        "ovro_search_bin_values": (I, [P, I, P, ctypes.c_longlong, P, P]),
        "ovro_search_candidates": (I, [P, ctypes.c_float, P, P, I, P, P]),
        "ovro_search_destroy": (None, [P]),
        "ovro_bh_layout": (I, [P, P, P]),
        "ovro_bh_bin_verdict": (I, [P, I, ctypes.c_uint32, D, D, I, P, P]),
        "ovro_bh_resolve": (I, [P, ctypes.c_longlong, ctypes.c_ulonglong, D, D, P]),
        "ovro_snr_bin_key": (ctypes.c_uint32, [ctypes.c_float]),
        "ovro_vet_default_params": (None, [P]),
        "ovro_vet_workspace_size": (S, [I, I]),
        "ovro_vet": (I, [P, P, I, I, D, I, P, P, P, I, ctypes.c_float, P, P, P, S, P]),
        "ovro_drift_workspace_size": (S, [I, I, I, P]),
        "ovro_drift_search": (I, [P, I, I, I, D, I, P, P, P, P, P, P, P, I, P, P, S, P]),
        "ovro_spectra_slice": (I, [P, I, I, I, I, I, P, P]),
        "ovro_pipeline_run_device": (I, [P, P, P]),
        "ovro_pipeline_search": (I, [P, P]),
        "ovro_autotune": (I, [I]),
        "ovro_tune_get": (I, [ctypes.c_char_p, P]),
        "ovro_tune_set": (I, [ctypes.c_char_p, I]),
        "ovro_tune_count": (I, []),
        "ovro_tune_clear": (I, []),
        "ovro_tune_save": (I, [ctypes.c_char_p]),
        "ovro_tune_load": (I, [ctypes.c_char_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def lib() -> ctypes.CDLL:
    return _lib


def launch_count() -> int:
    return int(_lib.ovro_launch_count())


def profile(enable: bool) -> None:
    """Start (clearing the trace) or stop per-kernel CUDA-event tracing."""
    _check("ovro_profile", _lib.ovro_profile(1 if enable else 0))


def profile_query(kernel: str):
    """(summed device ms, launches) of one traced kernel."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int(0)
    _check("ovro_profile_query", _lib.ovro_profile_query(kernel.encode(), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


TRACED_KERNELS = ("k_upchan", "k_upchan_mr", "k_vet_line", "k_vet_fit", "k_drift", "k_scorer_fwd", "k_xeng_tc", "k_xeng_simt", "k_grid_prep", "k_grid_tiles", "k_fft_rows", "k_fft_cols", "k_stats", "k_ztrans",
                  "k_rank", "k_walk", "k_median_sub", "k_mf", "k_nms_warp")


def _check(fn: str, status: int) -> int:
    if status != OVRO_OK:
        raise OvroError(fn, status)
    return status


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream: Optional[torch.cuda.Stream] = None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _host(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def _cuda(t: torch.Tensor, dtype: torch.dtype, name: str):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")


def workspace(nbytes: int, device=None) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device or "cuda")


def fine_elements(nfft: Sequence[int], n_time: int, n_input: int, n_taps: int = 1,
                  chan_count: int = 0) -> int:
    return int(sum((chan_count or n) * (n_time // n - n_taps + 1) * n_input * 2 for n in nfft))


class _UpchanOptions(ctypes.Structure):
    _fields_ = [("n_taps", ctypes.c_int32), ("h_taps", ctypes.c_void_p), ("chan_lo", ctypes.c_int32),
                ("chan_count", ctypes.c_int32)]


# ---------------------------------------------------------------------- a1-a3
def upchan(volt: torch.Tensor, nfft: Sequence[int], scales=None, want_f32: bool = False,
           out_q: Optional[torch.Tensor] = None, ws: Optional[torch.Tensor] = None, stream=None,
           taps: Optional[Sequence[torch.Tensor]] = None, window: Optional[Tuple[int, int]] = None):
    """volt: uint8 [n_coarse][n_time][n_input] on the GPU.  Returns (q int8, f32 or None),
    both flat in the coarse-major [C][K][n_input][2] block layout of ovro_upchan_ex.

    taps: None (plain FFT) or one contiguous CUDA float32 tensor of P N_c
    polyphase-filter coefficients per coarse channel, all with the same P.
    window: None or (chan_lo, chan_count), the fftshifted fine channels kept."""
    _cuda(volt, torch.uint8, "volt")
    n_coarse, n_time, n_input = volt.shape
    nf = _host(nfft, np.int32)
    n_taps = 1
    tap_ptrs = None
    if taps is not None:
        if len(taps) != n_coarse:
            raise ValueError("taps: one tensor per coarse channel")
        for t in taps:
            _cuda(t, torch.float32, "taps")
        n_taps = taps[0].numel() // int(nf[0])
        tap_ptrs = (ctypes.c_void_p * n_coarse)(*[t.data_ptr() for t in taps])
    lo, cnt = window if window is not None else (0, 0)
    opt = _UpchanOptions(n_taps, ctypes.cast(tap_ptrs, ctypes.c_void_p) if tap_ptrs is not None else None,
                         lo, cnt)
    total = fine_elements(nf, n_time, n_input, n_taps, cnt)
    q = out_q if out_q is not None else torch.empty(max(total, 1), dtype=torch.int8, device=volt.device)
    f = torch.empty(max(total, 1), dtype=torch.float32, device=volt.device) if want_f32 else None
    need = _lib.ovro_upchan_workspace_size(n_input, n_coarse)
    ws = ws if ws is not None and ws.numel() >= need else workspace(need, volt.device)
    sc = None if scales is None else _host(scales, np.float64)
    _check("ovro_upchan_ex", _lib.ovro_upchan_ex(
        _ptr(volt), n_input, n_coarse, n_time, nf.ctypes.data_as(ctypes.c_void_p),
        None if sc is None else sc.ctypes.data_as(ctypes.c_void_p), ctypes.byref(opt), _ptr(q), _ptr(f),
        _ptr(ws), ws.numel(), _stream(stream)))
    return q[:total], (None if f is None else f[:total])


# ------------------------------------------------------------------------- a4
def n_baselines(n_ant: int) -> int:
    return n_ant * (n_ant + 1) // 2


def correlate(q: torch.Tensor, n_ant: int, n_chan: int, n_spec: int, mode: int = XENG_TC,
              out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """q: int8 [n_chan][n_spec][2 n_ant][2] (flat ok).  Returns int32 [n_chan][n_bl][4][2]."""
    _cuda(q, torch.int8, "q")
    vis = out if out is not None else torch.empty((n_chan, n_baselines(n_ant), 4, 2), dtype=torch.int32,
                                                  device=q.device)
    _check("ovro_correlate", _lib.ovro_correlate(_ptr(q), n_ant, n_chan, n_spec, mode, _ptr(vis),
                                                 _stream(stream)))
    return vis


def correlate_status(stream=None) -> int:
    return _lib.ovro_correlate_status(_stream(stream))


# ---------------------------------------------------------------------- a5-a7
def grid_image_workspace_size(n_ant: int, n_chan: int, image_size: int, storage: int = STORE_FP32) -> int:
    return _lib.ovro_grid_image_workspace_size(n_ant, n_chan, image_size, storage)


class GridOptions(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int), ("d_gains_or_null", ctypes.c_void_p),
                ("uv_min_lambda", ctypes.c_double), ("uv_max_lambda", ctypes.c_double)]


def grid_image(vis: torch.Tensor, ant_enu_m, freqs_hz, image_size: int, cell: float,
               storage: int = STORE_FP32, out: Optional[torch.Tensor] = None,
               ws: Optional[torch.Tensor] = None, want_counts: bool = False, stream=None,
               gains: Optional[torch.Tensor] = None, uv_range=None):
    """vis: int32 [n_chan][n_bl][4][2].  Returns float images [n_chan][N][N] (and counts).
    gains: optional complex64 [n_chan][2 n_ant] calibration corrections on the GPU;
    uv_range: optional (uv_min, uv_max) in wavelengths (uv_max <= 0 or inf: no upper cut)."""
    if gains is not None or uv_range is not None:
        return _grid_image_ex(vis, ant_enu_m, freqs_hz, image_size, cell, storage, out, ws, want_counts, stream,
                              gains, uv_range)
    _cuda(vis, torch.int32, "vis")
    pos = _host(ant_enu_m, np.float64)
    fr = _host(freqs_hz, np.float64)
    n_ant, n_chan = pos.shape[0], fr.shape[0]
    img = out if out is not None else torch.empty((n_chan, image_size, image_size), dtype=torch.float32,
                                                  device=vis.device)
    cnt = torch.empty(n_chan, dtype=torch.int32, device=vis.device) if want_counts else None
    need = grid_image_workspace_size(n_ant, n_chan, image_size, storage)
    ws = ws if ws is not None and ws.numel() >= need else workspace(need, vis.device)
    _check("ovro_grid_image", _lib.ovro_grid_image(
        _ptr(vis), n_ant, pos.ctypes.data_as(ctypes.c_void_p), fr.ctypes.data_as(ctypes.c_void_p), n_chan,
        image_size, float(cell), storage, _ptr(img), _ptr(cnt), _ptr(ws), ws.numel(), _stream(stream)))
    return (img, cnt) if want_counts else img


def _grid_image_ex(vis, ant_enu_m, freqs_hz, image_size, cell, storage, out, ws, want_counts, stream, gains,
                   uv_range):
    _cuda(vis, torch.int32, "vis")
    pos = _host(ant_enu_m, np.float64)
    fr = _host(freqs_hz, np.float64)
    n_ant, n_chan = pos.shape[0], fr.shape[0]
    if gains is not None:
        _cuda(gains, torch.complex64, "gains")
        if tuple(gains.shape) != (n_chan, 2 * n_ant):
            raise ValueError("gains must be complex64 [n_chan][2 n_ant]")
    lo, hi = (0.0, 0.0) if uv_range is None else (float(uv_range[0]), float(uv_range[1]))
    if not np.isfinite(hi):
        hi = 0.0
    opt = GridOptions(storage, None if gains is None else gains.data_ptr(), lo, hi)
    img = out if out is not None else torch.empty((n_chan, image_size, image_size), dtype=torch.float32,
                                                  device=vis.device)
    cnt = torch.empty(n_chan, dtype=torch.int32, device=vis.device) if want_counts else None
    need = grid_image_workspace_size(n_ant, n_chan, image_size, storage)
    ws = ws if ws is not None and ws.numel() >= need else workspace(need, vis.device)
    _check("ovro_grid_image_ex", _lib.ovro_grid_image_ex(
        _ptr(vis), n_ant, pos.ctypes.data_as(ctypes.c_void_p), fr.ctypes.data_as(ctypes.c_void_p), n_chan,
        image_size, float(cell), ctypes.byref(opt), _ptr(img), _ptr(cnt), _ptr(ws), ws.numel(), _stream(stream)))
    return (img, cnt) if want_counts else img


def uvw(ant_enu_m, freqs_hz, image_size: int, cell: float, stream=None):
    """a5 alone: int32 (p_u, p_v) [n_chan][n_cross], positions in 1/1024 cell."""
    pos = _host(ant_enu_m, np.float64)
    fr = _host(freqs_hz, np.float64)
    n_ant, n_chan = pos.shape[0], fr.shape[0]
    n_cross = n_ant * (n_ant - 1) // 2
    pu = torch.empty((n_chan, n_cross), dtype=torch.int32, device="cuda")
    pv = torch.empty_like(pu)
    need = grid_image_workspace_size(n_ant, n_chan, image_size)
    ws = workspace(need)
    _check("ovro_uvw", _lib.ovro_uvw(pos.ctypes.data_as(ctypes.c_void_p), n_ant,
                                     fr.ctypes.data_as(ctypes.c_void_p), n_chan, image_size, float(cell),
                                     _ptr(pu), _ptr(pv), _ptr(ws), ws.numel(), _stream(stream)))
    return pu, pv


# --------------------------------------------------------------------- a8-a12
def default_widths() -> np.ndarray:
    n = _lib.ovro_default_widths(None)
    out = np.zeros(n, np.int32)
    _lib.ovro_default_widths(out.ctypes.data_as(ctypes.c_void_p))
    return out


def detect_params(mode: int = DETECT_BH, alpha: float = 0.01, nsigma: float = 10.0,
                  highpass_hz: float = 5000.0, coarse_bw_hz: float = 24000.0) -> DetectParams:
    return DetectParams(mode, alpha, nsigma, highpass_hz, coarse_bw_hz)


def detect_workspace_size(n_chan: int, image_size: int, nfft: Sequence[int]) -> int:
    nf = _host(nfft, np.int32)
    return _lib.ovro_detect_workspace_size(n_chan, image_size, len(nf), nf.ctypes.data_as(ctypes.c_void_p))


class ScorerParams(ctypes.Structure):
    _fields_ = [("d_w_bf16", ctypes.c_void_p), ("trigger_nsigma", ctypes.c_double), ("keep_prob", ctypes.c_float),
                ("max_triggers", ctypes.c_int), ("d_ws", ctypes.c_void_p), ("ws_bytes", ctypes.c_size_t)]


class DetectScorer:
    """The learned scorer as a stage of detect(): BF16 weights (a torch bf16
    tensor of scorer_n_params() values), the relaxed trigger threshold and
    the keep probability."""

    def __init__(self, w_bf16: torch.Tensor, trigger_nsigma: float = 5.0, keep_prob: float = 0.5,
                 max_triggers: int = 1 << 20):
        _cuda(w_bf16, torch.bfloat16, "w_bf16")
        self.w_bf16, self.trigger_nsigma, self.keep_prob = w_bf16, float(trigger_nsigma), float(keep_prob)
        self.max_triggers = int(max_triggers)


def detect(img: torch.Tensor, cell: float, nfft: Sequence[int], freqs_hz, params: Optional[DetectParams] = None,
           max_out: int = 1 << 20, ws: Optional[torch.Tensor] = None, scorer: Optional[DetectScorer] = None,
           stream=None) -> np.ndarray:
    """Stage I search; returns a structured array of candidates (CANDIDATE_DTYPE).
    With a scorer, its relaxed triggers are kept by the network's probability."""
    _cuda(img, torch.float32, "img")
    n_chan, n, _ = img.shape
    nf = _host(nfft, np.int32)
    fr = _host(freqs_hz, np.float64)
    prm = params or detect_params()
    need = detect_workspace_size(n_chan, n, nf)
    ws = ws if ws is not None and ws.numel() >= need else workspace(need, img.device)
    sp = None
    if scorer is not None:
        sws = workspace(_lib.ovro_scorer_detect_workspace_size(n_chan, n, len(nf), scorer.max_triggers), img.device)
        sp = ScorerParams(scorer.w_bf16.data_ptr(), scorer.trigger_nsigma, scorer.keep_prob, scorer.max_triggers,
                          sws.data_ptr(), sws.numel())
    out = np.zeros(max_out, CANDIDATE_DTYPE)
    n_out = ctypes.c_int(0)
    st = _lib.ovro_detect(_ptr(img), n_chan, n, float(cell), len(nf), nf.ctypes.data_as(ctypes.c_void_p),
                          fr.ctypes.data_as(ctypes.c_void_p), ctypes.byref(prm),
                          None if sp is None else ctypes.byref(sp),
                          out.ctypes.data_as(ctypes.c_void_p), max_out, ctypes.byref(n_out), _ptr(ws),
                          ws.numel(), _stream(stream))
    _check("ovro_detect", st)
    return out[: n_out.value]


# --------------------------------------------- Stage I re-evaluation, Stage II
VET_REEVAL, VET_EXTENDED, VET_NOISY, VET_FIT = 1, 2, 4, 8
VET_RESULT_DTYPE = np.dtype([("keep", "<i4"), ("flags", "<i4"), ("snr_re", "<f4"), ("area_ratio", "<f4"),
                             ("amp", "<f8"), ("col", "<f8"), ("row", "<f8"), ("sigma_col", "<f8"),
                             ("sigma_row", "<f8"), ("chi2_red", "<f8"), ("beam_fwhm", "<f8"),
                             ("sigma_therm", "<f8"), ("noise_std", "<f8"), ("iterations", "<i4"), ("pad_", "<i4")])


class VetParams(ctypes.Structure):
    _fields_ = [("offline_half", ctypes.c_int32), ("fit_half", ctypes.c_int32), ("max_area_ratio", ctypes.c_double),
                ("max_noise_std", ctypes.c_double), ("max_sigma_dev", ctypes.c_double)]


def vet_params(**kw) -> VetParams:
    p = VetParams()
    _lib.ovro_vet_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def psf_images(ant_enu_m, freqs_hz, image_size: int, cell: float, stream=None) -> torch.Tensor:
    """Point-spread images [n][N][N]: the dirty images of unit XX and YY
    visibilities on every cross baseline, one per frequency (ovro_grid_image)."""
    pos = _host(ant_enu_m, np.float64)
    n_ant = pos.shape[0]
    fr = _host(freqs_hz, np.float64)
    vis = torch.zeros((fr.size, n_baselines(n_ant), 4, 2), dtype=torch.int32, device="cuda")
    vis[:, :, 0, 0] = 1
    vis[:, :, 3, 0] = 1
    return grid_image(vis, pos, fr, image_size, cell, stream=stream)


def vet(img: torch.Tensor, stats: torch.Tensor, cell: float, nfft: Sequence[int], psf: torch.Tensor, cands,
        cut: float, params: Optional[VetParams] = None, stream=None) -> np.ndarray:
    """Re-evaluate and vet Stage I candidates (CANDIDATE_DTYPE records); returns
    VET_RESULT_DTYPE records in the same order."""
    _cuda(img, torch.float32, "img")
    _cuda(stats, torch.float64, "stats")
    _cuda(psf, torch.float32, "psf")
    n_chan, n, _ = img.shape
    nf = _host(nfft, np.int32)
    cd = np.ascontiguousarray(np.asarray(cands, CANDIDATE_DTYPE))
    out = np.zeros(max(cd.size, 1), VET_RESULT_DTYPE)
    ws = workspace(_lib.ovro_vet_workspace_size(cd.size, nf.size), img.device)
    _check("ovro_vet", _lib.ovro_vet(
        _ptr(img), _ptr(stats), n_chan, n, float(cell), nf.size, nf.ctypes.data_as(ctypes.c_void_p), _ptr(psf),
        cd.ctypes.data_as(ctypes.c_void_p), cd.size, float(cut), None if params is None else ctypes.byref(params),
        out.ctypes.data_as(ctypes.c_void_p), _ptr(ws), ws.numel(), _stream(stream)))
    return out[: cd.size]


# ------------------------------------------------------------ drift search
def spectra_slice(q: torch.Tensor, n_chan: int, n_spec: int, n_input: int, s0: int, count: int,
                  stream=None) -> torch.Tensor:
    """int8 [n_chan][count][n_input][2]: spectra s0 .. s0+count-1 of q [n_chan][n_spec][n_input][2]."""
    _cuda(q, torch.int8, "q")
    out = torch.empty((n_chan, count, n_input, 2), dtype=torch.int8, device=q.device)
    _check("ovro_spectra_slice", _lib.ovro_spectra_slice(_ptr(q), n_chan, n_spec, n_input, s0, count, _ptr(out),
                                                         _stream(stream)))
    return out


def drift_search(zp: torch.Tensor, cell: float, nfft: Sequence[int], freqs_hz, n_sigma: Optional[float] = None,
                 want_maps: bool = False, max_out: int = 1 << 20, stream=None, params: Optional[DetectParams] = None):
    """zp float [T][n_chan][N][N] (high-passed standardised sub-integration cubes).
    n_sigma: a fixed threshold; otherwise params (default Benjamini-Hochberg,
    alpha 0.01).  Returns (candidates CANDIDATE_DTYPE, signed drifts int32[, snr
    map, drift map])."""
    if params is None:
        params = detect_params(mode=DETECT_FIXED, nsigma=n_sigma) if n_sigma is not None else detect_params()
    _cuda(zp, torch.float32, "zp")
    T, n_chan, n, _ = zp.shape
    nf = _host(nfft, np.int32)
    fr = _host(freqs_hz, np.float64)
    ws = workspace(_lib.ovro_drift_workspace_size(n_chan, n, nf.size, nf.ctypes.data_as(ctypes.c_void_p)),
                   zp.device)
    snr = torch.empty((n_chan, n, n), dtype=torch.float32, device=zp.device) if want_maps else None
    drm = torch.empty((n_chan, n, n), dtype=torch.int32, device=zp.device) if want_maps else None
    out = np.zeros(max_out, CANDIDATE_DTYPE)
    dr = np.zeros(max_out, np.int32)
    n_out = ctypes.c_int(0)
    _check("ovro_drift_search", _lib.ovro_drift_search(
        _ptr(zp), T, n_chan, n, float(cell), nf.size, nf.ctypes.data_as(ctypes.c_void_p),
        fr.ctypes.data_as(ctypes.c_void_p), ctypes.byref(params), _ptr(snr), _ptr(drm),
        out.ctypes.data_as(ctypes.c_void_p),
        dr.ctypes.data_as(ctypes.c_void_p), max_out, ctypes.byref(n_out), _ptr(ws), ws.numel(), _stream(stream)))
    k = n_out.value
    return (out[:k], dr[:k], snr, drm) if want_maps else (out[:k], dr[:k])


def detect_stats(img: torch.Tensor, cell: float, stream=None) -> torch.Tensor:
    _cuda(img, torch.float32, "img")
    n_chan, n, _ = img.shape
    stats = torch.empty((n_chan, 2), dtype=torch.float64, device=img.device)
    ws = workspace(detect_workspace_size(n_chan, n, [n_chan]), img.device)
    _check("ovro_detect_stats", _lib.ovro_detect_stats(_ptr(img), n_chan, n, float(cell), _ptr(stats), _ptr(ws),
                                                       ws.numel(), _stream(stream)))
    return stats


def detect_filter(img: torch.Tensor, stats: torch.Tensor, cell: float, nfft: Sequence[int],
                  params: Optional[DetectParams] = None, want_zp: bool = False, stream=None):
    """Returns (zp or None, snr, width), each [n_chan][N][N]."""
    _cuda(img, torch.float32, "img")
    _cuda(stats, torch.float64, "stats")
    n_chan, n, _ = img.shape
    nf = _host(nfft, np.int32)
    prm = params or detect_params()
    zp = torch.empty_like(img) if want_zp else None
    snr = torch.empty_like(img)
    wid = torch.empty(img.shape, dtype=torch.int32, device=img.device)
    ws = workspace(detect_workspace_size(n_chan, n, nf), img.device)
    _check("ovro_detect_filter", _lib.ovro_detect_filter(
        _ptr(img), _ptr(stats), n_chan, n, float(cell), len(nf), nf.ctypes.data_as(ctypes.c_void_p),
        ctypes.byref(prm), _ptr(zp), _ptr(snr), _ptr(wid), _ptr(ws), ws.numel(), _stream(stream)))
    return zp, snr, wid


# ------------------------------------------------------------------------ a13
def scorer_n_params() -> int:
    return int(_lib.ovro_scorer_n_params())


def scorer_cutouts(zp: torch.Tensor, nfft: Sequence[int], trig: torch.Tensor, stream=None) -> torch.Tensor:
    """zp float [n_chan][N][N]; trig int32 [n][3] (channel, row, col) -> [n][1600]."""
    _cuda(zp, torch.float32, "zp")
    _cuda(trig, torch.int32, "trig")
    n_chan, n, _ = zp.shape
    nf = _host(nfft, np.int32)
    x = torch.empty((trig.shape[0], 1600), dtype=torch.float32, device=zp.device)
    ws = workspace(_lib.ovro_scorer_workspace_size(1, len(nf)), zp.device)
    _check("ovro_scorer_cutouts", _lib.ovro_scorer_cutouts(
        _ptr(zp), n_chan, n, len(nf), nf.ctypes.data_as(ctypes.c_void_p), _ptr(trig), trig.shape[0], _ptr(x),
        _ptr(ws), ws.numel(), _stream(stream)))
    return x


def scorer_forward(w_bf16: torch.Tensor, x: torch.Tensor, ws: Optional[torch.Tensor] = None, stream=None):
    _cuda(w_bf16, torch.bfloat16, "w_bf16")
    _cuda(x, torch.float32, "x")
    B = x.shape[0]
    logit = torch.empty(B, dtype=torch.float32, device=x.device)
    need = _lib.ovro_scorer_workspace_size(B, 1)
    ws = ws if ws is not None and ws.numel() >= need else workspace(need, x.device)
    _check("ovro_scorer_forward", _lib.ovro_scorer_forward(_ptr(w_bf16), _ptr(x), B, _ptr(logit), _ptr(ws),
                                                           ws.numel(), _stream(stream)))
    return logit


def scorer_grad(w: torch.Tensor, x: torch.Tensor, y: torch.Tensor, ws: Optional[torch.Tensor] = None,
                stream=None):
    """Returns (grad float [n_params], loss float [1]); w is BF16 or FP32."""
    _cuda(x, torch.float32, "x")
    _cuda(y, torch.float32, "y")
    if not (w.is_cuda and w.is_contiguous() and w.dtype in (torch.bfloat16, torch.float32)):
        raise ValueError("w must be a contiguous CUDA bf16 or float32 tensor")
    B = x.shape[0]
    g = torch.empty(scorer_n_params(), dtype=torch.float32, device=x.device)
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    need = _lib.ovro_scorer_workspace_size(B, 1)
    ws = ws if ws is not None and ws.numel() >= need else workspace(need, x.device)
    _check("ovro_scorer_grad", _lib.ovro_scorer_grad(_ptr(w), 1 if w.dtype == torch.bfloat16 else 0, _ptr(x),
                                                     _ptr(y), B, _ptr(g), _ptr(loss), _ptr(ws), ws.numel(),
                                                     _stream(stream)))
    return g, loss


def scorer_adam(master: torch.Tensor, m: torch.Tensor, v: torch.Tensor, grad: torch.Tensor, step: int,
                lr: float, w_bf16: Optional[torch.Tensor] = None, stream=None):
    _check("ovro_scorer_adam", _lib.ovro_scorer_adam(_ptr(master), _ptr(m), _ptr(v), _ptr(grad), step,
                                                     float(lr), _ptr(w_bf16), _stream(stream)))


def scorer_to_bf16(master: torch.Tensor, w_bf16: torch.Tensor, stream=None):
    _check("ovro_scorer_to_bf16", _lib.ovro_scorer_to_bf16(_ptr(master), _ptr(w_bf16), _stream(stream)))


# ---------------------------------------------------------------------- a14
class PipelineConfig(ctypes.Structure):
    _fields_ = [("n_ant", ctypes.c_int), ("n_coarse", ctypes.c_int), ("h_nfft", ctypes.c_void_p),
                ("h_coarse_hz", ctypes.c_void_p), ("n_time", ctypes.c_int64), ("h_ant_enu_m", ctypes.c_void_p),
                ("image_size", ctypes.c_int), ("cell_dircos", ctypes.c_double), ("xeng_mode", ctypes.c_int),
                ("detect", DetectParams), ("use_graph", ctypes.c_int)]


class Pipeline:
    """Batched driver (ovro_pipeline_*): streams the coarse channels of an
    integration through fixed buffers and returns the candidates of the whole
    integration.  Owns its device workspace (a torch tensor)."""

    def __init__(self, n_ant: int, nfft: Sequence[int], coarse_hz: Sequence[float], n_time: int, ant_enu_m,
                 image_size: int, cell: float, xeng_mode: int = XENG_TC, params: Optional[DetectParams] = None,
                 use_graph: bool = True, device=None, stream=None):
        self._nf = _host(nfft, np.int32)
        self._hz = _host(coarse_hz, np.float64)
        self._ant = _host(ant_enu_m, np.float64).reshape(-1, 3)
        if self._hz.size != self._nf.size or self._ant.shape[0] != n_ant:
            raise ValueError("nfft / coarse_hz / ant_enu_m sizes disagree")
        self.params = params or detect_params()
        cfg = PipelineConfig(n_ant, self._nf.size, self._nf.ctypes.data, self._hz.ctypes.data, int(n_time),
                             self._ant.ctypes.data, image_size, float(cell), xeng_mode, self.params,
                             1 if use_graph else 0)
        h = ctypes.c_void_p()
        _check("ovro_pipeline_create", _lib.ovro_pipeline_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self.n_time, self.n_input, self.n_coarse = int(n_time), 2 * n_ant, int(self._nf.size)
        self.ws = workspace(_lib.ovro_pipeline_workspace_size(h), device)
        _check("ovro_pipeline_bind", _lib.ovro_pipeline_bind(h, _ptr(self.ws), self.ws.numel(), _stream(stream)))

    def channels(self) -> np.ndarray:
        n = _lib.ovro_pipeline_channels(self._h, None)
        f = np.zeros(n, np.float64)
        _lib.ovro_pipeline_channels(self._h, f.ctypes.data_as(ctypes.c_void_p))
        return f

    def run(self, volt: torch.Tensor, max_out: int = 1 << 20, stream=None) -> np.ndarray:
        _cuda(volt, torch.uint8, "volt")
        if volt.numel() != self.n_coarse * self.n_time * self.n_input:
            raise ValueError("volt must be [n_coarse][n_time][2 n_ant] uint8")
        # one host buffer per pipeline, its pages touched once (a fresh array
        # every run would fault its pages in again); the result is a copy
        if getattr(self, "_out", None) is None or self._out.size != max_out:
            self._out = np.zeros(max_out, CANDIDATE_DTYPE)
        out = self._out
        n_out = ctypes.c_int(0)
        _check("ovro_pipeline_run", _lib.ovro_pipeline_run(self._h, _ptr(volt), out.ctypes.data_as(ctypes.c_void_p),
                                                           max_out, ctypes.byref(n_out), _stream(stream)))
        return out[: min(n_out.value, max_out)].copy()

    def run_device(self, volt: torch.Tensor, stream=None) -> None:
        """The device part of one integration (before the threshold); read the
        search with search() and threshold it, possibly across shards."""
        _cuda(volt, torch.uint8, "volt")
        if volt.numel() != self.n_coarse * self.n_time * self.n_input:
            raise ValueError("volt must be [n_coarse][n_time][2 n_ant] uint8")
        _check("ovro_pipeline_run_device", _lib.ovro_pipeline_run_device(self._h, _ptr(volt), _stream(stream)))

    def search(self) -> "Search":
        """The whole integration's search (a view; valid while the pipeline lives)."""
        h = ctypes.c_void_p()
        _check("ovro_pipeline_search", _lib.ovro_pipeline_search(self._h, ctypes.byref(h)))
        return Search._view(h, self._nf, self.params, owner=self)

    def stats(self):
        k = ctypes.c_longlong(0)
        g = ctypes.c_int(0)
        _check("ovro_pipeline_stats", _lib.ovro_pipeline_stats(self._h, ctypes.byref(k), ctypes.byref(g)))
        return int(k.value), bool(g.value)

    def gridded(self, stream=None) -> int:
        """Cross visibilities the last run gridded (summed over channels)."""
        n = ctypes.c_longlong(0)
        _check("ovro_pipeline_gridded", _lib.ovro_pipeline_gridded(self._h, ctypes.byref(n), _stream(stream)))
        return int(n.value)

    def close(self):
        if getattr(self, "_h", None):
            _lib.ovro_pipeline_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def autotune(enable: bool) -> None:
    _check("ovro_autotune", _lib.ovro_autotune(1 if enable else 0))


def tune_get(key: str) -> Optional[int]:
    v = ctypes.c_int(0)
    return int(v.value) if _lib.ovro_tune_get(key.encode(), ctypes.byref(v)) == OVRO_OK else None


def tune_set(key: str, value: int) -> None:
    _check("ovro_tune_set", _lib.ovro_tune_set(key.encode(), int(value)))


def tune_count() -> int:
    return int(_lib.ovro_tune_count())


def tune_clear() -> None:
    _check("ovro_tune_clear", _lib.ovro_tune_clear())


def tune_save(path: str) -> None:
    _check("ovro_tune_save", _lib.ovro_tune_save(os.fspath(path).encode()))


def tune_load(path: str) -> None:
    _check("ovro_tune_load", _lib.ovro_tune_load(os.fspath(path).encode()))


# ------------------------------------------------------- sharded search (a11)
class Search:
    """One shard of a Stage I search (ovro_search_*): add coarse-channel image
    blocks, read the SNR histogram and bin values, then NMS at a given cut."""

    def __init__(self, n_chan: int, image_size: int, cell: float, nfft: Sequence[int],
                 params: Optional[DetectParams] = None, device=None, stream=None):
        self._nf = _host(nfft, np.int32)
        self.params = params or detect_params()
        self.ws = workspace(detect_workspace_size(n_chan, image_size, self._nf), device)
        h = ctypes.c_void_p()
        _check("ovro_search_create", _lib.ovro_search_create(
            n_chan, image_size, float(cell), self._nf.size, self._nf.ctypes.data_as(ctypes.c_void_p),
            ctypes.byref(self.params), _ptr(self.ws), self.ws.numel(), _stream(stream), ctypes.byref(h)))
        self._h = h
        self._layout()

    @classmethod
    def _view(cls, h, nfft, params, owner):
        s = cls.__new__(cls)
        s._nf, s.params, s._h, s._owner = nfft, params, h, owner
        s._layout()
        return s

    def _layout(self):
        k0, nb, nt = ctypes.c_uint32(0), ctypes.c_int(0), ctypes.c_longlong(0)
        _check("ovro_search_layout", _lib.ovro_search_layout(self._h, ctypes.byref(k0), ctypes.byref(nb),
                                                             ctypes.byref(nt)))
        self.key0, self.n_bins, self.n_tests = int(k0.value), int(nb.value), int(nt.value)

    def reset(self, stream=None):
        _check("ovro_search_reset", _lib.ovro_search_reset(self._h, _stream(stream)))

    def add(self, coarse: int, img_block: torch.Tensor, stream=None):
        _cuda(img_block, torch.float32, "img_block")
        _check("ovro_search_add", _lib.ovro_search_add(self._h, coarse, _ptr(img_block), _stream(stream)))

    def histogram(self, stream=None) -> np.ndarray:
        h = np.zeros(self.n_bins, np.uint64)
        _check("ovro_search_histogram", _lib.ovro_search_histogram(self._h, h.ctypes.data_as(ctypes.c_void_p),
                                                                   self.n_bins, _stream(stream)))
        return h

    def bin_values(self, b: int, stream=None) -> np.ndarray:
        n = ctypes.c_longlong(0)
        st = _lib.ovro_search_bin_values(self._h, b, None, 0, ctypes.byref(n), _stream(stream))
        if st not in (OVRO_OK, -7):
            _check("ovro_search_bin_values", st)
        v = np.zeros(n.value, np.float32)
        if n.value:
            _check("ovro_search_bin_values", _lib.ovro_search_bin_values(
                self._h, b, v.ctypes.data_as(ctypes.c_void_p), n.value, ctypes.byref(n), _stream(stream)))
        return v

    def candidates(self, cut: float, freqs_hz, max_out: int = 1 << 20, stream=None) -> np.ndarray:
        fr = _host(freqs_hz, np.float64)
        out = np.zeros(max_out, CANDIDATE_DTYPE)
        n_out = ctypes.c_int(0)
        _check("ovro_search_candidates", _lib.ovro_search_candidates(
            self._h, ctypes.c_float(cut), fr.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p),
            max_out, ctypes.byref(n_out), _stream(stream)))
        return out[: n_out.value]

    def close(self):
        if getattr(self, "_h", None):
            _lib.ovro_search_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def bh_layout(params: Optional[DetectParams] = None):
    k0, nb = ctypes.c_uint32(0), ctypes.c_int(0)
    _check("ovro_bh_layout", _lib.ovro_bh_layout(ctypes.byref(params or detect_params()), ctypes.byref(k0),
                                                 ctypes.byref(nb)))
    return int(k0.value), int(nb.value)


def bh_bin_verdict(hist: np.ndarray, key0: int, n_tests: float, alpha: float, b: int):
    h = np.ascontiguousarray(hist, np.uint64)
    lo, above = ctypes.c_float(0), ctypes.c_ulonglong(0)
    v = _lib.ovro_bh_bin_verdict(h.ctypes.data_as(ctypes.c_void_p), h.size, key0, float(n_tests), float(alpha), b,
                                 ctypes.byref(lo), ctypes.byref(above))
    if v < 0:
        _check("ovro_bh_bin_verdict", v)
    return v, float(lo.value), int(above.value)


def bh_resolve(vals_desc: np.ndarray, above_next: int, n_tests: float, alpha: float) -> Optional[float]:
    v = np.ascontiguousarray(vals_desc, np.float32)
    cut = ctypes.c_float(0)
    r = _lib.ovro_bh_resolve(v.ctypes.data_as(ctypes.c_void_p), v.size, above_next, float(n_tests), float(alpha),
                             ctypes.byref(cut))
    if r < 0:
        _check("ovro_bh_resolve", r)
    return float(cut.value) if r == 1 else None


def snr_bin_key(snr: float) -> int:
    return int(_lib.ovro_snr_bin_key(ctypes.c_float(snr)))
