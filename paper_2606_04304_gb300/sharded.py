"""Stage I threshold across shards: coarse channels searched on several
processes (one GPU each), one Benjamini-Hochberg family over all of them.

Host logic only.  The shards' SNR histograms and test counts are summed, and
the values of a bin whose verdict the edges leave open are gathered, over a
torch.distributed process group on host tensors (gloo) -- no device
collective.  Every decision is the library's (ovro_bh_bin_verdict,
ovro_bh_resolve), so one shard reproduces ovro_detect exactly.
"""
from __future__ import annotations

from typing import Callable, List, Optional

import numpy as np
import torch
import torch.distributed as dist

from . import ovro


def _world(group) -> int:
    if not (dist.is_available() and dist.is_initialized()):
        return 1
    return dist.get_world_size(group)


def _sum(x: np.ndarray, group) -> np.ndarray:
    if _world(group) == 1:
        return x
    t = torch.from_numpy(np.ascontiguousarray(x, np.int64))
    dist.all_reduce(t, group=group)
    return t.numpy()


def _gather(v: np.ndarray, group) -> np.ndarray:
    w = _world(group)
    if w == 1:
        return v
    n = torch.tensor([v.size], dtype=torch.int64)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(w)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(s.item()) for s in sizes]
    top = max(sizes)
    if top == 0:
        return np.zeros(0, np.float32)
    buf = torch.zeros(top, dtype=torch.float32)
    buf[: v.size] = torch.from_numpy(np.ascontiguousarray(v, np.float32))
    parts = [torch.zeros(top, dtype=torch.float32) for _ in range(w)]
    dist.all_gather(parts, buf, group=group)
    return np.concatenate([p[:k].numpy() for p, k in zip(parts, sizes)])


def global_cut(hist_local: np.ndarray, key0: int, n_tests_local: int, params: ovro.DetectParams,
               bin_values: Callable[[int], np.ndarray], group=None,
               trace: Optional[List[int]] = None) -> Optional[float]:
    """The common SNR cut (None when Benjamini-Hochberg rejects nothing); the
    fixed threshold in fixed mode.  bin_values(b) returns this shard's SNR
    values in histogram bin b.  trace, if given, receives each bin's verdict."""
    if params.mode == ovro.DETECT_FIXED:
        return float(params.nsigma)
    hist = _sum(np.asarray(hist_local, np.int64), group).astype(np.uint64)
    m = float(_sum(np.array([n_tests_local], np.int64), group)[0])
    for b in range(hist.size):
        v, lo, above = ovro.bh_bin_verdict(hist, key0, m, params.alpha, b)
        if trace is not None:
            trace.append(v)
        if v in (0, 3):
            continue
        if v == 1:
            return lo
        vals = np.sort(_gather(bin_values(b), group))[::-1]
        if vals.size != int(hist[b]):
            raise RuntimeError(f"bin {b}: gathered {vals.size} values, histogram holds {int(hist[b])}")
        cut = ovro.bh_resolve(vals, above, m, params.alpha)
        if cut is not None:
            return cut
    return None


def sharded_detect(search: ovro.Search, freqs_hz, group=None, max_out: int = 1 << 20) -> np.ndarray:
    """a11-a12 for this shard's search at the cut common to every shard."""
    cut = global_cut(search.histogram(), search.key0, search.n_tests, search.params, search.bin_values, group)
    if cut is None:
        return np.zeros(0, ovro.CANDIDATE_DTYPE)
    return search.candidates(cut, freqs_hz, max_out=max_out)
