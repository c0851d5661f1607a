"""Training and serving driver of the learned candidate scorer.

Orchestration only: every computation runs in libovro.so (the pipeline calls,
ovro_scorer_cutouts / _forward / _grad / _adam).  Random numbers the training
draws (initial weights, batch order) come from a seeded NumPy generator and are
passed in.

The scorer proposes which Stage I triggers to keep; the plain threshold
detector remains the fallback and the reference its recall and false-alarm
rate are measured against.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Sequence

import numpy as np
import torch

from . import ovro


@dataclass
class Cube:
    img: torch.Tensor        # [n_chan][N][N] dirty images
    zp: torch.Tensor         # [n_chan][N][N] high-passed standardised cube
    nfft: List[int]
    freqs: np.ndarray
    cell: float


def run_pipeline(volt: np.ndarray, nfft: Sequence[int], n_ant: int, pos: np.ndarray, freqs: np.ndarray,
                 image_size: int, cell: float) -> Cube:
    """Voltages -> images -> high-passed cube, all on the GPU."""
    d = torch.from_numpy(volt).cuda()
    n_coarse, n_time, n_input = volt.shape
    q, _ = ovro.upchan(d, nfft)
    n_chan = int(sum(nfft))
    vis = torch.empty((n_chan, ovro.n_baselines(n_ant), 4, 2), dtype=torch.int32, device="cuda")
    qoff, c0 = 0, 0
    for n in nfft:
        k = n_time // n
        m = n * k * n_input * 2
        ovro.correlate(q[qoff:qoff + m], n_ant, n, k, ovro.XENG_TC, out=vis[c0:c0 + n])
        qoff += m
        c0 += n
    img = ovro.grid_image(vis, pos, freqs, image_size, cell)
    stats = ovro.detect_stats(img, cell)
    zp, _, _ = ovro.detect_filter(img, stats, cell, nfft, want_zp=True)
    return Cube(img, zp, list(nfft), freqs, cell)


def run_pipeline_streamed(volt: np.ndarray, nfft: Sequence[int], n_ant: int, pos: np.ndarray, freqs: np.ndarray,
                          image_size: int, cell: float) -> Cube:
    """As run_pipeline, one coarse channel at a time through one visibility
    buffer (the whole integration's visibilities need not fit on the device)."""
    n_coarse, n_time, n_input = volt.shape
    n_chan = int(sum(nfft))
    img = torch.empty((n_chan, image_size, image_size), dtype=torch.float32, device="cuda")
    vis = torch.empty((max(nfft), ovro.n_baselines(n_ant), 4, 2), dtype=torch.int32, device="cuda")
    c0 = 0
    for c, n in enumerate(nfft):
        d = torch.from_numpy(np.ascontiguousarray(volt[c:c + 1])).cuda()
        k = n_time // n
        q, _ = ovro.upchan(d, [n])
        ovro.correlate(q, n_ant, n, k, ovro.XENG_TC, out=vis[:n])
        ovro.grid_image(vis[:n], pos, freqs[c0:c0 + n], image_size, cell, out=img[c0:c0 + n])
        c0 += n
    del vis
    bounds = np.concatenate([[0], np.cumsum(nfft)])
    stats = torch.cat([ovro.detect_stats(img[bounds[c]:bounds[c + 1]], cell) for c in range(len(nfft))])
    zp, _, _ = ovro.detect_filter(img, stats, cell, nfft, want_zp=True)
    return Cube(img, zp, list(nfft), freqs, cell)


def label(cands: np.ndarray, tones, nfft: Sequence[int], n_time: int, f_coarse: float = 24000.0,
          pix_tol: int = 1, chan_tol: int = 2) -> np.ndarray:
    """1 where a candidate is an injected sky tone: same coarse channel, within
    pix_tol pixels of its position and within its drift span (+- chan_tol)."""
    y = np.zeros(len(cands), np.float32)
    T = n_time / f_coarse
    for t in tones:
        df = f_coarse / nfft[t.coarse]
        span = t.drift_hz_s * T / df
        lo, hi = t.fine - chan_tol, t.fine + span + chan_tol
        hit = ((cands["coarse"] == t.coarse) & (cands["fine"] >= lo) & (cands["fine"] <= hi) &
               (np.abs(cands["row"] - t.row) <= pix_tol) & (np.abs(cands["col"] - t.col) <= pix_tol))
        y[hit] = 1.0
    return y


def candidates(cube: Cube, nsigma: float) -> np.ndarray:
    return ovro.detect(cube.img, cube.cell, cube.nfft, cube.freqs,
                       ovro.detect_params(mode=ovro.DETECT_FIXED, nsigma=nsigma))


def cutouts(cube: Cube, cands: np.ndarray) -> torch.Tensor:
    trig = np.stack([cands["chan"], cands["row"], cands["col"]], axis=1).astype(np.int32)
    return ovro.scorer_cutouts(cube.zp, cube.nfft, torch.from_numpy(np.ascontiguousarray(trig)).cuda())


@dataclass
class Scorer:
    master: torch.Tensor     # FP32 master weights
    w_bf16: torch.Tensor     # BF16 serving copy
    losses: List[float]


def init_weights(seed: int) -> np.ndarray:
    """He-style initial weights for 1600 -> 128 -> 32 -> 1 (biases 0)."""
    g = np.random.default_rng(seed)
    parts = []
    for i, o in ((1600, 128), (128, 32), (32, 1)):
        parts.append(g.normal(0.0, math.sqrt(2.0 / i), o * i))
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)


def train(x: torch.Tensor, y: torch.Tensor, epochs: int = 30, batch: int = 256, lr: float = 1e-3,
          seed: int = 0, pos_weight: float = 1.0) -> Scorer:
    """Mini-batch Adam on the GPU kernels.  pos_weight > 1 repeats positives in
    every epoch's batch order to balance rare classes."""
    n = x.shape[0]
    master = torch.from_numpy(init_weights(seed)).cuda()
    m = torch.zeros_like(master)
    v = torch.zeros_like(master)
    wb = torch.empty(master.numel(), dtype=torch.bfloat16, device="cuda")
    ovro.scorer_to_bf16(master, wb)
    g = np.random.default_rng(seed + 1)
    yh = y.cpu().numpy()
    base = np.arange(n)
    if pos_weight > 1.0:
        pos = np.nonzero(yh > 0.5)[0]
        base = np.concatenate([base] + [pos] * (int(round(pos_weight)) - 1))
    ws = ovro.workspace(ovro.lib().ovro_scorer_workspace_size(batch, 1))
    step, losses = 0, []
    for _ in range(epochs):
        order = torch.from_numpy(g.permutation(base)).cuda()
        tot, cnt = 0.0, 0
        for b0 in range(0, len(order) - batch + 1, batch):
            idx = order[b0:b0 + batch]
            xb, yb = x[idx].contiguous(), y[idx].contiguous()
            grad, loss = ovro.scorer_grad(wb, xb, yb, ws=ws)
            step += 1
            ovro.scorer_adam(master, m, v, grad, step, lr, wb)
            tot += float(loss.item())
            cnt += 1
        losses.append(tot / max(cnt, 1))
    return Scorer(master, wb, losses)


def score(s: Scorer, x: torch.Tensor) -> np.ndarray:
    """Keep probabilities sigma(logit) of the BF16-served network."""
    if x.shape[0] == 0:
        return np.zeros(0)
    logit = ovro.scorer_forward(s.w_bf16, x).cpu().numpy().astype(np.float64)
    return 1.0 / (1.0 + np.exp(-logit))


def roc_auc(score_: np.ndarray, y: np.ndarray) -> float:
    """Area under the ROC curve (probability a positive outranks a negative)."""
    pos, neg = score_[y > 0.5], score_[y <= 0.5]
    if len(pos) == 0 or len(neg) == 0:
        return float("nan")
    order = np.argsort(np.concatenate([pos, neg]), kind="mergesort")
    ranks = np.empty(len(order))
    ranks[order] = np.arange(1, len(order) + 1)
    return float((ranks[: len(pos)].sum() - len(pos) * (len(pos) + 1) / 2) / (len(pos) * len(neg)))
