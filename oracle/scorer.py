"""Oracle: learned candidate scorer (not in the paper; the narrowband search of
Section 2.4 keeps or drops triggers by threshold alone).

A small multilayer perceptron scores cutouts of the high-passed standardised
cube around a trigger (64 fine channels x 5 x 5 pixels) and proposes which
candidates to keep.  Everything here is FP64:

* cutout(t)  = z'[k - 32 .. k + 31][r - 2 .. r + 2][c - 2 .. c + 2] for a trigger
  t = (channel k, row r, col c), flattened channel-major; entries outside the
  trigger's coarse channel or outside the image are 0.
* forward:   h_l = GELU(W_l h_{l-1} + b_l) for the hidden layers, logit =
  W_L h_{L-1} + b_L; GELU(x) = x Phi(x) (exact, erf form).
* loss:      mean binary cross-entropy with logits,
             softplus(z) - y z = max(z, 0) - y z + log(1 + exp(-|z|)).
* backward:  the chain rule written out layer by layer (GELU'(x) = Phi(x) + x phi(x)).
* Adam:      m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
             w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
* Weights are served in BF16 (round to nearest even of the FP32 master
  weights); the oracle evaluates the network with those BF16 values.

Parameters are one flat vector, layer by layer: W_l row-major [out][in], then b_l.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

LAYERS = (1600, 128, 32, 1)
CUT_CH = 64
CUT_PIX = 5


def n_params(layers=LAYERS) -> int:
    return sum(o * i + o for i, o in zip(layers[:-1], layers[1:]))


def unpack(theta: np.ndarray, layers=LAYERS):
    out, off = [], 0
    for i, o in zip(layers[:-1], layers[1:]):
        W = theta[off:off + o * i].reshape(o, i)
        off += o * i
        b = theta[off:off + o]
        off += o
        out.append((W, b))
    return out


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    phi = np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * phi


def forward(theta, X, layers=LAYERS):
    """Logits [B] and the pre-activations / activations needed by backward."""
    params = unpack(np.asarray(theta, dtype=np.float64), layers)
    h = np.asarray(X, dtype=np.float64)
    acts, pres = [h], []
    for li, (W, b) in enumerate(params):
        z = h @ W.T + b
        pres.append(z)
        h = gelu(z) if li < len(params) - 1 else z
        acts.append(h)
    return h[:, 0], (acts, pres)


def bce(logits, y) -> float:
    z = np.asarray(logits, dtype=np.float64)
    return float(np.mean(np.maximum(z, 0.0) - y * z + np.log1p(np.exp(-np.abs(z)))))


def backward(theta, X, y, layers=LAYERS):
    """(flat gradient of the mean BCE loss, loss)."""
    params = unpack(np.asarray(theta, dtype=np.float64), layers)
    logits, (acts, pres) = forward(theta, X, layers)
    B = X.shape[0]
    sig = 1.0 / (1.0 + np.exp(-logits))
    delta = ((sig - y) / B)[:, None]               # dL/dlogit
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        grads[li] = (delta.T @ acts[li], delta.sum(axis=0))
        if li > 0:
            delta = (delta @ W) * gelu_grad(pres[li - 1])
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return flat, bce(logits, y)


def adam(theta, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def bf16_round(x) -> np.ndarray:
    """Round FP32 values to the nearest BF16 (ties to even); returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed: int, layers=LAYERS) -> np.ndarray:
    """He-style initialisation (FP32 master weights); biases 0."""
    g = np.random.default_rng(seed)
    parts = []
    for i, o in zip(layers[:-1], layers[1:]):
        parts.append(g.normal(0.0, math.sqrt(2.0 / i), o * i))
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32).astype(np.float64)


def cutouts(zp, chan_bounds, trig, n_ch=CUT_CH, n_pix=CUT_PIX) -> np.ndarray:
    """zp: [n_chan][N][N]; trig: [n][3] (channel, row, col).  Returns [n][n_ch*n_pix*n_pix]."""
    n_chan, N, _ = zp.shape
    half_c, half_p = n_ch // 2, n_pix // 2
    out = np.zeros((len(trig), n_ch, n_pix, n_pix))
    for t, (k, r, c) in enumerate(trig):
        lo, hi = next((a, b) for a, b in chan_bounds if a <= k < b)
        for i in range(n_ch):
            kk = k - half_c + i
            if kk < lo or kk >= hi:
                continue
            for dr in range(n_pix):
                rr = r - half_p + dr
                if rr < 0 or rr >= N:
                    continue
                for dc in range(n_pix):
                    cc = c - half_p + dc
                    if 0 <= cc < N:
                        out[t, i, dr, dc] = zp[kk, rr, cc]
    return out.reshape(len(trig), -1)
