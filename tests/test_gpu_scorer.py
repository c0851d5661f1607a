"""GPU parity: learned scorer kernels (cutouts, forward, gradients, Adam) against
the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import scorer as S

pytestmark = pytest.mark.gpu


def _theta(seed=0):
    return S.init_params(seed)


def _blocks(v):
    """Per-parameter-block views (W1, b1, W2, b2, W3, b3)."""
    out, off = [], 0
    for i, o in zip(S.LAYERS[:-1], S.LAYERS[1:]):
        out.append(v[off:off + o * i]); off += o * i
        out.append(v[off:off + o]); off += o
    return out


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


def test_cutouts_exact(lib):
    g = np.random.default_rng(0)
    n_chan, n = 300, 24
    nfft = [100, 200]
    zp = g.normal(size=(n_chan, n, n)).astype(np.float32)
    trig = np.array([[50, 10, 10], [99, 0, 23], [100, 23, 0], [299, 12, 1], [150, 2, 2]], np.int32)
    x = lib.scorer_cutouts(torch.from_numpy(zp).cuda(), nfft, torch.from_numpy(trig).cuda()).cpu().numpy()
    ref = S.cutouts(zp.astype(np.float64), [(0, 100), (100, 300)], trig)
    assert np.array_equal(x, ref.astype(np.float32))


def test_forward_and_gradients(lib):
    g = np.random.default_rng(1)
    B = 300
    x = g.normal(size=(B, 1600)).astype(np.float32)
    y = (g.uniform(size=B) < 0.4).astype(np.float32)
    theta = _theta(2) + g.normal(size=S.n_params()) * 0.01        # nonzero biases
    theta32 = theta.astype(np.float32)
    w32 = torch.from_numpy(theta32).cuda()
    wb = w32.to(torch.bfloat16)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    # BF16-served weights: oracle evaluated at the BF16 values
    tb = S.bf16_round(theta32)
    assert np.array_equal(tb, wb.to(torch.float64).cpu().numpy())
    logit = lib.scorer_forward(wb, xd).cpu().numpy()
    ref_logit, _ = S.forward(tb, x.astype(np.float64))
    assert _rel(logit, ref_logit) < 1e-5
    grad, loss = lib.scorer_grad(wb, xd, yd)
    ref_g, ref_loss = S.backward(tb, x.astype(np.float64), y.astype(np.float64))
    assert abs(loss.item() - ref_loss) < 1e-5 * max(1.0, ref_loss)
    for gb, rb in zip(_blocks(grad.cpu().numpy().astype(np.float64)), _blocks(ref_g)):
        assert _rel(gb, rb) < 1e-3
    # FP32 master weights
    grad32, _ = lib.scorer_grad(w32, xd, yd)
    ref32, _ = S.backward(theta32.astype(np.float64), x.astype(np.float64), y.astype(np.float64))
    for gb, rb in zip(_blocks(grad32.cpu().numpy().astype(np.float64)), _blocks(ref32)):
        assert _rel(gb, rb) < 1e-5


def test_adam_step(lib):
    g = np.random.default_rng(3)
    n = lib.scorer_n_params()
    w = g.normal(size=n).astype(np.float32)
    m = (g.normal(size=n) * 1e-3).astype(np.float32)
    v = (g.uniform(size=n) * 1e-4).astype(np.float32)
    gr = g.normal(size=n).astype(np.float32)
    dw, dm, dv, dg = (torch.from_numpy(a.copy()).cuda() for a in (w, m, v, gr))
    wb = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    lib.scorer_adam(dw, dm, dv, dg, 3, 1e-3, wb)
    rw, rm, rv = S.adam(w.astype(np.float64), m.astype(np.float64), v.astype(np.float64), gr.astype(np.float64),
                        3, 1e-3)
    assert _rel(dm.cpu().numpy(), rm) < 1e-6 and _rel(dv.cpu().numpy(), rv) < 1e-6
    assert np.abs(dw.cpu().numpy() - rw).max() < 1e-6
    assert torch.equal(wb, dw.to(torch.bfloat16))
