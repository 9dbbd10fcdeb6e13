"""Adjoint derivatives of G_pq(w) on the GPU (row a10) against the oracle's closed forms and finite
differences (needs a GB300)."""
import numpy as np
import pytest

from oracle import bc, grad, hbar
from oracle import sigma as sg

from gpu_util import inputs, need_gpu, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


@pytest.mark.parametrize("o,v,seed", [(4, 8, 1001), (7, 13, 103)])
def test_green_derivatives_match_oracle(torch, o, v, seed):
    from paper_1902_06016_gb300 import Context
    inp = inputs(o, v, seed)
    M = sg.dense_matrix(hbar.build(inp))
    porb, qorb = list(range(o + 2)), [0, 2, o + 1]
    ws = np.linspace(-1.0, -0.1, 5)
    ctx = Context(inp, tol=1e-11)
    G, dw, de = ctx.green_derivatives(ws, 0.02, porb, qorb)
    Go, dwo, deo = grad.derivatives(M, bc.b_vectors(inp, porb), bc.c_vectors(inp, qorb), ws, 0.02)
    assert rel_err(G, Go) <= 1e-8
    assert rel_err(dw, dwo) <= 1e-8
    assert rel_err(de, deo) <= 1e-8


def test_autograd_matches_finite_differences(torch):
    from paper_1902_06016_gb300 import Context
    from paper_1902_06016_gb300.autograd import green, spectral
    inp = inputs(4, 8, 1001)
    ctx = Context(inp, tol=1e-12)
    porb = [0, 1, 2, 3]
    w = torch.tensor([-0.8, -0.5, -0.3], dtype=torch.float64, requires_grad=True)
    eta = torch.tensor(0.02, dtype=torch.float64, requires_grad=True)
    loss = (spectral(green(w, eta, ctx, porb)) ** 2).sum() + green(w, eta, ctx, porb).abs().pow(2).sum()
    loss.backward()

    def f(wv, ev):
        with torch.no_grad():
            wt = torch.tensor(wv, dtype=torch.float64)
            et = torch.tensor(ev, dtype=torch.float64)
            G = green(wt, et, ctx, porb)
            return float((spectral(G) ** 2).sum() + G.abs().pow(2).sum())

    h = 1e-5
    base = w.detach().numpy()
    fd_w = []
    for k in range(3):
        wp, wm = base.copy(), base.copy()
        wp[k] += h
        wm[k] -= h
        fd_w.append((f(wp, 0.02) - f(wm, 0.02)) / (2 * h))
    fd_e = (f(base, 0.02 + h) - f(base, 0.02 - h)) / (2 * h)
    assert np.allclose(w.grad.numpy(), fd_w, rtol=1e-5, atol=1e-8)
    assert abs(eta.grad.item() - fd_e) <= 1e-5 * abs(fd_e) + 1e-8
