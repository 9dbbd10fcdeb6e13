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


def antisymmetrised(g):
    """Derivative along the independent amplitudes t_ij^ab (i<j, a<b) from an array-element gradient."""
    o, v = g.shape[0], g.shape[2]
    out = np.zeros_like(g)
    for i in range(o):
        for j in range(i + 1, o):
            for a in range(v):
                for b in range(a + 1, v):
                    out[i, j, a, b] = g[i, j, a, b] - g[j, i, a, b] - g[i, j, b, a] + g[j, i, b, a]
    return out


@pytest.mark.parametrize("o,v,seed", [(3, 5, 11), (4, 8, 1001)])
def test_t2_gradient_matches_oracle(torch, o, v, seed):
    """dL/dt2 (L = Re sum conj(Gbar) G) by the adjoint method on the GPU against the oracle's chain rule
    with exact operator derivatives, at random (not MP2-like) amplitudes, with occupied and virtual
    orbitals in both sets (so that b_a and c_i contribute)."""
    import synth
    from paper_1902_06016_gb300 import Context
    inp = synth.random_amplitudes(inputs(o, v, seed), seed + 3)
    porb, qorb = list(range(o + 3)), [0, o - 1, o, o + 2]
    ws, eta = np.array([-0.8, -0.45, -0.1]), 0.05
    rng = np.random.default_rng(seed)
    Gb = rng.standard_normal((3, len(porb), len(qorb))) + 1j * rng.standard_normal((3, len(porb), len(qorb)))
    ctx = Context(inp, tol=1e-12)
    G, g = ctx.green_grad_t2(ws, eta, porb, Gb, qorb)
    go = grad.green_t2_gradient(inp, porb, qorb, ws, eta, Gb)
    assert rel_err(antisymmetrised(g), go) <= 1e-7
    M = sg.dense_matrix(hbar.build(inp))
    Go = grad.derivatives(M, bc.b_vectors(inp, porb), bc.c_vectors(inp, qorb), ws, eta)[0]
    assert rel_err(G, Go) <= 1e-9


def test_autograd_t2_gradient(torch):
    """The autograd Function returns dL/dt2 for a real loss of G (here sum_w A(w)^2 weighted)."""
    import synth
    from paper_1902_06016_gb300 import Context
    from paper_1902_06016_gb300.autograd import green, spectral
    inp = synth.random_amplitudes(inputs(3, 5, 11), 14)
    porb = [0, 1, 2]
    ctx = Context(inp, tol=1e-12)
    w = torch.tensor([-0.7, -0.3], dtype=torch.float64)
    eta = torch.tensor(0.05, dtype=torch.float64)
    t2 = torch.tensor(inp.t2, dtype=torch.float64, requires_grad=True)
    loss = (spectral(green(w, eta, ctx, porb, t2=t2)) ** 2).sum()
    loss.backward()
    g = antisymmetrised(t2.grad.numpy())
    # the same loss by finite differences of the oracle along two amplitudes
    def L(inp2):
        Mx = sg.dense_matrix(hbar.build(inp2))
        Gx = grad.derivatives(Mx, bc.b_vectors(inp2, porb), bc.c_vectors(inp2, porb), w.numpy(), 0.05)[0]
        A = -np.imag(np.einsum("wpp->w", Gx)) / np.pi
        return float((A ** 2).sum())
    h = 1e-5
    for (i, j, a, b) in [(0, 1, 0, 1), (1, 2, 2, 4)]:
        d = (L(grad._perturbed(inp, i, j, a, b, h)) - L(grad._perturbed(inp, i, j, a, b, -h))) / (2 * h)
        assert abs(d - g[i, j, a, b]) <= 1e-6 * np.abs(g).max()


@pytest.mark.parametrize("prec,hi", [("tf32", 2.0 ** -12), ("bf16", 2.0 ** -9)])
@pytest.mark.parametrize("o,v,seed", [(4, 8, 1001), (7, 13, 103)])
def test_transposed_tensor_core_sigma(torch, prec, hi, o, v, seed):
    """M^T X on the tensor cores: the low-precision transposed sigma within its operand rounding, and the
    exact-slice transposed sigma to FP64 level, against X M from the oracle's dense matrix."""
    from paper_1902_06016_gb300 import Context
    from gpu_util import random_vectors
    inp = inputs(o, v, seed)
    M = sg.dense_matrix(hbar.build(inp))
    X = random_vectors(inp.dim, 5, seed + 9)
    ref = X @ M
    ctx = Context(inp, precision=prec)
    err = rel_err(ctx.sigma(X, precision=prec, transpose=True), ref)
    assert 1e-7 < err < hi, err
    Y = ctx.sigma(X, precision="fp64_tc", transpose=True)
    for k in range(5):
        assert np.abs(Y[k] - ref[k]).max() <= 1e-12 * np.abs(ref[k]).max()


@pytest.mark.parametrize("o,v,seed", [(4, 8, 1001), (7, 13, 103)])
def test_adjoint_solves_on_tensor_cores_match_oracle(torch, o, v, seed):
    """A TF32 context runs the adjoint (transposed) solves of dG/dw, dG/deta and dL/dt2 as GMRES-IR with
    the TF32 transposed sigma and exact-slice residuals; results as accurate as the FP64 path."""
    import synth
    from paper_1902_06016_gb300 import Context
    inp = inputs(o, v, seed)
    M = sg.dense_matrix(hbar.build(inp))
    porb, qorb = list(range(o + 2)), [0, 2, o + 1]
    ws = np.linspace(-1.0, -0.1, 5)
    ctx = Context(inp, tol=1e-11, precision="tf32")
    G, dw, de = ctx.green_derivatives(ws, 0.02, porb, qorb)
    Go, dwo, deo = grad.derivatives(M, bc.b_vectors(inp, porb), bc.c_vectors(inp, qorb), ws, 0.02)
    assert rel_err(G, Go) <= 1e-8 and rel_err(dw, dwo) <= 1e-8 and rel_err(de, deo) <= 1e-8
    inp2 = synth.random_amplitudes(inputs(3, 5, 11), 14)
    p2, q2 = [0, 1, 2, 3], [0, 2, 4]
    w2, eta2 = np.array([-0.8, -0.45, -0.1]), 0.05
    rng = np.random.default_rng(3)
    Gb = rng.standard_normal((3, 4, 3)) + 1j * rng.standard_normal((3, 4, 3))
    ctx2 = Context(inp2, tol=1e-11, precision="tf32")
    _, g = ctx2.green_grad_t2(w2, eta2, p2, Gb, q2)
    assert rel_err(antisymmetrised(g), grad.green_t2_gradient(inp2, p2, q2, w2, eta2, Gb)) <= 1e-7
