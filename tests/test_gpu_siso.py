"""Per-orbital (SISO) reduced models of G_pp on the GPU against the oracle's (needs a GB300).

Each model is the adaptive reduced model of one orbital p (input b_p, output c_p, subspace from
X_p(w_k) alone); the GPU solves all models' new frequencies in one batch per round. It must choose
the oracle's frequencies model by model, reach the same orders, and give the same Ghat_pp.
"""
import numpy as np
import pytest

from oracle import bc, hbar, mor
from oracle import sigma as sg
from oracle import solve as sv

from gpu_util import inputs, need_gpu, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


@pytest.mark.parametrize("o,v,seed,prec", [(4, 8, 1001, "fp64"), (7, 13, 103, "tf32")])
def test_siso_models_match_oracle(torch, o, v, seed, prec):
    from paper_1902_06016_gb300 import Context
    inp = inputs(o, v, seed)
    hb = hbar.build(inp)
    M = sg.dense_matrix(hb)
    porb = list(range(o)) + [o, o + 2]                 # occupied and two virtual orbitals
    B, C = bc.b_vectors(inp, porb), bc.c_vectors(inp, porb)
    wmin, wmax, eta, tol = -1.0, -0.2, 0.01, 1e-6
    seeds = np.linspace(wmin, wmax, 3)
    ctx = Context(inp, tol=1e-11, precision=prec)
    ctx.mor_build_siso(seeds, eta, porb)
    res = ctx.mor_refine(wmin, wmax, 301, tol, 10 ** 6)
    assert res["converged"] and res["max_err"] <= tol
    orc = mor.build_and_refine_siso(hb, B, C, seeds, wmin, wmax, 301, eta, tol, 10 ** 6, solver="dense", M=M)
    total = 0
    for k, r in enumerate(orc):
        mi = ctx.mor_model_info(k)
        assert mi["orbital"] == porb[k]
        assert np.array_equal(mi["sampled"], np.array(r.sampled)), k
        assert mi["m"] == r.model.m
        total += r.model.m
    info = ctx.mor_info()
    assert info["m"] == total and info["np"] == len(porb) == info["nq"]
    grid = np.linspace(wmin, wmax, 201)
    ev = ctx.mor_eval(grid, want_res=True)
    Go = mor.siso_green(orc, grid, eta)
    assert rel_err(ev["G"], Go) <= 1e-8
    assert np.all(ev["G"][:, 0, 1] == 0)
    A_full = sv.spectral(sv.green(C, sv.dense_solve(M, B, grid, eta)))
    assert np.abs(ev["A"] - A_full).max() <= 10 * tol * np.abs(A_full).max()
    # residual estimates: the max over the models, small everywhere on the refinement grid's span
    assert np.all(np.isfinite(ev["maxres"])) and ev["maxres"].max() <= 1e-3
    # and at every model's own sampled frequencies Ghat_pp is the full G_pp (Galerkin property)
    for k, r in enumerate(orc):
        Gs = sv.green(C[k:k + 1], sv.dense_solve(M, B[k:k + 1], r.sampled, eta))[:, 0, 0]
        assert rel_err(ctx.mor_eval(r.sampled)["G"][:, k, k], Gs) <= 1e-8


def test_siso_set_state_and_errors(torch):
    from paper_1902_06016_gb300 import Context, GfccError
    inp = inputs(4, 8, 1001)
    ctx = Context(inp, tol=1e-11)
    with pytest.raises(GfccError) as e:
        ctx.mor_build_siso([-1.0, -0.5], 0.01, [0, 1, 0])       # repeated orbital
    assert e.value.code == -1
    ctx.mor_build_siso([-1.0, -0.5, 0.0], 0.01, [0, 1])
    with pytest.raises(GfccError) as e:
        ctx.mor_save("/nonexistent/unused")
    assert e.value.code == -7
    with pytest.raises(GfccError) as e:
        ctx.mor_model_info(2)
    assert e.value.code == -1
    # a MIMO build replaces the set
    ctx.mor_build([-1.0, -0.5, 0.0], 0.01, [0, 1])
    assert ctx.mor_model_info(0)["orbital"] == -1
    with pytest.raises(GfccError):
        ctx.mor_model_info(1)
    ctx2 = Context(inp, tol=1e-11, deriv_indicator=True)
    ctx2.mor_build_siso([-1.0, 0.0], 0.01, [0])
    with pytest.raises(GfccError) as e:
        ctx2.mor_refine(-1.0, 0.0, 11, 1e-6, 100)
    assert e.value.code == -1
