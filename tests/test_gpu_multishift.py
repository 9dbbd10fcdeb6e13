"""Reduced models on a block Krylov space of M (multi-shift reuse: one space for every frequency) on the
GPU against the oracle and the full solutions (needs a GB300)."""
import numpy as np
import pytest

import synth
from oracle import bc, hbar, mor
from oracle import sigma as sg
from oracle import solve as sv

from gpu_util import inputs, need_gpu, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


@pytest.mark.parametrize("o,v,seed,prec", [(4, 8, 1001, "fp64"), (7, 13, 103, "tf32")])
def test_krylov_model_matches_oracle(torch, o, v, seed, prec):
    from paper_1902_06016_gb300 import Context
    inp = inputs(o, v, seed)
    hb = hbar.build(inp)
    M = sg.dense_matrix(hb)
    porb = list(range(o))
    B, C = bc.b_vectors(inp, porb), bc.c_vectors(inp, porb)
    eta, tol = 0.01, 1e-6
    ctx = Context(inp, tol=1e-11, precision=prec)
    ctx.mor_build_krylov(3, eta, porb)
    rm, st = mor.build_krylov(hb, B, C, 3)
    assert ctx.mor_info()["m"] == rm.m and len(ctx.mor_info()["sampled"]) == 0
    grid = np.linspace(-1.0, -0.2, 101)
    assert rel_err(ctx.mor_eval(grid)["G"], mor.reduced_green(rm, grid, eta)) <= 1e-8
    res = ctx.mor_refine(-1.0, -0.2, 201, tol, 10 ** 6)
    assert res["converged"] and res["max_err"] <= tol
    rm2, st2, hist, ok = mor.refine_krylov(hb, B, C, 3, -1.0, -0.2, 201, eta, tol, 10 ** 6)
    assert ok and res["m"] == rm2.m
    assert rel_err(ctx.mor_eval(grid)["G"], mor.reduced_green(rm2, grid, eta)) <= 1e-8
    A_full = sv.spectral(sv.green(C, sv.dense_solve(M, B, grid, eta)))
    assert np.abs(ctx.mor_eval(grid)["A"] - A_full).max() <= 10 * tol * np.abs(A_full).max()


def test_krylov_model_co_size_matches_full_solution(torch):
    """CO size (D = 3,836), the 14 occupied orbitals: the Krylov model refined to a residual estimate of
    1e-6 over [-1.2, -0.3] Ha reproduces the dense solutions' A(w) and G on a grid."""
    from paper_1902_06016_gb300 import Context
    W = synth.WORKLOADS["co_o14_v42"]
    inp = synth.make_inputs(W["o"], W["v"], W["seed"])
    M = sg.dense_matrix(hbar.build(inp))
    porb = list(range(W["o"]))
    B, C = bc.b_vectors(inp, porb), bc.c_vectors(inp, porb)
    ctx = Context(inp, tol=1e-10, precision="tf32")
    ctx.mor_build_krylov(4, W["eta"], porb)
    res = ctx.mor_refine(W["wmin"], W["wmax"], 201, 1e-6, inp.dim)
    assert res["converged"]
    grid = np.linspace(W["wmin"], W["wmax"], 41)
    Gf = sv.green(C, sv.dense_solve(M, B, grid, W["eta"]))
    ev = ctx.mor_eval(grid)
    assert rel_err(ev["G"], Gf) <= 1e-5
    assert np.abs(ev["A"] - sv.spectral(Gf)).max() <= 1e-5 * np.abs(sv.spectral(Gf)).max()
    with pytest.raises(Exception):
        ctx.mor_save("/nonexistent/unused")
