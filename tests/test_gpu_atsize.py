"""GPU path vs the FP64 oracle on the code paths the benchmark takes (needs a GB300).

* The exact-slice products keep the int32 split sums of all their diagonals side by side when those
  fit in a 4 GB bound, and otherwise accumulate diagonal by diagonal in FP64 over column chunks. At
  benzene size the second branch runs; GFCC_OZ_SLAB_BYTES lowers the bound so that it also runs at
  small sizes, where the oracle is cheap.
* CO size (o = 14, v = 42, D = 3,836): full solves of all 56 orbitals against dense LU of the
  oracle's matrix, and the adaptive reduced model from 8 seeds against the oracle's.
* Benzene size (o = 42, v = 186, D = 160,188): sigma on random vectors element by element, and G at
  the middle of the window from the full solve and from the reduced model, against oracle GMRES.

Tolerances as in the other parity tests: FP64-accurate sigma 1e-12 (relative, per column), solutions
1e-8, TF32 sigma within one unit of its operand rounding (2^-12 relative) and well above FP64 rounding.
"""
import numpy as np
import pytest

import synth
from oracle import bc, hbar, mor
from oracle import sigma as sg
from oracle import solve as sv

from gpu_util import inputs, need_gpu, random_vectors, rel_err

pytestmark = pytest.mark.gpu

TINY_SLAB = "4096"   # bytes: every exact product takes the per-diagonal branch, real outputs in chunks


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def ctx_for(inp, **kw):
    from paper_1902_06016_gb300 import Context
    return Context(inp, **kw)


# ---- per-diagonal FP64 accumulation of the exact-slice products --------------------------------
@pytest.mark.parametrize("o,v,seed", [(7, 13, 103), (14, 42, 1002)])
def test_per_diagonal_exact_products_build_and_sigma(torch, monkeypatch, o, v, seed):
    """H-bar build (real outputs, column chunks of 256) and FP64-accurate sigma (complex outputs) on the
    per-diagonal branch: the operator and the products must still match the oracle to FP64 level."""
    monkeypatch.setenv("GFCC_OZ_MIN_MACS", "0")
    monkeypatch.setenv("GFCC_OZ_SLAB_BYTES", TINY_SLAB)
    inp = inputs(o, v, seed)
    hb = hbar.build(inp)
    ctx = ctx_for(inp)
    X = random_vectors(inp.dim, 70, seed + 3)
    Yo = sg.sigma(hb, X)
    assert rel_err(ctx.sigma(X), Yo) <= 1e-12
    Y = ctx.sigma(X, precision="fp64_tc")
    for k in range(0, 70, 7):
        assert np.abs(Y[k] - Yo[k]).max() <= 1e-12 * np.abs(Yo[k]).max()


def test_per_diagonal_exact_products_solve_and_mor(torch, monkeypatch):
    """GMRES-IR with FP64-accurate residuals and the reduced model's exact-slice projections, all on the
    per-diagonal branch: same solutions as dense LU, same sampled frequencies and Ghat as the oracle."""
    monkeypatch.setenv("GFCC_OZ_MIN_MACS", "0")
    monkeypatch.setenv("GFCC_OZ_SLAB_BYTES", TINY_SLAB)
    inp = inputs(7, 13, 103)
    hb = hbar.build(inp)
    M = sg.dense_matrix(hb)
    porb = list(range(7))
    B, C = bc.b_vectors(inp, porb), bc.c_vectors(inp, porb)
    ws = np.linspace(-1.0, -0.2, 5)
    ctx = ctx_for(inp, tol=1e-11, precision="tf32", residual_precision="fp64_tc")
    r = ctx.solve_full(ws, 0.01, porb, want_X=True)
    assert r["converged"]
    Xo = sv.dense_solve(M, B, ws, 0.01)
    assert rel_err(r["X"], Xo) <= 1e-8
    assert rel_err(r["G"], sv.green(C, Xo)) <= 1e-8
    ctx.mor_build(np.linspace(-1.0, -0.2, 3), 0.01, porb)
    res = ctx.mor_refine(-1.0, -0.2, 301, 1e-6, 10 ** 6)
    assert res["converged"]
    orc = mor.build_and_refine(hb, B, C, np.linspace(-1.0, -0.2, 3), -1.0, -0.2, 301, 0.01, 1e-6, 10 ** 6,
                               solver="dense", M=M)
    info = ctx.mor_info()
    assert np.array_equal(info["sampled"], np.array(orc.sampled)) and info["m"] == orc.model.m
    grid = np.linspace(-1.0, -0.2, 101)
    assert rel_err(ctx.mor_eval(grid)["G"], mor.reduced_green(orc.model, grid, 0.01)) <= 1e-8


# ---- CO size: o = 14, v = 42, D = 3,836 ----------------------------------------------------------
@pytest.fixture(scope="module")
def co():
    W = synth.WORKLOADS["co_o14_v42"]
    inp = synth.make_inputs(W["o"], W["v"], W["seed"])
    hb = hbar.build(inp)
    M = sg.dense_matrix(hb)
    porb = list(range(inp.n))                        # all 56 spin-orbitals
    return W, inp, hb, M, porb, bc.b_vectors(inp, porb), bc.c_vectors(inp, porb)


@pytest.mark.parametrize("precision", ["tf32", "fp64_tc"])
def test_co_size_full_solve_all_orbitals_matches_dense(torch, co, precision):
    """Full-dimension batched GMRES-IR for all 56 orbitals at every 50th frequency of the 500-point grid
    on [-1.2, -0.3] Ha (eta = 0.01), against dense LU of the oracle's matrix."""
    W, inp, hb, M, porb, B, C = co
    grid = np.linspace(W["wmin"], W["wmax"], W["nw"])
    ws = grid[::50]
    ctx = ctx_for(inp, tol=1e-10, precision=precision)
    r = ctx.solve_full(ws, W["eta"], porb)
    assert r["converged"] and r["stats"].max_rel_res <= 1e-10
    Go = sv.green(C, sv.dense_solve(M, B, ws, W["eta"]))
    assert rel_err(r["G"], Go) <= 1e-8
    assert rel_err(r["A"], sv.spectral(Go)) <= 1e-8


def test_co_size_mor_matches_oracle(torch, co):
    """Reduced model from 8 seed frequencies, refined to a residual estimate of 1e-6 on a 201-point
    grid: the GPU (TF32 inner sigma, FP64-accurate residuals) picks the oracle's frequencies, reaches
    its model order, and its Ghat matches the oracle's reduced model; A matches the full solution."""
    W, inp, hb, M, porb, B, C = co
    wmin, wmax, eta, tol = W["wmin"], W["wmax"], W["eta"], 1e-6
    seeds = np.linspace(wmin, wmax, 8)
    ctx = ctx_for(inp, tol=1e-10, precision="tf32")
    ctx.mor_build(seeds, eta, porb)
    res = ctx.mor_refine(wmin, wmax, 201, tol, 10 ** 6)
    assert res["converged"] and res["max_err"] <= tol
    orc = mor.build_and_refine(hb, B, C, seeds, wmin, wmax, 201, eta, tol, 10 ** 6, solver="dense", M=M)
    info = ctx.mor_info()
    assert np.array_equal(info["sampled"], np.array(orc.sampled))
    assert info["m"] == orc.model.m
    grid = np.linspace(wmin, wmax, W["nw"])[::10]
    ev = ctx.mor_eval(grid)
    assert rel_err(ev["G"], mor.reduced_green(orc.model, grid, eta)) <= 1e-8
    A_full = sv.spectral(sv.green(C, sv.dense_solve(M, B, grid[::5], eta)))
    assert np.abs(ev["A"][::5] - A_full).max() <= 10 * tol * np.abs(A_full).max()


# ---- benzene size: o = 42, v = 186, D = 160,188 --------------------------------------------------
@pytest.fixture(scope="module")
def benzene():
    W = synth.WORKLOADS["benzene_o42_v186"]
    inp = synth.make_inputs(W["o"], W["v"], W["seed"])
    return W, inp, hbar.build(inp)


def test_benzene_size_sigma_matches_oracle(torch, benzene):
    """The sigma on 8 random complex vectors at the benchmark's size: FP64 (CUDA cores) and
    FP64-accurate (exact slices) to 1e-12 per column; TF32 within its operand rounding."""
    W, inp, hb = benzene
    X = random_vectors(inp.dim, 8, 42)
    Yo = sg.sigma(hb, X)
    ctx = ctx_for(inp, precision="tf32")
    for prec in ("fp64", "fp64_tc"):
        Y = ctx.sigma(X, precision=prec)
        for k in range(8):
            assert np.abs(Y[k] - Yo[k]).max() <= 1e-12 * np.abs(Yo[k]).max(), (prec, k)
    err = rel_err(ctx.sigma(X, precision="tf32"), Yo)
    assert 1e-7 < err < 2.0 ** -12, err


def test_benzene_size_green_matches_oracle(torch, benzene):
    """G_pq at w = -0.6 Ha (middle of the window) for p = 0, 1 and all 42 q: the full-dimension FP64-accurate
    solve to 1e-8, and the benchmark's reduced model (8 seeds, refined to 1e-6 on 500 points, TF32 inner
    sigma) to 1e-6, against the oracle's GMRES solutions (tolerance 1e-10)."""
    W, inp, hb = benzene
    porb = list(range(W["o"]))
    wmid = 0.5 * (W["wmin"] + W["wmax"])
    Xo, reso = sv.gmres_solve(hb, bc.b_vectors(inp, [0, 1]), [wmid], W["eta"], tol=1e-10)
    assert reso.max() <= 1e-10
    Go = sv.green(bc.c_vectors(inp, porb), Xo)[0]            # [2, 42]
    ctx = ctx_for(inp, tol=1e-8, precision="tf32")
    ctx.mor_build(synth.omega_grid(W["wmin"], W["wmax"], 8), W["eta"], porb)
    ref = ctx.mor_refine(W["wmin"], W["wmax"], 500, 1e-6, 1700)
    assert ref["converged"]
    Gm = ctx.mor_eval([wmid])["G"][0][:2]
    assert rel_err(Gm, Go) <= 1e-6
    ctx.set_opts(tol=1e-10, precision="fp64_tc")
    r = ctx.solve_full([wmid], W["eta"], [0, 1], qorb=porb)
    assert r["converged"]
    assert rel_err(r["G"][0], Go) <= 1e-8
