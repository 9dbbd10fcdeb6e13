"""GPU path vs the FP64 oracle, element by element, through the C ABI (needs a GB300).

Sizes span several GEMM tiles with ragged tails (o = 3..14, v = 5..42); tolerances follow from FP64
arithmetic: sigma 1e-12 relative (normwise per block), solutions 1e-8 (GMRES stops at 1e-10..1e-11
relative residual, condition number <= ~1e3), A(w) 1e-8 normwise.
"""
import numpy as np
import pytest

import synth
from oracle import bc, hbar, mor
from oracle import sigma as sg
from oracle import solve as sv

from gpu_util import inputs, need_gpu, random_vectors, rel_err

pytestmark = pytest.mark.gpu

SHAPES = [(3, 5, 101), (4, 8, 1001), (7, 13, 103), (14, 42, 1002)]


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def ctx_for(inp, **kw):
    from paper_1902_06016_gb300 import Context
    return Context(inp, **kw)


@pytest.mark.parametrize("o,v,seed", SHAPES)
def test_sigma_matches_oracle(torch, o, v, seed):
    inp = inputs(o, v, seed)
    hb = hbar.build(inp)
    ctx = ctx_for(inp)
    X = random_vectors(inp.dim, 5, seed)
    Y = ctx.sigma(X)
    Yo = sg.sigma(hb, X)
    assert rel_err(Y, Yo) <= 1e-12
    # single vector and device buffers give the same
    Y1 = ctx.sigma(X[2])
    assert rel_err(Y1, Yo[2]) <= 1e-12
    Xd = torch.from_numpy(X).cuda()
    Yd = ctx.sigma(Xd)
    assert rel_err(Yd.cpu().numpy(), Yo) <= 1e-12


@pytest.mark.parametrize("o,v,seed", SHAPES[:3])
def test_sigma_transpose_matches_oracle(torch, o, v, seed):
    inp = inputs(o, v, seed)
    M = sg.dense_matrix(hbar.build(inp))
    ctx = ctx_for(inp)
    X = random_vectors(inp.dim, 3, seed + 1)
    assert rel_err(ctx.sigma(X, transpose=True), X @ M) <= 1e-12


@pytest.mark.parametrize("o,v,seed", SHAPES)
def test_b_and_c_vectors(torch, o, v, seed):
    inp = inputs(o, v, seed)
    ctx = ctx_for(inp)
    orb = list(range(inp.n))
    assert rel_err(ctx.vectors(orb), bc.b_vectors(inp)) <= 1e-14
    assert rel_err(ctx.vectors(orb, left=True), bc.c_vectors(inp)) <= 1e-13


@pytest.mark.parametrize("o,v,seed", SHAPES[:3])
def test_solve_full_matches_dense(torch, o, v, seed):
    inp = inputs(o, v, seed)
    hb = hbar.build(inp)
    M = sg.dense_matrix(hb)
    porb = list(range(inp.n))
    ws = np.linspace(-1.0, 0.0, 9)
    eta = 0.01
    ctx = ctx_for(inp, tol=1e-11, restart=20)
    r = ctx.solve_full(ws, eta, porb, want_X=True)
    assert r["converged"] and r["stats"].max_rel_res <= 1e-11
    Xo = sv.dense_solve(M, bc.b_vectors(inp, porb), ws, eta)
    Go = sv.green(bc.c_vectors(inp, porb), Xo)
    assert rel_err(r["X"], Xo) <= 1e-8
    assert rel_err(r["G"], Go) <= 1e-8
    assert rel_err(r["A"], sv.spectral(Go)) <= 1e-8


def test_solve_full_q_subset_and_ragged_batches(torch):
    inp = inputs(7, 13, 103)
    hb = hbar.build(inp)
    M = sg.dense_matrix(hb)
    porb = [0, 3, 6, 9]
    qorb = [6, 0, 12]
    ws = np.linspace(-1.2, -0.3, 7)
    ctx = ctx_for(inp, tol=1e-11, max_batch=5)   # 28 columns in ragged batches of 5
    r = ctx.solve_full(ws, 0.02, porb, qorb=qorb)
    Xo = sv.dense_solve(M, bc.b_vectors(inp, porb), ws, 0.02)
    Go = sv.green(bc.c_vectors(inp, qorb), Xo)
    assert rel_err(r["G"], Go) <= 1e-8
    Ao = sv.spectral(Go, diag_index=[1, None, 0, None]) if False else None
    # A sums p that also appear in the q set: p=0 (q pos 1) and p=6 (q pos 0)
    Aexp = -(Go[:, 0, 1].imag + Go[:, 2, 0].imag) / np.pi
    assert rel_err(r["A"], Aexp) <= 1e-8


@pytest.mark.parametrize("o,v,seed", [(4, 8, 1001), (7, 13, 103)])
def test_mor_matches_oracle_and_full(torch, o, v, seed):
    inp = inputs(o, v, seed)
    hb = hbar.build(inp)
    M = sg.dense_matrix(hb)
    porb = list(range(o))
    B, C = bc.b_vectors(inp, porb), bc.c_vectors(inp, porb)
    wmin, wmax, eta, tol = -1.0, -0.2, 0.01, 1e-6
    ctx = ctx_for(inp, tol=1e-11)
    ctx.mor_build(np.linspace(wmin, wmax, 3), eta, porb)
    res = ctx.mor_refine(wmin, wmax, 301, tol, 10 ** 6)
    assert res["converged"] and res["max_err"] <= tol
    info = ctx.mor_info()
    orc = mor.build_and_refine(hb, B, C, np.linspace(wmin, wmax, 3), wmin, wmax, 301, eta, tol, 10 ** 6,
                               solver="dense", M=M)
    # same refinement decisions (frequencies are exact midpoints)
    assert np.array_equal(info["sampled"], np.array(orc.sampled))
    assert info["m"] == orc.model.m
    grid = np.linspace(wmin, wmax, 301)
    ev = ctx.mor_eval(grid, want_res=True)
    Gh_o = mor.reduced_green(orc.model, grid, eta)
    assert rel_err(ev["G"], Gh_o) <= 1e-8
    A_full = sv.spectral(sv.green(C, sv.dense_solve(M, B, grid, eta)))
    assert np.abs(ev["A"] - A_full).max() <= 10 * tol * np.abs(A_full).max()
    # residual estimate tracks the oracle's explicit residual
    res_o = mor.residuals(orc.model, B, grid, eta).max(axis=1)
    assert np.abs(ev["maxres"] - res_o).max() <= 1e-7
    # interpolation at the sampled frequencies
    Gs = sv.green(C, sv.dense_solve(M, B, info["sampled"], eta))
    assert rel_err(ctx.mor_eval(info["sampled"])["G"], Gs) <= 1e-8


@pytest.mark.parametrize("o,v,seed", [(4, 8, 1001), (7, 13, 103)])
def test_mor_derivative_indicator_matches_oracle(torch, o, v, seed):
    """Refinement driven by the dG/dw mismatch at the sampled frequencies: with a two-point residual
    grid (no interior points, so the residual estimate alone stops at the seeds) the derivative
    indicator adds midpoints; the GPU must choose the same frequencies as the oracle."""
    inp = inputs(o, v, seed)
    hb = hbar.build(inp)
    M = sg.dense_matrix(hb)
    porb = list(range(3))
    B, C = bc.b_vectors(inp, porb), bc.c_vectors(inp, porb)
    seeds, eta, tol = [-1.0, -0.6, -0.2], 0.02, 1e-6
    orc = mor.build_and_refine(hb, B, C, seeds, -1.0, -0.2, 2, eta, tol, 10 ** 6, solver="dense", M=M, deriv=True)
    assert len(orc.sampled) > len(seeds)
    ctx = ctx_for(inp, tol=1e-11, deriv_indicator=True)
    ctx.mor_build(seeds, eta, porb)
    res = ctx.mor_refine(-1.0, -0.2, 2, tol, 10 ** 6)
    assert res["converged"]
    info = ctx.mor_info()
    assert np.array_equal(info["sampled"], np.array(orc.sampled))
    # the reduced model's dG/dw at the samples now matches the exact one within the tolerance
    dG = mor.reduced_green_derivative(orc.model, orc.sampled, eta)
    grid = np.linspace(-1.0, -0.2, 41)
    assert rel_err(ctx.mor_eval(grid)["G"], mor.reduced_green(orc.model, grid, eta)) <= 1e-8
    assert np.isfinite(dG).all()
    # without the indicator the same call stops at the seeds
    ctx2 = ctx_for(inp, tol=1e-11)
    ctx2.mor_build(seeds, eta, porb)
    ctx2.mor_refine(-1.0, -0.2, 2, tol, 10 ** 6)
    assert np.array_equal(ctx2.mor_info()["sampled"], np.array(seeds))


def test_mor_save_load_roundtrip(torch, tmp_path):
    inp = inputs(4, 8, 1001)
    porb = list(range(4))
    ctx = ctx_for(inp)
    ctx.mor_build([-1.0, -0.5, 0.0], 0.01, porb)
    grid = np.linspace(-1, 0, 50)
    A1 = ctx.mor_eval(grid)["A"]
    path = str(tmp_path / "model.bin")
    ctx.mor_save(path)
    ctx2 = ctx_for(inp)
    ctx2.mor_load(path)
    assert ctx2.mor_info()["m"] == ctx.mor_info()["m"]
    assert np.array_equal(ctx2.mor_eval(grid)["A"], A1)


def test_errors_are_status_codes(torch):
    from paper_1902_06016_gb300 import GfccError
    inp = inputs(4, 8, 1001)
    ctx = ctx_for(inp)
    with pytest.raises(GfccError) as e:
        ctx.mor_eval([0.0])
    assert e.value.code == -7
    with pytest.raises(GfccError) as e:
        ctx.solve_full([np.nan], 0.01, [0])
    assert e.value.code == -4
    with pytest.raises(GfccError) as e:
        ctx.solve_full([0.0], 0.01, [99])
    assert e.value.code == -1
    bad = synth.make_inputs(4, 8, 1001)
    bad.t2 = bad.t2.copy()
    bad.t2[0, 1, 2, 3] = np.inf
    with pytest.raises(GfccError) as e:
        ctx_for(bad)
    assert e.value.code == -4
    # iteration cap reached -> status, outputs still written
    ctx3 = ctx_for(inp, tol=1e-14, restart=2, max_restarts=2)
    r = ctx3.solve_full([-0.5], 0.01, [0, 1])
    assert not r["converged"] and r["stats"].not_converged > 0 and np.all(np.isfinite(r["A"]))


def test_mor_extrapolated_guess_same_model_less_work(torch):
    """Refinement solves started from the reduced model's prediction: same sampled frequencies and the
    same reduced Green's function as from zero guesses, with fewer Arnoldi steps."""
    inp = inputs(7, 13, 103)
    porb = list(range(7))
    out = {}
    for guess in (False, True):
        # solver tolerance 1e-9: well above the floor of the FP64-accurate residuals, so that the step
        # counts measure convergence and not stagnation at that floor
        ctx = ctx_for(inp, tol=1e-9, precision="tf32", mor_guess=guess)
        ctx.mor_build([-1.0, -0.2], 0.01, porb)
        s0 = ctx.mor_stats()["arnoldi_steps"]
        ctx.mor_refine(-1.0, -0.2, 201, 1e-6, 10 ** 6)
        out[guess] = (ctx.mor_info()["sampled"], ctx.mor_eval(np.linspace(-1.0, -0.2, 51))["G"],
                      ctx.mor_stats()["arnoldi_steps"] - s0)
    assert np.array_equal(out[True][0], out[False][0]) and len(out[True][0]) > 2
    assert rel_err(out[True][1], out[False][1]) <= 1e-7
    assert out[True][2] < out[False][2]
