"""Tensor-core (tcgen05) paths vs the FP64 oracle (needs a GB300).

* the raw GEMM against the same rounded operands multiplied in FP64: FP32 accumulation error only
  (ragged tiles, K tails, several tiles in every direction);
* the low-precision sigma: error of the order of the operand rounding (bf16 2^-9, tf32 2^-12 relative)
  and clearly above FP64 rounding;
* GMRES with iterative refinement: low-precision inner sigma, FP64 residuals, same solution as dense LU.
"""
import numpy as np
import pytest

from oracle import bc, hbar
from oracle import sigma as sg
from oracle import solve as sv

from gpu_util import inputs, need_gpu, random_vectors, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def round_bf16(x):
    """Round float64 directly to the nearest bf16 (8 significant bits, ties to even)."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def round_tf32(x):
    f = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    # round to nearest, ties away from zero, on the 13 dropped mantissa bits
    f = ((f + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return f.view(np.float32).astype(np.float64)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (1, 1, 1), (130, 260, 70), (300, 513, 1000), (77, 1000, 33)])
def test_tc_gemm_matches_rounded_fp64(torch, prec, M, N, K):
    from paper_1902_06016_gb300.gfcc import tc_gemm
    rng = np.random.default_rng(M * 7 + N + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    C = tc_gemm(A, B, prec)
    rnd = round_bf16 if prec == "bf16" else round_tf32
    ref = rnd(A) @ rnd(B).T
    # FP32 accumulation inside the tensor core: bound by 2^-17 of the sum of |products| per entry
    bound = 2.0 ** -17 * (np.abs(rnd(A)) @ np.abs(rnd(B)).T) + 1e-6
    assert np.all(np.abs(C - ref) <= bound)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("M,N,K", [(1000, 9000, 200), (2000, 3000, 1100)])
def test_tc_gemm_more_tiles_than_sms(torch, prec, M, N, K):
    """Several output tiles per persistent CTA (288 and 192 tiles on 152 SMs): the double-buffered
    TMEM accumulators are handed between the MMA issuer and the epilogue warps many times."""
    from paper_1902_06016_gb300.gfcc import tc_gemm
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    C = tc_gemm(A, B, prec)
    rnd = round_bf16 if prec == "bf16" else round_tf32
    ref = rnd(A) @ rnd(B).T
    bound = 2.0 ** -17 * (np.abs(rnd(A)) @ np.abs(rnd(B)).T) + 1e-6
    assert np.all(np.abs(C - ref) <= bound)


# windows: above FP64 rounding, below one unit of the operand rounding (bf16 2^-9, tf32 2^-12 relative);
# measured on a GB300: bf16 5.4e-4, 2.9e-4, 1.5e-4 and tf32 7.0e-5, 3.5e-5, 2.1e-5 for the three shapes
@pytest.mark.parametrize("prec,lo,hi", [("bf16", 1e-6, 2.0 ** -9), ("tf32", 1e-7, 2.0 ** -12)])
@pytest.mark.parametrize("o,v,seed", [(4, 8, 1001), (7, 13, 103), (14, 42, 1002)])
def test_lowprec_sigma_error_is_rounding_sized(torch, prec, lo, hi, o, v, seed):
    from paper_1902_06016_gb300 import Context
    inp = inputs(o, v, seed)
    hb = hbar.build(inp)
    ctx = Context(inp, precision=prec)
    X = random_vectors(inp.dim, 6, seed)
    Yo = sg.sigma(hb, X)
    Y = ctx.sigma(X, precision=prec)
    err = rel_err(Y, Yo)
    assert lo < err < hi, err
    # FP64 sigma on the same context is unaffected
    assert rel_err(ctx.sigma(X), Yo) <= 1e-12


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_mixed_precision_solve_reaches_fp64_accuracy(torch, prec):
    from paper_1902_06016_gb300 import Context
    inp = inputs(7, 13, 103)
    hb = hbar.build(inp)
    M = sg.dense_matrix(hb)
    porb = list(range(inp.n))
    ws = np.linspace(-1.0, 0.0, 7)
    ctx = Context(inp, tol=1e-11, precision=prec, restart=20)
    r = ctx.solve_full(ws, 0.01, porb, want_X=True)
    assert r["converged"] and r["stats"].max_rel_res <= 1e-11
    Xo = sv.dense_solve(M, bc.b_vectors(inp, porb), ws, 0.01)
    Go = sv.green(bc.c_vectors(inp, porb), Xo)
    assert rel_err(r["X"], Xo) <= 1e-8
    assert rel_err(r["A"], sv.spectral(Go)) <= 1e-8


@pytest.mark.parametrize("o,v,seed", [(4, 8, 1001), (7, 13, 103), (14, 42, 1002)])
def test_exact_slice_sigma_is_fp64_accurate(torch, o, v, seed):
    """GFCC_PREC_FP64_TC: integer bf16 slices on the tensor cores, exact FP32 partials, FP64
    recombination; must match the oracle like the FP64 CUDA-core sigma does."""
    from paper_1902_06016_gb300 import Context
    inp = inputs(o, v, seed)
    hb = hbar.build(inp)
    ctx = Context(inp)
    X = random_vectors(inp.dim, 70, seed)          # more than one 64-column chunk
    Yo = sg.sigma(hb, X)
    Y = ctx.sigma(X, precision="fp64_tc")
    assert rel_err(Y, Yo) <= 1e-12
    # and per column, relative to that column
    for k in (0, 33, 69):
        assert np.abs(Y[k] - Yo[k]).max() <= 1e-12 * np.abs(Yo[k]).max()


def test_exact_slice_sigma_many_tiles(torch):
    """200 vectors at o=14, v=42: the exact-slice ring GEMM has 110 output tiles x 2 K splits, so the
    persistent exact kernel runs several work units per CTA, each over several exact accumulations."""
    from paper_1902_06016_gb300 import Context
    inp = inputs(14, 42, 1002)
    hb = hbar.build(inp)
    ctx = Context(inp)
    X = random_vectors(inp.dim, 200, 7)
    Yo = sg.sigma(hb, X)
    Y = ctx.sigma(X, precision="fp64_tc")
    assert rel_err(Y, Yo) <= 1e-12
    for k in (0, 101, 199):
        assert np.abs(Y[k] - Yo[k]).max() <= 1e-12 * np.abs(Yo[k]).max()


def test_solve_with_exact_slice_inner_sigma(torch):
    """GFCC_PREC_FP64_TC as the inner precision: FP64 Krylov basis, FP64-accurate sigma throughout."""
    from paper_1902_06016_gb300 import Context
    inp = inputs(7, 13, 103)
    M = sg.dense_matrix(hbar.build(inp))
    porb = list(range(inp.n))
    ws = np.linspace(-1.0, 0.0, 4)
    ctx = Context(inp, tol=1e-11, precision="fp64_tc", restart=20)
    r = ctx.solve_full(ws, 0.01, porb, want_X=True)
    assert r["converged"] and r["stats"].max_rel_res <= 1e-11
    Xo = sv.dense_solve(M, bc.b_vectors(inp, porb), ws, 0.01)
    Go = sv.green(bc.c_vectors(inp, porb), Xo)
    assert rel_err(r["X"], Xo) <= 1e-8
    assert rel_err(r["A"], sv.spectral(Go)) <= 1e-8


def test_mixed_solve_with_exact_slice_residuals(torch):
    from paper_1902_06016_gb300 import Context
    inp = inputs(7, 13, 103)
    M = sg.dense_matrix(hbar.build(inp))
    porb = list(range(inp.n))
    ws = np.linspace(-1.0, 0.0, 5)
    ctx = Context(inp, tol=1e-11, precision="tf32", residual_precision="fp64_tc")
    r = ctx.solve_full(ws, 0.01, porb, want_X=True)
    assert r["converged"] and r["stats"].max_rel_res <= 1e-11
    Xo = sv.dense_solve(M, bc.b_vectors(inp, porb), ws, 0.01)
    assert rel_err(r["X"], Xo) <= 1e-8


def test_hbar_build_through_exact_slices_matches_oracle(torch, monkeypatch):
    """The large H-bar contractions run as 8-slice exact GEMMs on the tensor cores; forced on at a
    small size, the resulting operator must still match the oracle to FP64 level."""
    from paper_1902_06016_gb300 import Context
    monkeypatch.setenv("GFCC_OZ_MIN_MACS", "0")
    inp = inputs(7, 13, 103)
    hb = hbar.build(inp)
    ctx = Context(inp)
    X = random_vectors(inp.dim, 4, 5)
    assert rel_err(ctx.sigma(X), sg.sigma(hb, X)) <= 1e-12
    assert rel_err(ctx.sigma(X, transpose=True), X @ sg.dense_matrix(hb)) <= 1e-12


def test_mor_with_exact_slice_projections_matches_oracle(torch, monkeypatch):
    """The reduced-model projections (complex GEMMs over the full dimension) run as exact-slice
    tensor-core GEMMs at large sizes; forced on here, the model must match the oracle's."""
    from paper_1902_06016_gb300 import Context
    from oracle import mor
    monkeypatch.setenv("GFCC_OZ_MIN_MACS", "0")
    inp = inputs(7, 13, 103)
    hb = hbar.build(inp)
    M = sg.dense_matrix(hb)
    porb = list(range(7))
    B, C = bc.b_vectors(inp, porb), bc.c_vectors(inp, porb)
    ctx = Context(inp, tol=1e-11, precision="tf32")
    ctx.mor_build(np.linspace(-1.0, -0.2, 3), 0.01, porb)
    res = ctx.mor_refine(-1.0, -0.2, 301, 1e-6, 10 ** 6)
    assert res["converged"]
    orc = mor.build_and_refine(hb, B, C, np.linspace(-1.0, -0.2, 3), -1.0, -0.2, 301, 0.01, 1e-6, 10 ** 6,
                               solver="dense", M=M)
    info = ctx.mor_info()
    assert np.array_equal(info["sampled"], np.array(orc.sampled)) and info["m"] == orc.model.m
    grid = np.linspace(-1.0, -0.2, 101)
    assert rel_err(ctx.mor_eval(grid)["G"], mor.reduced_green(orc.model, grid, 0.01)) <= 1e-8
