"""Pins of the FP64 oracle against things other than itself (CPU only).

* brute-force second quantisation (explicit determinants, e^{-T} H e^{T}) for M, b_p, c_q at
  random amplitudes and several shapes: a dropped term, wrong sign, factor or index fails here;
* closed forms: Koopmans poles when T = Lambda = 0 and v = 0; the exact resolvent of Eq. gfxn0 over
  the whole N-1 sector when T = Lambda = 0 and o = 2;
* linear algebra: dense LU and GMRES agree; the reduced model interpolates the full one at its
  sampled frequencies, is exact when S spans the space, and is invariant under a unitary change of
  basis of S; the refinement loop reaches its tolerance;
* the generator: SplitMix64's published first output, Box-Muller moments, 8-fold symmetry.
"""
import numpy as np
import pytest

import synth
from oracle import bc, fockspace, hbar, mor
from oracle import sigma as sg
from oracle import solve as sv


def _random_case(o, v, seed):
    return synth.random_amplitudes(synth.make_inputs(o, v, seed, scale_mode="literal"), seed + 1)


@pytest.mark.parametrize("o,v,seed", [(2, 3, 5), (3, 3, 11), (3, 5, 12), (4, 4, 13), (5, 3, 14),
                                      (2, 6, 15), (4, 6, 16)])
def test_sigma_b_c_match_brute_force(o, v, seed):
    inp = _random_case(o, v, seed)
    bf = fockspace.build_from_inputs(inp)
    hb = hbar.build(inp)
    M = sg.dense_matrix(hb)
    scale = np.abs(bf.M).max()
    assert np.abs(M - bf.M).max() <= 1e-12 * scale
    assert np.abs(bc.b_vectors(inp) - bf.b).max() <= 1e-12
    assert np.abs(bc.c_vectors(inp) - bf.c).max() <= 1e-12


@pytest.mark.parametrize("part", ["t1", "t2", "l1", "l2"])
def test_each_amplitude_block_matters(part):
    """Zeroing one amplitude block changes M (or c): the pins above are not vacuous."""
    inp = _random_case(3, 4, 21)
    bf = fockspace.build_from_inputs(inp)
    getattr(inp, part)[:] = 0.0
    hb = hbar.build(inp)
    dM = np.abs(sg.dense_matrix(hb) - bf.M).max()
    dc = np.abs(bc.c_vectors(inp) - bf.c).max()
    db = np.abs(bc.b_vectors(inp) - bf.b).max()
    assert max(dM, dc, db) > 1e-4


def test_tiny_workload_brute_force():
    """The o=4, v=8 workload with its MP2-like amplitudes (495-determinant N sector)."""
    W = synth.WORKLOADS["tiny_o4_v8"]
    inp = synth.make_inputs(W["o"], W["v"], W["seed"])
    bf = fockspace.build_from_inputs(inp)
    hb = hbar.build(inp)
    assert np.abs(sg.dense_matrix(hb) - bf.M).max() <= 1e-12
    assert np.abs(bc.b_vectors(inp) - bf.b).max() <= 1e-13
    assert np.abs(bc.c_vectors(inp) - bf.c).max() <= 1e-13
    # G from the brute-force objects equals the oracle's
    ws = np.linspace(W["wmin"], W["wmax"], 7)
    Xb = sv.dense_solve(bf.M, bf.b, ws, W["eta"])
    Xo = sv.dense_solve(sg.dense_matrix(hb), bc.b_vectors(inp), ws, W["eta"])
    Gb = sv.green(bf.c, Xb)
    Go = sv.green(bc.c_vectors(inp), Xo)
    assert np.abs(Gb - Go).max() <= 1e-10 * np.abs(Gb).max()


def test_koopmans_limit():
    """T = Lambda = 0, v = 0: G_ii(w) = 1/(w - eps_i - i eta), no other poles."""
    inp = synth.make_inputs(5, 0, 3, with_t=False, with_lambda=False)
    hb = hbar.build(inp)
    M = sg.dense_matrix(hb)
    ws = np.linspace(-2, 0, 11)
    eta = 0.01
    G = sv.green(bc.c_vectors(inp), sv.dense_solve(M, bc.b_vectors(inp), ws, eta))
    ref = np.zeros_like(G)
    for i in range(5):
        ref[:, i, i] = 1.0 / (ws - inp.eps[i] - 1j * eta)
    assert np.abs(G - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("v,seed", [(3, 7), (6, 8)])
def test_exact_resolvent_when_space_is_complete(v, seed):
    """T = Lambda = 0 and o = 2: 1h+2h1p is the whole N-1 sector, so Eq. gfxn0 (with Psi = Phi,
    E_0 = E_HF) is reproduced exactly, for every (p, q)."""
    inp = synth.make_inputs(2, v, seed, scale_mode="literal", with_t=False, with_lambda=False)
    bf = fockspace.build_from_inputs(inp)
    hb = hbar.build(inp)
    ws = np.linspace(-1.5, 0.5, 9)
    eta = 0.02
    G = sv.green(bc.c_vectors(inp), sv.dense_solve(sg.dense_matrix(hb), bc.b_vectors(inp), ws, eta))
    Gx = fockspace.exact_resolvent(bf, ws, eta)
    assert np.abs(G - Gx).max() <= 1e-12 * np.abs(Gx).max()


def test_gmres_matches_dense():
    inp = synth.make_inputs(6, 12, 31)
    hb = hbar.build(inp)
    B = bc.b_vectors(inp, range(8))
    ws = [-1.0, -0.55, -0.2]
    Xd = sv.dense_solve(sg.dense_matrix(hb), B, ws, 0.01)
    Xg, res = sv.gmres_solve(hb, B, ws, 0.01, tol=1e-11)
    assert res.max() <= 1e-11
    assert np.abs(Xd - Xg).max() <= 1e-9 * np.abs(Xd).max()


def _mor_case():
    inp = synth.make_inputs(5, 10, 41)
    hb = hbar.build(inp)
    p = list(range(5))
    return inp, hb, bc.b_vectors(inp, p), bc.c_vectors(inp, p), sg.dense_matrix(hb)


def test_mor_interpolates_at_sampled_frequencies():
    inp, hb, B, C, M = _mor_case()
    seeds = [-1.1, -0.8, -0.5]
    X = sv.dense_solve(M, B, seeds, 0.01)
    S, kept = mor.orthonormalise(None, X.reshape(-1, X.shape[-1]).T)
    assert all(kept)
    rm = mor.project(hb, S, B, C)
    Gh = mor.reduced_green(rm, seeds, 0.01)
    G = sv.green(C, X)
    assert np.abs(Gh - G).max() <= 1e-11 * np.abs(G).max()
    # and it is NOT exact away from the samples (the test is not vacuous)
    Gm = sv.green(C, sv.dense_solve(M, B, [-0.65], 0.01))
    assert np.abs(mor.reduced_green(rm, [-0.65], 0.01) - Gm).max() > 1e-6 * np.abs(Gm).max()


def test_mor_exact_when_subspace_is_whole_space():
    inp, hb, B, C, M = _mor_case()
    D = M.shape[0]
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D)))
    rm = mor.project(hb, Q, B, C)
    ws = np.linspace(-1.2, -0.3, 13)
    G = sv.green(C, sv.dense_solve(M, B, ws, 0.01))
    assert np.abs(mor.reduced_green(rm, ws, 0.01) - G).max() <= 1e-10 * np.abs(G).max()


def test_mor_invariant_under_unitary_change_of_basis():
    inp, hb, B, C, M = _mor_case()
    X = sv.dense_solve(M, B, [-1.0, -0.4], 0.01)
    S, _ = mor.orthonormalise(None, X.reshape(-1, X.shape[-1]).T)
    rng = np.random.default_rng(1)
    U, _ = np.linalg.qr(rng.standard_normal((S.shape[1],) * 2) + 1j * rng.standard_normal((S.shape[1],) * 2))
    ws = np.linspace(-1.2, -0.3, 9)
    G1 = mor.reduced_green(mor.project(hb, S, B, C), ws, 0.01)
    G2 = mor.reduced_green(mor.project(hb, S @ U, B, C), ws, 0.01)
    assert np.abs(G1 - G2).max() <= 1e-11 * np.abs(G1).max()


def test_orthonormalise_drops_dependent_columns():
    rng = np.random.default_rng(2)
    Y = rng.standard_normal((40, 5)) + 1j * rng.standard_normal((40, 5))
    Y = np.concatenate([Y, Y[:, :2] @ np.array([[1.0, 2.0], [3.0, -1.0]])], axis=1)
    S, kept = mor.orthonormalise(None, Y)
    assert kept == [True] * 5 + [False, False]
    assert np.abs(S.conj().T @ S - np.eye(5)).max() <= 1e-14


def test_refinement_reaches_tolerance_and_matches_full():
    inp, hb, B, C, M = _mor_case()
    r = mor.build_and_refine(hb, B, C, [-1.2, -0.75, -0.3], -1.2, -0.3, 300, 0.01, 1e-6,
                             10 ** 6, solver="dense", M=M)
    assert r.converged and r.history[-1][1] <= 1e-6
    grid = np.linspace(-1.2, -0.3, 300)
    A = sv.spectral(sv.green(C, sv.dense_solve(M, B, grid, 0.01)))
    Ah = sv.spectral(mor.reduced_green(r.model, grid, 0.01))
    assert np.abs(A - Ah).max() <= 1e-6 * np.abs(A).max()
    # the error estimate decreases from round to round
    assert r.history[0][1] > r.history[-1][1]


def test_refinement_respects_order_bound():
    inp, hb, B, C, M = _mor_case()
    r = mor.build_and_refine(hb, B, C, [-1.2, -0.3], -1.2, -0.3, 300, 0.01, 1e-12, 20,
                             solver="dense", M=M)
    assert r.model.m <= 20 and not r.converged


def test_siso_models_interpolate_their_diagonal_and_refine():
    """Per-orbital models: model p is built from X_p(w_k) alone, so by the Galerkin property its Ghat_pp
    equals the full G_pp at each of its own sampled frequencies; each model refines to the tolerance,
    its order is at most its number of samples, and A from the diagonal models matches the full A."""
    inp, hb, B, C, M = _mor_case()
    res = mor.build_and_refine_siso(hb, B, C, [-1.2, -0.75, -0.3], -1.2, -0.3, 300, 0.01, 1e-6, 10 ** 6,
                                    solver="dense", M=M)
    assert len(res) == B.shape[0]
    for p, r in enumerate(res):
        assert r.converged and r.model.m <= len(r.sampled)
        Gs = sv.green(C[p:p + 1], sv.dense_solve(M, B[p:p + 1], r.sampled, 0.01))[:, 0, 0]
        Gh = mor.reduced_green(r.model, r.sampled, 0.01)[:, 0, 0]
        assert np.abs(Gh - Gs).max() <= 1e-10 * np.abs(Gs).max()
    grid = np.linspace(-1.2, -0.3, 300)
    Gf = sv.green(C, sv.dense_solve(M, B, grid, 0.01))
    Gd = mor.siso_green(res, grid, 0.01)
    assert np.all(Gd[:, 0, 1] == 0.0)
    assert np.abs(sv.spectral(Gd) - sv.spectral(Gf)).max() <= 1e-5 * np.abs(sv.spectral(Gf)).max()
    # the refinement ran (frequencies beyond the three seeds)
    assert all(len(r.sampled) > 3 for r in res)


def test_splitmix64_published_value_and_normals():
    # SplitMix64 from state 0: first output 0xE220A8397B1DCDAF (Steele et al. reference code)
    assert int(synth._mix(np.array([0x9E3779B97F4A7C15], dtype=np.uint64))[0]) == 0xE220A8397B1DCDAF
    z = synth.normal(5, 9, np.arange(200000))
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    g = synth.make_inputs(3, 4, 9).full_antisym()
    assert np.abs(g + g.transpose(1, 0, 2, 3)).max() == 0.0
    assert np.abs(g + g.transpose(0, 1, 3, 2)).max() == 0.0
    assert np.abs(g - g.transpose(2, 3, 0, 1)).max() == 0.0


def test_generator_blocks_are_slices_of_the_full_tensor():
    inp = synth.make_inputs(3, 4, 9, scale_mode="literal")
    g = inp.full_antisym()
    o = 3
    assert np.array_equal(inp.oooo, g[:o, :o, :o, :o])
    assert np.array_equal(inp.ooov, g[:o, :o, :o, o:])
    assert np.array_equal(inp.oovv, g[:o, :o, o:, o:])
    assert np.array_equal(inp.ovov, g[:o, o:, :o, o:])
    assert np.array_equal(inp.ovvv, g[:o, o:, o:, o:])


def test_green_derivatives_match_finite_differences():
    """dG/dw = -y^T x and dG/deta = i y^T x against central differences of the dense solves
    (step 1e-5, error O(h^2))."""
    from oracle import grad
    inp = synth.make_inputs(4, 8, 1001)
    hb = hbar.build(inp)
    M = sg.dense_matrix(hb)
    B, C = bc.b_vectors(inp, range(6)), bc.c_vectors(inp, range(6))
    ws = np.array([-0.9, -0.55, -0.2])
    eta, h = 0.02, 1e-5
    G, dw, de = grad.derivatives(M, B, C, ws, eta)
    Gp = sv.green(C, sv.dense_solve(M, B, ws + h, eta))
    Gm = sv.green(C, sv.dense_solve(M, B, ws - h, eta))
    assert np.abs((Gp - Gm) / (2 * h) - dw).max() <= 1e-6 * np.abs(dw).max()
    Gp = sv.green(C, sv.dense_solve(M, B, ws, eta + h))
    Gm = sv.green(C, sv.dense_solve(M, B, ws, eta - h))
    assert np.abs((Gp - Gm) / (2 * h) - de).max() <= 1e-6 * np.abs(de).max()
    # G itself is the forward product
    assert np.abs(G - sv.green(C, sv.dense_solve(M, B, ws, eta))).max() <= 1e-12 * np.abs(G).max()


def test_t2_gradient_matches_finite_differences_of_the_loss():
    """dL/dt_ij^ab (L = Re sum conj(Gbar) G) from the chain rule with exact operator derivatives,
    against central differences of L itself (step 1e-5: O(h^2) truncation), with p and q sets that
    include virtual orbitals (b_a and c_i depend on T2)."""
    from oracle import grad
    inp = synth.random_amplitudes(synth.make_inputs(3, 5, 11), 7)
    porb, qorb = list(range(8)), [0, 2, 5, 7]
    ws, eta = np.array([-0.7, -0.3]), 0.05
    rng = np.random.default_rng(0)
    Gb = rng.standard_normal((2, 8, 4)) + 1j * rng.standard_normal((2, 8, 4))
    g = grad.green_t2_gradient(inp, porb, qorb, ws, eta, Gb)
    h = 1e-5
    for (i, j, a, b) in [(0, 1, 0, 1), (0, 2, 1, 4), (1, 2, 2, 3), (0, 1, 3, 4)]:
        Lp = grad.green_loss(grad._perturbed(inp, i, j, a, b, h), porb, qorb, ws, eta, Gb)
        Lm = grad.green_loss(grad._perturbed(inp, i, j, a, b, -h), porb, qorb, ws, eta, Gb)
        assert abs((Lp - Lm) / (2 * h) - g[i, j, a, b]) <= 1e-7 * np.abs(g).max()
    # entries that are not independent amplitudes stay zero
    assert np.all(g[1, 0] == 0.0) and np.all(g[:, :, 2, 1] == 0.0)


def test_operator_is_affine_in_t2():
    """M, b and c are affine in T2 at fixed T1 (every H-bar element is at most linear in T2), so
    central differences of any step give the same derivative; this is what makes the oracle's
    operator derivatives exact."""
    from oracle import grad
    inp = synth.random_amplitudes(synth.make_inputs(3, 5, 12), 8)
    porb = qorb = list(range(8))
    for (i, j, a, b) in [(0, 1, 0, 1), (1, 2, 3, 4)]:
        d = []
        for h in (1e-3, 0.3):
            Mp, Bp, Cp = grad._operators(grad._perturbed(inp, i, j, a, b, h), porb, qorb)
            Mm, Bm, Cm = grad._operators(grad._perturbed(inp, i, j, a, b, -h), porb, qorb)
            d.append([(Mp - Mm) / (2 * h), (Bp - Bm) / (2 * h), (Cp - Cm) / (2 * h)])
        for x, y in zip(d[0], d[1]):
            assert np.abs(x - y).max() <= 1e-9 * max(np.abs(y).max(), 1.0)


def test_reduced_green_derivative_and_derivative_indicator():
    """dGhat/dw = -chat^T (w - i eta + Hhat)^{-2} bhat against central differences of Ghat; with a
    two-point residual grid the derivative indicator alone drives the refinement, which ends with every
    sampled derivative mismatch below the tolerance."""
    from oracle import mor
    inp = synth.make_inputs(4, 8, 1001)
    hb = hbar.build(inp)
    M = sg.dense_matrix(hb)
    porb = list(range(3))
    B, C = bc.b_vectors(inp, porb), bc.c_vectors(inp, porb)
    S, _ = mor.orthonormalise(None, sv.dense_solve(M, B, [-0.9, -0.5], 0.02).reshape(-1, inp.dim).T)
    rm = mor.project(hb, S, B, C)
    ws, h = np.array([-0.8, -0.3]), 1e-6
    d = mor.reduced_green_derivative(rm, ws, 0.02)
    fd = (mor.reduced_green(rm, ws + h, 0.02) - mor.reduced_green(rm, ws - h, 0.02)) / (2 * h)
    assert np.abs(d - fd).max() <= 1e-6 * np.abs(d).max()
    r0 = mor.build_and_refine(hb, B, C, [-1.0, -0.6, -0.2], -1.0, -0.2, 2, 0.02, 1e-6, 10 ** 6, M=M)
    assert r0.sampled == [-1.0, -0.6, -0.2]
    r1 = mor.build_and_refine(hb, B, C, [-1.0, -0.6, -0.2], -1.0, -0.2, 2, 0.02, 1e-6, 10 ** 6, M=M, deriv=True)
    assert r1.converged and len(r1.sampled) > 3
    dG = {}
    for w in r1.sampled:
        X = sv.dense_solve(M, B, [w], 0.02)[0]
        A = (w - 0.02j) * np.eye(M.shape[0]) + M
        dG[w] = -(C @ np.linalg.solve(A, X.T)).T
    assert mor.derivative_mismatch(r1.model, r1.sampled, dG, 0.02).max() <= 1e-6


def test_model_extrapolated_initial_guess():
    """Solves at refinement frequencies started from the reduced model's prediction x0 = S yhat: the
    initial residual equals the model's residual estimate (Galerkin), the refined model and samples are
    the same as from zero guesses, and the GMRES iterations of those solves drop."""
    from oracle import mor
    inp = synth.make_inputs(7, 13, 103)
    hb = hbar.build(inp)
    porb = list(range(3))
    B, C = bc.b_vectors(inp, porb), bc.c_vectors(inp, porb)
    S, _ = mor.orthonormalise(None, sv.gmres_solve(hb, B, [-0.9, -0.3], 0.02, tol=1e-11)[0].reshape(-1, inp.dim).T)
    rm = mor.project(hb, S, B, C)
    w = -0.6
    x0 = S @ mor.reduced_solve(rm, [w], 0.02)[0].T                 # [D, np]
    r0 = np.linalg.norm(B.T - ((w - 0.02j) * x0 + sg.sigma(hb, x0.T).T), axis=0) / np.linalg.norm(B, axis=1)
    assert np.allclose(r0, mor.residuals(rm, B, [w], 0.02)[0], rtol=1e-8)
    runs = {}
    for g in (False, True):
        st = {}
        runs[g] = (mor.build_and_refine(hb, B, C, [-1.0, -0.2], -1.0, -0.2, 41, 0.02, 1e-6, 10 ** 6,
                                        solver="gmres", solve_tol=1e-11, guess=g, stats=st), st)
    assert runs[True][0].sampled == runs[False][0].sampled
    grid = np.linspace(-1.0, -0.2, 17)
    G0 = mor.reduced_green(runs[False][0].model, grid, 0.02)
    G1 = mor.reduced_green(runs[True][0].model, grid, 0.02)
    assert np.abs(G1 - G0).max() <= 1e-8 * np.abs(G0).max()
    assert runs[True][1]["gmres_iters"] < runs[False][1]["gmres_iters"]


def test_krylov_model_matches_moments_and_is_exact_when_complete():
    """Galerkin projection onto K_k(M, B): the reduced model reproduces the moments c_q^T M^j b_p for
    j = 0 .. k-1 (the leading terms of G's expansion in 1/(w - i eta)), for every p, q; once the space
    is invariant (it holds every M^j b_p) the model is exact at every frequency; and the refinement
    grows the space until its residuals meet the tolerance."""
    inp, hb, B, C, M = _mor_case()
    k = 4
    rm, st = mor.build_krylov(hb, B, C, k)
    assert st.blocks == k and rm.m == k * B.shape[0]
    Mj_B = B.T.astype(complex)
    Hj_b = rm.bhat
    for j in range(k):
        ref = C @ Mj_B                                   # [nq, np]
        assert np.abs(rm.chat @ Hj_b - ref).max() <= 1e-10 * np.abs(ref).max(), j
        Mj_B = M @ Mj_B
        Hj_b = rm.Hhat @ Hj_b
    # moment k is not matched in general (the test is not vacuous)
    assert np.abs(rm.chat @ Hj_b - C @ Mj_B).max() > 1e-8 * np.abs(C @ Mj_B).max()
    rm_full, st_full = mor.build_krylov(hb, B, C, 200)
    assert rm_full.m == M.shape[0] and st_full.newest == 0
    ws = np.linspace(-1.2, -0.3, 11)
    G = sv.green(C, sv.dense_solve(M, B, ws, 0.01))
    assert np.abs(mor.reduced_green(rm_full, ws, 0.01) - G).max() <= 1e-9 * np.abs(G).max()
    rm_r, st_r, hist, ok = mor.refine_krylov(hb, B, C, 2, -1.2, -0.3, 200, 0.01, 1e-6, 10 ** 6)
    assert ok and hist[-1][1] <= 1e-6 and hist[0][1] > 1e-6 and rm_r.m < M.shape[0]
