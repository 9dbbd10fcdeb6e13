"""Pins of the electron-attachment (1p + 2p1h) oracle against things other than itself (CPU only).

* brute-force second quantisation in the N+1 sector (explicit determinants, e^{-T} H e^{T}) for M, b_q,
  c_p at random amplitudes and several shapes, each amplitude block shown to matter;
* closed forms: Koopmans poles 1/(w - eps_a + i eta) when T = Lambda = 0 and v = 1 (no 2p1h space);
  the exact attachment resolvent over the whole N+1 sector when T = Lambda = 0 and v = 2;
* the IP form of the same systems (negated frequencies, negated free terms) gives the same G, with
  the IP oracle's dense solver and reduced model;
* the generator's packed vvvv block is a slice of the full integral tensor.
"""
import numpy as np
import pytest

import synth
from oracle import ea, fockspace, mor
from oracle import solve as sv


def _random_case(o, v, seed):
    return synth.random_amplitudes(synth.make_inputs(o, v, seed, scale_mode="literal"), seed + 1)


@pytest.mark.parametrize("o,v,seed", [(2, 3, 5), (3, 4, 11), (2, 5, 7), (4, 3, 17), (3, 5, 19), (1, 6, 23)])
def test_ea_sigma_b_c_match_brute_force(o, v, seed):
    inp = _random_case(o, v, seed)
    bf = fockspace.build_ea_from_inputs(inp)
    M = ea.dense_matrix(ea.build(inp))
    assert np.abs(M - bf.M).max() <= 1e-12 * np.abs(bf.M).max()
    assert np.abs(ea.b_vectors(inp) - bf.b).max() <= 1e-12
    assert np.abs(ea.c_vectors(inp) - bf.c).max() <= 1e-12


@pytest.mark.parametrize("part", ["t1", "t2", "l1", "l2"])
def test_ea_each_amplitude_block_matters(part):
    inp = _random_case(3, 4, 21)
    bf = fockspace.build_ea_from_inputs(inp)
    getattr(inp, part)[:] = 0.0
    dM = np.abs(ea.dense_matrix(ea.build(inp)) - bf.M).max()
    db = np.abs(ea.b_vectors(inp) - bf.b).max()
    dc = np.abs(ea.c_vectors(inp) - bf.c).max()
    assert max(dM, db, dc) > 1e-4


def test_ea_each_hbar_term_matters():
    """Dropping the vvvv integrals or the three-body term changes M: both are exercised by the pin."""
    inp = _random_case(3, 4, 29)
    bf = fockspace.build_ea_from_inputs(inp)
    hb = ea.build(inp, vvvv=np.zeros((4, 4, 4, 4)))
    assert np.abs(ea.dense_matrix(hb) - bf.M).max() > 1e-3
    hb = ea.build(inp)
    hb.Vmnef = np.zeros_like(hb.Vmnef)
    assert np.abs(ea.dense_matrix(hb) - bf.M).max() > 1e-4


def test_ea_tiny_workload_brute_force():
    """The o=4, v=8 workload with its MP2-like amplitudes (792-determinant N+1 sector)."""
    W = synth.WORKLOADS["tiny_o4_v8"]
    inp = synth.make_inputs(W["o"], W["v"], W["seed"])
    bf = fockspace.build_ea_from_inputs(inp)
    M = ea.dense_matrix(ea.build(inp))
    assert np.abs(M - bf.M).max() <= 1e-12
    assert np.abs(ea.b_vectors(inp) - bf.b).max() <= 1e-13
    assert np.abs(ea.c_vectors(inp) - bf.c).max() <= 1e-13


def test_ea_koopmans_limit():
    """T = Lambda = 0, v = 1: G^EA_aa(w) = 1/(w - eps_a + i eta), zero for occupied p or q."""
    inp = synth.make_inputs(3, 1, 4, with_t=False, with_lambda=False)
    M = ea.dense_matrix(ea.build(inp))
    ws = np.linspace(-1, 3, 11)
    eta = 0.01
    G = ea.green(ea.c_vectors(inp), ea.dense_solve(M, ea.b_vectors(inp), ws, eta))
    ref = np.zeros_like(G)
    ref[:, 3, 3] = 1.0 / (ws - inp.eps[3] + 1j * eta)
    assert np.abs(G - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("o,seed", [(2, 7), (4, 8)])
def test_ea_exact_resolvent_when_space_is_complete(o, seed):
    """T = Lambda = 0 and v = 2: 1p+2p1h is the whole N+1 sector, so the attachment term of the retarded
    Green's function is reproduced exactly for every (p, q)."""
    inp = synth.make_inputs(o, 2, seed, scale_mode="literal", with_t=False, with_lambda=False)
    bf = fockspace.build_ea_from_inputs(inp)
    M = ea.dense_matrix(ea.build(inp))
    ws = np.linspace(-0.5, 2.5, 9)
    eta = 0.02
    G = ea.green(ea.c_vectors(inp), ea.dense_solve(M, ea.b_vectors(inp), ws, eta))
    Gx = fockspace.exact_resolvent_ea(bf, ws, eta)
    assert np.abs(G - Gx).max() <= 1e-12 * np.abs(Gx).max()


def test_ea_ip_form_gives_the_same_green_function():
    """(w' - i eta + M) y = -b at w' = -w with the IP oracle's solver and read-out = G^EA (transposed
    read-out: column q is the free term, row p the left vector); and the IP oracle's reduced model on the
    IP form interpolates G^EA at its sampled frequencies."""
    inp = synth.make_inputs(3, 6, 41)
    hb = ea.build(inp)
    M = ea.dense_matrix(hb)
    qorb = list(range(9))
    B, C = ea.b_vectors(inp, qorb), ea.c_vectors(inp, qorb)
    ws = np.linspace(0.2, 2.0, 7)
    eta = 0.01
    G = ea.green(C, ea.dense_solve(M, B, ws, eta))                     # [w, p, q]
    Bp, Cp = ea.ip_form(inp, hb, qorb, qorb)
    Gip = sv.green(Cp, sv.dense_solve(M, Bp, -ws, eta))                # [w, q, p]
    assert np.abs(Gip.transpose(0, 2, 1) - G).max() <= 1e-12 * np.abs(G).max()
    seeds = -np.array([0.3, 1.1, 1.9])
    rm = mor.project(hb, mor.orthonormalise(None, sv.dense_solve(M, Bp, seeds, eta).reshape(-1, M.shape[0]).T)[0],
                     Bp, Cp)
    Gh = mor.reduced_green(rm, seeds, eta)
    Gf = sv.green(Cp, sv.dense_solve(M, Bp, seeds, eta))
    assert np.abs(Gh - Gf).max() <= 1e-10 * np.abs(Gf).max()


def test_vvvv_pairs_is_a_slice_of_the_full_tensor():
    inp = synth.make_inputs(3, 5, 9, scale_mode="literal")
    g = inp.full_antisym()
    full = ea.unpack_vvvv(inp.vvvv_pairs(), 5)
    assert np.array_equal(full, g[3:, 3:, 3:, 3:])
