"""Frequency and broadening derivatives of the IP-GFCC Green's function (oracle, FP64).

Test infrastructure: only tests, the smoke check and the CPU baseline use the oracle.

G_pq(w) = c_q^T A(w)^{-1} b_p with A(w) = w - i eta + M (Eqs. gfcclineqn and xplin). Since dA/dw = 1 and
dA/deta = -i:
  dG_pq/dw   = -c_q^T A^{-1} A^{-1} b_p = -y_q^T x_p,
  dG_pq/deta = +i c_q^T A^{-2} b_p      =  i y_q^T x_p,
with x_p = A^{-1} b_p and the adjoint (left) solutions y_q = A^{-T} c_q. Computed here with dense LU.
"""
from __future__ import annotations

import numpy as np


def derivatives(M: np.ndarray, B: np.ndarray, C: np.ndarray, omegas, eta: float):
    """Returns (G, dG/dw, dG/deta), each [nw, np, nq], by dense solves of A and A^T."""
    D = M.shape[0]
    I = np.eye(D)
    G, dw, de = [], [], []
    for w in omegas:
        A = (w - 1j * eta) * I + M
        X = np.linalg.solve(A, B.T.astype(complex))          # [D, np]
        Y = np.linalg.solve(A.T, C.T.astype(complex))        # [D, nq]
        G.append((C @ X).T)
        YX = (Y.T @ X).T                                     # [np, nq] = y_q^T x_p
        dw.append(-YX)
        de.append(1j * YX)
    return np.array(G), np.array(dw), np.array(de)


# ---- gradient with respect to the doubles amplitudes ---------------------------------------------
# L = Re sum_{w,p,q} conj(Gbar_wpq) G_pq(w) for given weights Gbar (the vector-Jacobian product that an
# autograd backward pass needs). With x_p = A^{-1} b_p and y_q = A^{-T} c_q, the chain rule gives, for
# any amplitude t,
#   dL/dt = Re sum conj(Gbar_wpq) [ (dc_q/dt)^T x_p + y_q^T (db_p/dt) - y_q^T (dM/dt) x_p ].
# M, b and c are affine in t_ij^ab (every H-bar element above is at most linear in T2 at fixed T1), so
# their derivatives are exact as central differences of the oracle's own builds.

def _perturbed(inp, i, j, a, b, h):
    """Inputs with the independent amplitude t_ij^ab (i<j, a<b) moved by h (antisymmetry kept)."""
    import dataclasses
    t2 = inp.t2.copy()
    t2[i, j, a, b] += h
    t2[j, i, a, b] -= h
    t2[i, j, b, a] -= h
    t2[j, i, b, a] += h
    return dataclasses.replace(inp, t2=t2)


def _operators(inp, porb, qorb):
    from . import bc, hbar
    from . import sigma as sg
    return sg.dense_matrix(hbar.build(inp)), bc.b_vectors(inp, porb), bc.c_vectors(inp, qorb)


def green_loss(inp, porb, qorb, omegas, eta, Gbar) -> float:
    """L = Re sum conj(Gbar) G by dense solves."""
    M, B, C = _operators(inp, porb, qorb)
    G = derivatives(M, B, C, omegas, eta)[0]
    return float(np.real(np.sum(np.conj(Gbar) * G)))


def green_t2_gradient(inp, porb, qorb, omegas, eta, Gbar, h: float = 1e-3) -> np.ndarray:
    """dL/dt_ij^ab for every independent amplitude (i<j, a<b), as an [o,o,v,v] array holding the
    value at [i,j,a,b] (zero elsewhere). Dense solves; small sizes only."""
    o, v = inp.o, inp.v
    M, B, C = _operators(inp, porb, qorb)
    D = M.shape[0]
    I = np.eye(D)
    XS, YS = [], []
    for w in omegas:
        A = (w - 1j * eta) * I + M
        XS.append(np.linalg.solve(A, B.T.astype(complex)))     # [D, np]
        YS.append(np.linalg.solve(A.T, C.T.astype(complex)))   # [D, nq]
    out = np.zeros((o, o, v, v))
    for i in range(o):
        for j in range(i + 1, o):
            for a in range(v):
                for b in range(a + 1, v):
                    Mp, Bp, Cp = _operators(_perturbed(inp, i, j, a, b, h), porb, qorb)
                    Mm, Bm, Cm = _operators(_perturbed(inp, i, j, a, b, -h), porb, qorb)
                    dM, dB, dC = (Mp - Mm) / (2 * h), (Bp - Bm) / (2 * h), (Cp - Cm) / (2 * h)
                    s = 0.0
                    for k in range(len(omegas)):
                        X, Y = XS[k], YS[k]
                        dG = (dC @ X).T + (Y.T @ dB.T).T - (Y.T @ dM @ X).T    # [np, nq]
                        s += np.real(np.sum(np.conj(Gbar[k]) * dG))
                    out[i, j, a, b] = s
    return out
