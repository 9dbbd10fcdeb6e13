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
