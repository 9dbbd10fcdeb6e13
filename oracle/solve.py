"""Full-dimension solves of the IP-GFCC systems and the Green's function read-out (oracle, FP64).

Test infrastructure: only tests, the smoke check and the CPU baseline use the oracle.

* Eq. xplin: (w - i eta + M) X_p(w) = b_p, solved either by dense LU of the explicit matrix
  (small D) or by plain restarted GMRES (Saad and Schultz 1986) with a Jacobi right
  preconditioner and modified Gram-Schmidt Arnoldi (large D). The paper solved the same systems
  with a complex DIIS solver; any convergent solver reaches the same solution.
* Eq. gfxn2 / gfcclineqn: G_pq(w) = c_q^T X_p(w) (plain transpose, no conjugation).
* Spectral function A(w) = -(1/pi) sum_p Im G_pp(w), taken literally (with the -i eta sign of
  Eq. gfxn0 the peaks of this formula are negative; plots negate it).
"""
from __future__ import annotations

import numpy as np

from . import sigma as sg


def dense_solve(M: np.ndarray, B: np.ndarray, omegas, eta: float) -> np.ndarray:
    """X[w, p, :] = (w - i eta + M)^{-1} b_p for every w, by dense LU (np.linalg.solve)."""
    D = M.shape[0]
    I = np.eye(D)
    out = np.empty((len(omegas), B.shape[0], D), dtype=complex)
    for k, w in enumerate(omegas):
        out[k] = np.linalg.solve((w - 1j * eta) * I + M, B.T.astype(complex)).T
    return out


def gmres(matvec, b: np.ndarray, shift: complex, diag: np.ndarray, tol: float = 1e-10,
          restart: int = 30, maxiter: int = 2000, x0=None):
    """Solve (shift + M) x = b with right Jacobi preconditioning (shift + diag)^{-1}.

    Returns (x, relative residual history per iteration, converged flag). The residual that
    decides convergence is recomputed explicitly at every restart."""
    b = b.astype(complex)
    pinv = 1.0 / (shift + diag)
    x = np.zeros_like(b) if x0 is None else x0.astype(complex).copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, [0.0], True
    hist = []
    it = 0
    while it < maxiter:
        r = b - (shift * x + matvec(x))
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta / bnorm <= tol:
            return x, hist, True
        V = [r / beta]
        H = np.zeros((restart + 1, restart), dtype=complex)
        cs = np.zeros(restart, dtype=complex)
        sn = np.zeros(restart, dtype=complex)
        g = np.zeros(restart + 1, dtype=complex)
        g[0] = beta
        k_done = 0
        for j in range(restart):
            z = pinv * V[j]
            w = shift * z + matvec(z)
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            hnext = np.linalg.norm(w)
            H[j + 1, j] = hnext
            for i in range(j):                           # apply earlier rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + np.conj(cs[i]) * H[i + 1, j]
                H[i, j] = t
            a, bb = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            cs[j] = np.conj(a) / den if den else 1.0
            sn[j] = np.conj(bb) / den if den else 0.0
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            k_done = j + 1
            it += 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= tol * 0.5 or it >= maxiter:
                break
            if hnext == 0.0:                             # exact (happy) breakdown
                break
            V.append(w / hnext)
        y = np.linalg.solve(np.triu(H[:k_done, :k_done]), g[:k_done])
        x = x + pinv * sum(y[i] * V[i] for i in range(k_done))
    r = b - (shift * x + matvec(x))
    hist.append(np.linalg.norm(r) / bnorm)
    return x, hist, hist[-1] <= tol


def gmres_solve(hb, B: np.ndarray, omegas, eta: float, tol: float = 1e-10, restart: int = 30,
                maxiter: int = 3000, x0=None, stats: dict | None = None) -> tuple[np.ndarray, np.ndarray]:
    """X[w, p, :] by GMRES for every (w, p), with the oracle sigma as the matvec; x0[w, p, :] (optional)
    initial guesses; stats["gmres_iters"] (optional) accumulates the iterations.

    Returns (X, final relative residuals [nw, np])."""
    diag = sg.diagonal(hb)
    mv = lambda x: sg.sigma(hb, x)  # noqa: E731
    X = np.empty((len(omegas), B.shape[0], B.shape[1]), dtype=complex)
    res = np.empty((len(omegas), B.shape[0]))
    for k, w in enumerate(omegas):
        for p in range(B.shape[0]):
            x, hist, _ = gmres(mv, B[p], w - 1j * eta, diag, tol=tol, restart=restart,
                               maxiter=maxiter, x0=None if x0 is None else x0[k, p])
            if stats is not None:
                stats["gmres_iters"] = stats.get("gmres_iters", 0) + len(hist) - 1
            X[k, p] = x
            res[k, p] = hist[-1]
    return X, res


def green(C: np.ndarray, X: np.ndarray) -> np.ndarray:
    """G[w, p, q] = c_q^T X[w, p] (Eq. gfxn2)."""
    return np.einsum("qd,wpd->wpq", C, X)


def spectral(G: np.ndarray, diag_index=None) -> np.ndarray:
    """A(w) = -(1/pi) sum_p Im G_pp(w); ``diag_index[p]`` gives the q position of orbital p
    (default: the p and q sets are the same list)."""
    nw, npp, nq = G.shape
    if diag_index is None:
        diag_index = list(range(npp))
    tr = sum(G[:, p, diag_index[p]] for p in range(npp))
    return -np.imag(tr) / np.pi
