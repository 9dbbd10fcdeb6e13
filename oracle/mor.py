"""Model-order reduction of the IP-GFCC MIMO system (oracle, FP64).

Test infrastructure: only tests, the smoke check and the CPU baseline use the oracle.

Follows the MOR section of the paper (Eqs. gfcclineqn and model, and the text after them):
* the subspace S holds the orthonormalised auxiliary vectors X_p(w_k) solved at selected
  frequencies w_k; orthonormality <v_i|v_j> = delta_ij is taken in the complex inner product, so the
  projections written S^T in Eq. model are read as S^H (conjugate transpose);
* the reduced model is Hhat = S^H M S, bhat = S^H b, chat^T = c^T S, solved as
  (w - i eta + Hhat) yhat_p(w) = bhat_p, Ghat_pq(w) = chat_q^T yhat_p(w);
* adaptive refinement: start from frequencies spread evenly over [w_min, w_max] (both ends
  included); estimate the error between adjacent sampled frequencies; add the midpoints of the
  intervals whose estimate is above the threshold; stop when every estimate is below it or the
  model order would exceed its bound.

Readings where the paper is silent (each listed in the design notes):
* orthonormalisation: each new column in turn loses its components along the current basis by
  two classical Gram-Schmidt passes; it is kept when its remaining norm is at least 1e-10 of its
  norm before the passes, else dropped (rank truncation);
* error estimate of an interval: the largest relative residual ||(w - i eta + M) S yhat_p - b_p|| /
  ||b_p|| over the grid points strictly inside it and over all p; here computed with explicit
  D-length vectors;
* every interval above the threshold gets its midpoint in one round; if the order bound would be
  exceeded, the largest estimates go first (ties: lower frequency first).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import sigma as sg
from . import solve as sv


def orthonormalise(S: np.ndarray | None, Y: np.ndarray, drop_tol: float = 1e-10):
    """Append the columns of Y ([D, k]) to the orthonormal columns of S ([D, m]). Returns (S', kept)."""
    cols = [] if S is None else [S[:, j] for j in range(S.shape[1])]
    kept = []
    for j in range(Y.shape[1]):
        y = Y[:, j].astype(complex)
        n0 = np.linalg.norm(y)
        if n0 == 0.0:
            kept.append(False)
            continue
        for _ in range(2):
            if cols:
                B = np.stack(cols, axis=1)
                y = y - B @ (B.conj().T @ y)
        n1 = np.linalg.norm(y)
        if n1 >= drop_tol * n0:
            cols.append(y / n1)
            kept.append(True)
        else:
            kept.append(False)
    return np.stack(cols, axis=1), kept


@dataclass
class ReducedModel:
    S: np.ndarray            # [D, m]
    Z: np.ndarray            # [D, m] = M S
    Hhat: np.ndarray         # [m, m]
    bhat: np.ndarray         # [m, np]
    chat: np.ndarray         # [nq, m]
    sampled: list = field(default_factory=list)

    @property
    def m(self) -> int:
        return self.S.shape[1]


def project(hb, S: np.ndarray, B: np.ndarray, C: np.ndarray) -> ReducedModel:
    """Galerkin projection of Eq. model with explicit sigma columns Z = M S."""
    Z = sg.sigma(hb, S.T).T
    return ReducedModel(S=S, Z=Z, Hhat=S.conj().T @ Z, bhat=S.conj().T @ B.T, chat=C @ S)


def reduced_solve(rm: ReducedModel, omegas, eta: float) -> np.ndarray:
    """yhat[w, p, :] = (w - i eta + Hhat)^{-1} bhat_p."""
    I = np.eye(rm.m)
    return np.array([np.linalg.solve((w - 1j * eta) * I + rm.Hhat, rm.bhat).T for w in omegas])


def reduced_green(rm: ReducedModel, omegas, eta: float) -> np.ndarray:
    """Ghat[w, p, q] = chat_q^T yhat_p(w)."""
    Y = reduced_solve(rm, omegas, eta)
    return np.einsum("qm,wpm->wpq", rm.chat, Y)


def residuals(rm: ReducedModel, B: np.ndarray, omegas, eta: float) -> np.ndarray:
    """Relative residual ||(w - i eta) S y + Z y - b_p|| / ||b_p|| for every (w, p)."""
    Y = reduced_solve(rm, omegas, eta)
    bn = np.linalg.norm(B, axis=1)
    out = np.empty((len(omegas), B.shape[0]))
    for k, w in enumerate(omegas):
        R = (w - 1j * eta) * (rm.S @ Y[k].T) + rm.Z @ Y[k].T - B.T
        out[k] = np.linalg.norm(R, axis=0) / bn
    return out


def interval_errors(sampled, grid, res) -> np.ndarray:
    """e_k = max residual over grid points strictly inside (sampled[k], sampled[k+1])."""
    s = np.sort(np.asarray(sampled))
    per_w = res.max(axis=1)
    e = np.zeros(len(s) - 1)
    for k in range(len(s) - 1):
        inside = (grid > s[k]) & (grid < s[k + 1])
        if inside.any():
            e[k] = per_w[inside].max()
    return e


def choose_midpoints(sampled, errors, tol: float, max_new: int):
    s = np.sort(np.asarray(sampled))
    cand = [(-errors[k], 0.5 * (s[k] + s[k + 1])) for k in range(len(errors)) if errors[k] > tol]
    cand.sort()
    return sorted(w for _, w in cand[:max(max_new, 0)])


def reduced_green_derivative(rm: ReducedModel, omegas, eta: float) -> np.ndarray:
    """dGhat/dw [w, p, q] = -chat_q^T (w - i eta + Hhat)^{-2} bhat_p."""
    I = np.eye(rm.m)
    out = []
    for w in omegas:
        A = (w - 1j * eta) * I + rm.Hhat
        Y = np.linalg.solve(A, np.linalg.solve(A, rm.bhat))      # [m, np]
        out.append(-(rm.chat @ Y).T)
    return np.array(out)


def derivative_mismatch(rm: ReducedModel, sampled, dG_exact: dict, eta: float) -> np.ndarray:
    """d_k = max_pq |dGhat/dw - dG/dw| / max_pq |dG/dw| at every sampled frequency (sorted)."""
    s = sorted(sampled)
    dh = reduced_green_derivative(rm, s, eta)
    return np.array([np.abs(dh[k] - dG_exact[w]).max() / max(np.abs(dG_exact[w]).max(), 1e-300)
                     for k, w in enumerate(s)])


@dataclass
class MorResult:
    model: ReducedModel
    sampled: list
    history: list            # (m, max interval error) per round
    converged: bool


def build_and_refine(hb, B: np.ndarray, C: np.ndarray, seeds, wmin: float, wmax: float,
                     ngrid: int, eta: float, tol: float, m_max: int, solver="dense",
                     M: np.ndarray | None = None, solve_tol: float = 1e-10, deriv: bool = False,
                     guess: bool = False, stats: dict | None = None) -> MorResult:
    """Adaptive MOR: solve at the seeds, orthonormalise, project, refine until tolerance.

    deriv: add the frequency-derivative indicator (reading of the derivative-driven selection): at
    every sampled w_k the exact dG/dw = -c^T A^{-1} x (one more solve per column) is compared with the
    reduced model's, d_k = max |dGhat/dw - dG/dw| / max |dG/dw|, and an interval's error becomes
    max(e_k, d_k, d_{k+1}).
    guess: (GMRES solver) solves at added frequencies start from the current model's prediction
    x0_p(w) = S yhat_p(w) instead of zero; stats["gmres_iters"] counts the iterations of those solves."""
    grid = np.linspace(wmin, wmax, ngrid)
    npp = B.shape[0]

    def full(ws, model=None):
        if solver == "dense":
            return sv.dense_solve(M, B, ws, eta)
        if model is None or not guess:
            X, _ = sv.gmres_solve(hb, B, ws, eta, tol=solve_tol, stats=stats)
            return X
        Y = reduced_solve(model, ws, eta)                      # [nw, np, m]
        X0 = np.einsum("dm,wpm->wpd", model.S, Y)
        X, _ = sv.gmres_solve(hb, B, ws, eta, tol=solve_tol, x0=X0, stats=stats)
        return X

    def dfull(ws, X):
        """exact dG/dw [p, q] per w: -C A^{-1} x_p (dense or GMRES solves of A z = x)."""
        out = {}
        for k, w in enumerate(ws):
            if solver == "dense":
                A = (w - 1j * eta) * np.eye(M.shape[0]) + M
                Zk = np.linalg.solve(A, X[k].T).T                 # [np, D]
            else:
                Zk, _ = sv.gmres_solve(hb, X[k], [w], eta, tol=solve_tol)
                Zk = Zk[0]
            out[float(w)] = -(C @ Zk.T).T
        return out

    sampled = sorted(float(w) for w in seeds)
    X = full(sampled)                                    # [nw, np, D]
    dG = dfull(sampled, X) if deriv else {}
    S, _ = orthonormalise(None, X.reshape(-1, X.shape[-1]).T)
    rm = project(hb, S, B, C)
    history = []
    converged = False
    while True:
        res = residuals(rm, B, grid, eta)
        e = interval_errors(sampled, grid, res)
        if deriv:
            d = derivative_mismatch(rm, sampled, dG, eta)
            e = np.maximum(e, np.maximum(d[:-1], d[1:]))
        emax = float(e.max()) if len(e) else 0.0
        history.append((rm.m, emax))
        if emax <= tol:
            converged = True
            break
        max_new = (m_max - rm.m) // npp
        new = choose_midpoints(sampled, e, tol, max_new)
        if not new:
            break
        Xn = full(new, rm)
        if deriv:
            dG.update(dfull(new, Xn))
        S, _ = orthonormalise(rm.S, Xn.reshape(-1, Xn.shape[-1]).T)
        sampled = sorted(sampled + new)
        rm = project(hb, S, B, C)
    rm.sampled = sampled
    return MorResult(model=rm, sampled=sampled, history=history, converged=converged)


def build_and_refine_siso(hb, B: np.ndarray, C: np.ndarray, seeds, wmin: float, wmax: float, ngrid: int,
                          eta: float, tol: float, m_max: int, solver="dense", M: np.ndarray | None = None,
                          solve_tol: float = 1e-10) -> list:
    """Separate single-input single-output reduced models of the diagonal elements G_pp (the conclusion's
    proposal): for every orbital p (row p of B and of C, the same orbital), the adaptive reduced model
    above built from X_p(w_k) alone, with b_p as its only input and c_p as its only output. Returns one
    MorResult per orbital; each model refines its own frequencies, and m_max bounds each model's order."""
    return [build_and_refine(hb, B[p:p + 1], C[p:p + 1], seeds, wmin, wmax, ngrid, eta, tol, m_max,
                             solver=solver, M=M, solve_tol=solve_tol) for p in range(B.shape[0])]


def siso_green(results: list, omegas, eta: float) -> np.ndarray:
    """G[w, p, q] with Ghat_pp of the per-orbital models on the diagonal and zeros elsewhere."""
    npp = len(results)
    G = np.zeros((len(omegas), npp, npp), dtype=complex)
    for p, r in enumerate(results):
        G[:, p, p] = reduced_green(r.model, omegas, eta)[:, 0, 0]
    return G


class KrylovState:
    """Block Krylov basis under construction: S (orthonormal columns so far), X (the next block to add),
    blocks added, and the number of columns the newest block kept."""

    def __init__(self, B: np.ndarray):
        self.S = None
        self.X = B.T.astype(complex)                     # first block: [D, np]
        self.blocks = 0
        self.newest = 0

    @property
    def m(self) -> int:
        return 0 if self.S is None else self.S.shape[1]

    def extend(self, hb, nblocks: int, m_max: int, drop_tol: float = 1e-10) -> None:
        """Add up to nblocks blocks; stop before a block whose columns would exceed m_max, or when the
        space is invariant (a block keeps no column). Each block is orthonormalised against the basis
        (two classical Gram-Schmidt passes per column, rank truncation as in orthonormalise); the next
        block is M applied to the columns just kept."""
        for _ in range(nblocks):
            if self.X.shape[1] == 0 or self.m + self.X.shape[1] > m_max:
                return
            m0 = self.m
            self.S, _ = orthonormalise(self.S, self.X, drop_tol)
            self.blocks += 1
            self.newest = self.S.shape[1] - m0
            self.X = sg.sigma(hb, self.S[:, m0:].T).T    # M times the new orthonormal columns
            if self.newest == 0:
                return


def build_krylov(hb, B: np.ndarray, C: np.ndarray, nblocks: int, drop_tol: float = 1e-10):
    """Reduced model on the block Krylov space K_k(M, B) = span[B, M B, ..., M^(k-1) B], k = nblocks
    (multi-shift reuse: the space is the same for every shifted matrix w - i eta + M)."""
    st = KrylovState(B)
    st.extend(hb, nblocks, 2 ** 31 - 1, drop_tol)
    return project(hb, st.S, B, C), st


def refine_krylov(hb, B: np.ndarray, C: np.ndarray, nblocks0: int, wmin: float, wmax: float, ngrid: int,
                  eta: float, tol: float, m_max: int, drop_tol: float = 1e-10):
    """Grow the Krylov model until the largest relative residual over the whole grid is <= tol: each round
    adds max(1, floor(k/4)) blocks (k the blocks so far) within the order bound m_max. Returns (model,
    KrylovState, history of (m, max residual), converged)."""
    grid = np.linspace(wmin, wmax, ngrid)
    st = KrylovState(B)
    st.extend(hb, nblocks0, 2 ** 31 - 1, drop_tol)
    rm = project(hb, st.S, B, C)
    history = []
    while True:
        e = float(residuals(rm, B, grid, eta).max())
        history.append((rm.m, e))
        if e <= tol:
            return rm, st, history, True
        m0 = st.m
        st.extend(hb, max(1, st.blocks // 4), m_max, drop_tol)
        if st.m == m0:
            return rm, st, history, False
        rm = project(hb, st.S, B, C)
