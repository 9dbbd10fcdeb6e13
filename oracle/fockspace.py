"""Brute-force Fock-space construction of the IP-GFCC objects (test infrastructure, CPU only).

Part of the oracle: only tests, the smoke check and the CPU baseline use it.

Everything here is built from second quantisation on explicit determinants, with no
coupled-cluster algebra at all, so that it can pin the oracle's closed-form intermediates,
sigma equations and free/left vectors:

* Slater determinants are bit strings over n spin-orbitals; a_p carries the Jordan-Wigner
  sign (-1)^(number of occupied orbitals below p).
* H = sum h_pq a_p^+ a_q + 1/4 sum <pq||rs> a_p^+ a_q^+ a_s a_r, with h_pq = f_pq - sum_i <pi||qi>
  and f = diag(eps), so that the reference Phi (lowest o orbitals) has Fock matrix diag(eps).
* T = sum t_i^a a_a^+ a_i + 1/4 sum t_ij^ab a_a^+ a_b^+ a_j a_i,
  Lambda = sum l_a^i a_i^+ a_a + 1/4 sum l_ab^ij a_i^+ a_j^+ a_b a_a.
* Hbar = e^{-T} H e^{T} (Eq. gfxn1 text), built as dense matrices in the N and N-1 electron sectors.
* M_{mu,nu} = <mu| Hbar R_nu |Phi> - <mu| R_nu Hbar |Phi> over the 1h + 2h1p operators
  R = {a_k} u {a_c^+ a_l a_k, k<l} of Eq. xp: the connected action of Hbar_N on X_p|Phi>
  (equal to Hbar - E_0 of Eq. xplin whenever T solves the CC equations).
* b_p = projection of e^{-T} a_p e^{T} |Phi> on the 1h+2h1p determinants (right side of Eq. xplin).
* c_q[nu] = <Phi| (1 + Lambda) e^{-T} a_q^+ e^{T} R_nu |Phi> (Eq. gfxn2, G_pq = c_q^T X_p).
* The exact resolvent <Phi| a_q^+ (w - i eta + H - E_HF)^{-1} a_p |Phi> over the whole N-1 sector
  (Eq. gfxn0 with Psi = Phi), which the truncated method must reproduce when T = Lambda = 0 and
  the 1h+2h1p space is the whole N-1 sector (o = 2).

Basis order of the 1h+2h1p space: index k for a_k|Phi>, then o + pair(k,l)*v + c for
a_{o+c}^+ a_l a_k |Phi> with k < l and pair(k,l) = l(l-1)/2 + k.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np


def sector(n: int, N: int) -> tuple[list[int], dict[int, int]]:
    dets = [sum(1 << b for b in c) for c in itertools.combinations(range(n), N)] if N >= 0 else []
    dets.sort()
    return dets, {d: k for k, d in enumerate(dets)}


def annihilator(n: int, p: int, N: int) -> np.ndarray:
    """Matrix of a_p from the N-electron sector to the (N-1)-electron sector."""
    src, _ = sector(n, N)
    dst, dst_idx = sector(n, N - 1)
    A = np.zeros((len(dst), len(src)))
    for k, d in enumerate(src):
        if d >> p & 1:
            sign = -1.0 if bin(d & ((1 << p) - 1)).count("1") % 2 else 1.0
            A[dst_idx[d & ~(1 << p)], k] = sign
    return A


class Sector:
    """Dense second-quantised operators inside the K-electron sector."""

    def __init__(self, n: int, K: int):
        self.n, self.K = n, K
        self.dets, self.index = sector(n, K)
        self.dim = len(self.dets)
        self.A = [annihilator(n, p, K) for p in range(n)]                 # K -> K-1
        self.A1 = [annihilator(n, p, K - 1) for p in range(n)] if K >= 1 else None  # K-1 -> K-2
        self.pairs = [(p, q) for q in range(n) for p in range(q)]
        # D[(p,q)] = a_q a_p (apply a_p first), K -> K-2
        self.D = {pq: self.A1[pq[1]] @ self.A[pq[0]] for pq in self.pairs} if K >= 2 else {}

    def one_body(self, h: np.ndarray) -> np.ndarray:
        """sum_pr h_pr a_p^+ a_r."""
        out = np.zeros((self.dim, self.dim))
        for p in range(self.n):
            for r in range(self.n):
                if h[p, r] != 0.0:
                    out += h[p, r] * (self.A[p].T @ self.A[r])
        return out

    def two_body(self, g: np.ndarray) -> np.ndarray:
        """1/4 sum_pqrs g_pqrs a_p^+ a_q^+ a_s a_r for g antisymmetric in (p,q) and in (r,s)."""
        if self.K < 2:
            return np.zeros((self.dim, self.dim))
        X = np.stack([self.D[pq] for pq in self.pairs])                  # [npair, d2, dK]
        gp = np.array([[g[p, q, r, s] for (r, s) in self.pairs] for (p, q) in self.pairs])
        W = np.tensordot(gp, X, axes=(1, 0))                              # [npair, d2, dK]
        return X.reshape(-1, self.dim).T @ W.reshape(-1, self.dim)

    def cluster(self, o: int, t1: np.ndarray, t2: np.ndarray) -> np.ndarray:
        """T = sum t_i^a a_a^+ a_i + 1/4 sum t_ij^ab a_a^+ a_b^+ a_j a_i."""
        n = self.n
        h = np.zeros((n, n))
        h[o:, :o] = t1.T
        g = np.zeros((n, n, n, n))
        g[o:, o:, :o, :o] = t2.transpose(2, 3, 0, 1)                     # g[a,b,i,j] = t_ij^ab
        return self.one_body(h) + self.two_body(g)

    def deexcitation(self, o: int, l1: np.ndarray, l2: np.ndarray) -> np.ndarray:
        """Lambda = sum l_a^i a_i^+ a_a + 1/4 sum l_ab^ij a_i^+ a_j^+ a_b a_a."""
        n = self.n
        h = np.zeros((n, n))
        h[:o, o:] = l1
        g = np.zeros((n, n, n, n))
        g[:o, :o, o:, o:] = l2                                           # g[i,j,a,b] = l_ab^ij
        return self.one_body(h) + self.two_body(g)


def expm_nilpotent(T: np.ndarray, max_order: int = 64) -> np.ndarray:
    """exp(T) by its terminating power series (T raises the excitation level, so T^k -> 0)."""
    out = np.eye(T.shape[0])
    term = np.eye(T.shape[0])
    for k in range(1, max_order + 1):
        term = term @ T / k
        if not np.any(term):
            return out
        out = out + term
    raise RuntimeError("cluster operator is not nilpotent within max_order")


@dataclass
class BruteForce:
    M: np.ndarray          # [D, D]
    b: np.ndarray          # [n, D]  row p = b_p
    c: np.ndarray          # [n, D]  row q = c_q
    e_cc: float
    e_hf: float
    h_n1: np.ndarray       # bare H in the N-1 sector (for the exact resolvent)
    ann_phi: np.ndarray    # [n, dim(N-1)]  a_p |Phi>
    phi_cre: np.ndarray    # [n, dim(N-1)]  <Phi| a_q^+ as row vectors


def build(o: int, v: int, eps: np.ndarray, g: np.ndarray, t1: np.ndarray, t2: np.ndarray,
          l1: np.ndarray, l2: np.ndarray) -> BruteForce:
    """Build M, b, c by brute force for o occupied and v virtual spin-orbitals (n = o+v <= 14)."""
    n = o + v
    f = np.diag(eps)
    h = f - np.einsum("piqi->pq", g[:, :o, :, :o])
    SN = Sector(n, o)
    S1 = Sector(n, o - 1)

    H_N = SN.one_body(h) + SN.two_body(g)
    H_1 = S1.one_body(h) + S1.two_body(g)
    T_N = SN.cluster(o, t1, t2)
    T_1 = S1.cluster(o, t1, t2)
    L_N = SN.deexcitation(o, l1, l2)
    eT_N, emT_N = expm_nilpotent(T_N), expm_nilpotent(-T_N)
    eT_1, emT_1 = expm_nilpotent(T_1), expm_nilpotent(-T_1)
    Hb_N = emT_N @ H_N @ eT_N
    Hb_1 = emT_1 @ H_1 @ eT_1

    phi = np.zeros(SN.dim)
    phi[SN.index[(1 << o) - 1]] = 1.0
    e_hf = float(phi @ H_N @ phi)
    e_cc = float(phi @ Hb_N @ phi)

    # R_nu as operators N -> N-1, and the basis vectors R_nu |Phi>
    ops = [SN.A[k] for k in range(o)]
    pairs = [(k, l) for l in range(o) for k in range(l)]
    for (k, l) in pairs:
        for c in range(v):
            # a_c^+ a_l a_k : N -> N-1  (a_k first, then a_l, then a_c^+)
            ops.append(S1.A[o + c].T @ (S1.A[l] @ SN.A[k]))
    D = len(ops)
    basis = np.stack([R @ phi for R in ops], axis=1)                      # [dim(N-1), D]
    norms = np.einsum("ij,ij->j", basis, basis)
    assert np.allclose(norms, 1.0), "1h+2h1p basis vectors must be normalised determinants"

    Hb_phi = Hb_N @ phi
    RH = np.stack([R @ Hb_phi for R in ops], axis=1)                      # R_nu Hbar |Phi>
    M = basis.T @ Hb_1 @ basis - basis.T @ RH

    b = np.stack([basis.T @ (emT_1 @ SN.A[p] @ eT_N @ phi) for p in range(n)])
    left = phi @ (np.eye(SN.dim) + L_N) @ emT_N                          # <Phi|(1+Lambda)e^{-T}
    c = np.stack([(left @ SN.A[q].T @ eT_1) @ basis for q in range(n)])
    ann_phi = np.stack([SN.A[p] @ phi for p in range(n)])
    phi_cre = np.stack([phi @ SN.A[q].T for q in range(n)])
    return BruteForce(M=M, b=b, c=c, e_cc=e_cc, e_hf=e_hf, h_n1=H_1, ann_phi=ann_phi,
                      phi_cre=phi_cre)


def build_from_inputs(inp) -> BruteForce:
    """Brute force for a ``synth.Inputs`` object (uses its full n^4 integral tensor)."""
    return build(inp.o, inp.v, inp.eps, inp.full_antisym(), inp.t1, inp.t2, inp.l1, inp.l2)


def exact_resolvent(bf: BruteForce, omegas: np.ndarray, eta: float) -> np.ndarray:
    """G[w, p, q] = <Phi| a_q^+ (w - i eta + H - E_HF)^{-1} a_p |Phi> over the full N-1 sector."""
    dim = bf.h_n1.shape[0]
    out = []
    for w in omegas:
        A = (w - 1j * eta - bf.e_hf) * np.eye(dim) + bf.h_n1
        X = np.linalg.solve(A, bf.ann_phi.T.astype(complex))              # [dim, n]
        out.append((bf.phi_cre @ X).T)                                    # [p, q]
    return np.array(out)


# ---- electron attachment: the (N+1)-electron sector ------------------------------------------
#
# Basis of the 1p + 2p1h space: index c for a_{o+c}^+ |Phi>, then v + pair(a,b)*o + j for
# a_{o+a}^+ a_{o+b}^+ a_j |Phi> with a < b (a_j applied first) and pair(a,b) = b(b-1)/2 + a.
#   M_EA[mu,nu] = <mu| Hbar R_nu |Phi> - <mu| R_nu Hbar |Phi>     (connected action of Hbar_N)
#   b_q = projection of e^{-T} a_q^+ e^{T} |Phi>                   (the attachment free term)
#   c_p[nu] = <Phi| (1 + Lambda) e^{-T} a_p e^{T} R_nu |Phi>       (the attachment left vector)
# so that G^EA_pq(w) = c_p^T (w + i eta - M_EA)^{-1} b_q approximates the second (attachment) term
# <Psi| a_p (w - (H - E_0) + i eta)^{-1} a_q^+ |Psi> of the retarded Green's function (Eq. gfxn0
# written out for both orderings of the field operators).

@dataclass
class BruteForceEA:
    M: np.ndarray          # [D, D]
    b: np.ndarray          # [n, D]  row q = b_q
    c: np.ndarray          # [n, D]  row p = c_p
    e_hf: float
    h_np1: np.ndarray      # bare H in the N+1 sector
    cre_phi: np.ndarray    # [n, dim(N+1)]  a_q^+ |Phi>
    phi_ann: np.ndarray    # [n, dim(N+1)]  <Phi| a_p as row vectors


def build_ea(o: int, v: int, eps: np.ndarray, g: np.ndarray, t1: np.ndarray, t2: np.ndarray,
             l1: np.ndarray, l2: np.ndarray) -> BruteForceEA:
    """Build M_EA, b, c by brute force in the N+1 sector (n = o+v <= 14)."""
    n = o + v
    f = np.diag(eps)
    h = f - np.einsum("piqi->pq", g[:, :o, :, :o])
    SN = Sector(n, o)
    SP = Sector(n, o + 1)

    H_N = SN.one_body(h) + SN.two_body(g)
    H_P = SP.one_body(h) + SP.two_body(g)
    T_N = SN.cluster(o, t1, t2)
    T_P = SP.cluster(o, t1, t2)
    L_N = SN.deexcitation(o, l1, l2)
    eT_N, emT_N = expm_nilpotent(T_N), expm_nilpotent(-T_N)
    eT_P, emT_P = expm_nilpotent(T_P), expm_nilpotent(-T_P)
    Hb_N = emT_N @ H_N @ eT_N
    Hb_P = emT_P @ H_P @ eT_P

    phi = np.zeros(SN.dim)
    phi[SN.index[(1 << o) - 1]] = 1.0
    e_hf = float(phi @ H_N @ phi)

    # R_nu as operators N -> N+1 (creation from N to N+1 is the transpose of SP.A)
    ops = [SP.A[o + c].T for c in range(v)]
    for b_ in range(v):
        for a_ in range(b_):
            for j in range(o):
                # a_a^+ a_b^+ a_j : a_j (N -> N-1), a_b^+ (N-1 -> N), a_a^+ (N -> N+1)
                ops.append(SP.A[o + a_].T @ SN.A[o + b_].T @ SN.A[j])
    basis = np.stack([R @ phi for R in ops], axis=1)                      # [dim(N+1), D]
    norms = np.einsum("ij,ij->j", basis, basis)
    assert np.allclose(norms, 1.0), "1p+2p1h basis vectors must be normalised determinants"

    Hb_phi = Hb_N @ phi
    RH = np.stack([R @ Hb_phi for R in ops], axis=1)
    M = basis.T @ Hb_P @ basis - basis.T @ RH

    b = np.stack([basis.T @ (emT_P @ SP.A[q].T @ eT_N @ phi) for q in range(n)])
    left = phi @ (np.eye(SN.dim) + L_N) @ emT_N
    c = np.stack([(left @ SP.A[p] @ eT_P) @ basis for p in range(n)])
    cre_phi = np.stack([SP.A[q].T @ phi for q in range(n)])
    phi_ann = np.stack([phi @ SP.A[p] for p in range(n)])
    return BruteForceEA(M=M, b=b, c=c, e_hf=e_hf, h_np1=H_P, cre_phi=cre_phi, phi_ann=phi_ann)


def build_ea_from_inputs(inp) -> BruteForceEA:
    return build_ea(inp.o, inp.v, inp.eps, inp.full_antisym(), inp.t1, inp.t2, inp.l1, inp.l2)


def exact_resolvent_ea(bf: BruteForceEA, omegas: np.ndarray, eta: float) -> np.ndarray:
    """G[w, p, q] = <Phi| a_p (w + i eta - (H - E_HF))^{-1} a_q^+ |Phi> over the full N+1 sector."""
    dim = bf.h_np1.shape[0]
    out = []
    for w in omegas:
        A = (w + 1j * eta + bf.e_hf) * np.eye(dim) - bf.h_np1
        Y = np.linalg.solve(A, bf.cre_phi.T.astype(complex))              # [dim, n] columns q
        out.append(bf.phi_ann @ Y)                                         # [p, q]
    return np.array(out)
