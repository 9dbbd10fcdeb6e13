"""Free terms b_p and left vectors c_q of the IP-GFCC system (oracle, FP64).

Test infrastructure: only tests, the smoke check and the CPU baseline use the oracle.

Eq. xplin has right side abar_p|Phi> with abar_p = e^{-T} a_p e^{T}; Eqs. gfxn1/gfxn2 read the
Green's function out with the row <Phi|(1+Lambda) abar_q^+ (abar_q^+ = e^{-T} a_q^+ e^{T}), so that
G_pq(w) = c_q^T X_p(w) (the MIMO form of Eq. gfcclineqn: b columns, c rows, plain transpose).

Expanding the similarity transforms (the commutator series terminates):
  abar_i = a_i                       (occupied annihilators commute with T)
  abar_a = a_a + t_k^a a_k + sum_{k<l,c} t_kl^{ac} a_c^+ a_l a_k
  abar_i^+ = a_i^+ - t_i^e a_e^+ - 1/2 t_in^ef a_e^+ a_f^+ a_n,   abar_a^+ = a_a^+
which gives, on the basis a_k|Phi>, a_c^+ a_l a_k|Phi> (k<l):
  b_i[k] = delta_ik,                       b_i[klc] = 0
  b_a[k] = t_k^a,                          b_a[klc] = t_kl^ac
  c_a[k] = l_a^k,                          c_a[klc] = l_ac^kl
  c_i[k] = delta_ik - t_i^e l_e^k - 1/2 t_in^ef l_ef^kn
  c_i[klc] = delta_ik l_c^l - delta_il l_c^k - t_i^e l_ec^kl
Each entry is pinned against the brute-force Fock-space vectors of ``oracle.fockspace``.
"""
from __future__ import annotations

import numpy as np

from .sigma import pack

einsum = lambda *a: np.einsum(*a, optimize=True)  # noqa: E731


def b_vectors(inp, orbitals=None) -> np.ndarray:
    """Rows b_p for p in ``orbitals`` (default all n spin-orbitals): [np, D]."""
    o, v = inp.o, inp.v
    n = o + v
    orbitals = list(range(n)) if orbitals is None else list(orbitals)
    out = []
    for p in orbitals:
        r1 = np.zeros(o)
        r2 = np.zeros((o, o, v))
        if p < o:
            r1[p] = 1.0
        else:
            a = p - o
            r1[:] = inp.t1[:, a]
            r2[:] = inp.t2[:, :, a, :]
        out.append(pack(r1, r2))
    return np.array(out)


def c_vectors(inp, orbitals=None) -> np.ndarray:
    """Rows c_q for q in ``orbitals`` (default all n spin-orbitals): [nq, D]."""
    o, v = inp.o, inp.v
    n = o + v
    orbitals = list(range(n)) if orbitals is None else list(orbitals)
    t1, t2, l1, l2 = inp.t1, inp.t2, inp.l1, inp.l2
    out = []
    for q in orbitals:
        if q >= o:
            a = q - o
            r1 = l1[:, a].copy()
            r2 = l2[:, :, a, :].copy()
        else:
            i = q
            r1 = np.zeros(o)
            r1[i] = 1.0
            r1 -= einsum("e,ke->k", t1[i], l1)
            r1 -= 0.5 * einsum("nef,knef->k", t2[i], l2)
            r2 = np.zeros((o, o, v))
            r2[i, :, :] += l1
            r2[:, i, :] -= l1
            r2 -= einsum("e,klec->klc", t1[i], l2)
        out.append(pack(r1, r2))
    return np.array(out)
