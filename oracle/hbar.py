"""Similarity-transformed Hamiltonian elements needed by the IP (1h + 2h1p) sigma (oracle, FP64).

Test infrastructure: only tests, the smoke check and the CPU baseline use the oracle.

The paper defines Hbar_N = e^{-T} H e^{T} - E_0 (text after Eq. gfxn1) and solves
(w + Hbar_N - i eta) X_p = abar_p |Phi> over the 1h + 2h1p space (Eqs. xp, xplin). Acting on that
space, Hbar enters through its one- and two-body elements below (spin-orbital form, f = diag(eps),
tau_ij^ab = t_ij^ab + t_i^a t_j^b - t_i^b t_j^a). Every term, sign and factor is pinned against the
brute-force e^{-T} H e^{T} of ``oracle.fockspace`` at random amplitudes.

Index names: m,n,i,j occupied; a,b,e,f virtual. Integral blocks come in as
oooo[m,n,i,j] = <mn||ij>, ooov[m,n,i,e] = <mn||ie>, oovv[m,n,e,f] = <mn||ef>,
ovov[m,a,n,e] = <ma||ne>, ovvv[m,a,e,f] = <ma||ef>; the other orderings follow from the
antisymmetry <pq||rs> = -<qp||rs> = -<pq||sr> and, for real orbitals, <pq||rs> = <rs||pq>.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

einsum = lambda *a: np.einsum(*a, optimize=True)  # noqa: E731


@dataclass
class Hbar:
    o: int
    v: int
    Fmi: np.ndarray    # [m,i]
    Fme: np.ndarray    # [m,e]
    Fae: np.ndarray    # [a,e]
    Wmnij: np.ndarray  # [m,n,i,j]
    Wmnie: np.ndarray  # [m,n,i,e]
    Wmbij: np.ndarray  # [m,b,i,j]
    Wmbej: np.ndarray  # [m,b,e,j]
    Vmnef: np.ndarray  # [m,n,e,f]  bare <mn||ef> (three-body term)
    t2: np.ndarray     # [i,j,a,b]


def build(inp) -> Hbar:
    o, v = inp.o, inp.v
    eo, ev = inp.eps[:o], inp.eps[o:]
    t1, t2 = inp.t1, inp.t2
    v_oooo, v_ooov, v_oovv = inp.oooo, inp.ooov, inp.oovv
    v_ovvv = inp.ovvv
    v_ovvo = -inp.ovov.transpose(0, 1, 3, 2)          # <mb||ej> = -<mb||je>
    v_ovoo = inp.ooov.transpose(2, 3, 0, 1)           # <mb||ij> = <ij||mb>
    v_vovv = -v_ovvv.transpose(1, 0, 2, 3)            # <am||ef> = -<ma||ef>
    v_oovo = -v_ooov.transpose(0, 1, 3, 2)            # <mn||ej> = -<mn||je>
    tau = t2 + einsum("ia,jb->ijab", t1, t1) - einsum("ib,ja->ijab", t1, t1)

    # one-body elements
    Fme = einsum("nf,mnef->me", t1, v_oovv)
    Fmi = (np.diag(eo) + einsum("ne,mnie->mi", t1, v_ooov)
           + 0.5 * einsum("inef,mnef->mi", tau, v_oovv))
    Fae = (np.diag(ev) + einsum("mf,amef->ae", t1, v_vovv)
           - 0.5 * einsum("mnaf,mnef->ae", tau, v_oovv))

    # two-body elements
    tmp = einsum("je,mnie->mnij", t1, v_ooov)
    Wmnij = v_oooo + tmp - tmp.transpose(0, 1, 3, 2) + 0.5 * einsum("ijef,mnef->mnij", tau, v_oovv)
    Wmnie = v_ooov + einsum("if,mnfe->mnie", t1, v_oovv)
    Wmbej = (v_ovvo + einsum("jf,mbef->mbej", t1, v_ovvv)
             - einsum("nb,mnej->mbej", t1, v_oovo)
             - einsum("jnfb,mnef->mbej", t2, v_oovv)
             - einsum("jf,nb,mnef->mbej", t1, t1, v_oovv))
    # Wmbij
    Wmbij = (v_ovoo - einsum("me,ijbe->mbij", Fme, t2)
             - einsum("nb,mnij->mbij", t1, Wmnij)
             + 0.5 * einsum("mbef,ijef->mbij", v_ovvv, tau))
    tmp = einsum("mnje,inbe->mbij", v_ooov, t2)
    Wmbij = Wmbij - tmp + tmp.transpose(0, 1, 3, 2)
    tmp = einsum("ie,mbej->mbij", t1, v_ovvo - einsum("njbf,mnef->mbej", t2, v_oovv))
    Wmbij = Wmbij + tmp - tmp.transpose(0, 1, 3, 2)
    return Hbar(o=o, v=v, Fmi=Fmi, Fme=Fme, Fae=Fae, Wmnij=Wmnij, Wmnie=Wmnie, Wmbij=Wmbij,
                Wmbej=Wmbej, Vmnef=v_oovv, t2=t2)
