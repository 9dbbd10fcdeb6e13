"""Electron-attachment (EA, 1p + 2p1h) half of the GFCC Green's function (oracle, FP64).

Test infrastructure: only tests, the smoke check and the CPU baseline use the oracle.

The retarded Green's function that the paper starts from (Eq. gfxn0 and the text around it, which
names the IP and EA halves) has a second, attachment term <Psi| a_p (w - (H - E_0) + i eta)^{-1} a_q^+ |Psi>.
In the bi-orthogonal CC form (Eqs. gfxn1/gfxn2 with the roles of a_p and a_q^+ exchanged) it reads
  G^EA_pq(w) = <Phi|(1 + Lambda) abar_p (w - Hbar_N + i eta)^{-1} abar_q^+ |Phi>,
and with an EA-EOM operator Y_q(w) = sum_a y^a a_a^+ + sum_{a<b,j} y^{ab}_j a_a^+ a_b^+ a_j the linear
systems are (w + i eta - M) y_q(w) = b_q, G^EA_pq(w) = c_p^T y_q(w), M the matrix of Hbar_N on the
1p + 2p1h space. The paper writes out the IP half only; this module is the same construction for the
attachment half, pinned against the brute-force N+1 sector of ``oracle.fockspace``.

Packed layout (batch-last vectors [..., D], D = v + V*o, V = v(v-1)/2): [y^0 .. y^{v-1} |
y^{pair(a,b)}_j at v + pair(a,b)*o + j], pair(a,b) = b(b-1)/2 + a.

Sigma (summation over repeated indices; P(ab) g_ab = g_ab - g_ba; r^{ab}_j antisymmetric in ab):
  s_a     = F_ae r_e + F_me r^{ae}_m + 1/2 W_amef r^{ef}_m
  s^{ab}_j = W_abej r_e - F_mj r^{ab}_m + P(ab) F_ae r^{eb}_j + 1/2 W_abef r^{ef}_j
             + P(ab) W_mbej r^{ae}_m - 1/2 <mn||ef> r^{ef}_n t_mj^ab
with the H-bar elements (tau as in ``oracle.hbar``)
  W_abef = <ab||ef> - P(ab) t_m^b <am||ef> + 1/2 tau_mn^ab <mn||ef>
  W_amef = <am||ef> - t_n^a <nm||ef>
  W_abej = <ab||ej> - F_me t_mj^ab + t_j^f W_abef + 1/2 <mn||ej> tau_mn^ab
           - P(ab) <mb||ef> t_mj^af - P(ab) t_m^a (<mb||ej> - t_nj^bf <mn||ef>)
and F_ae, F_mi, F_me, W_mbej shared with the IP space.

Solved in the form of the IP systems: (w' - i eta + M) y = -b_q with w' = -w is the same system, so the
IP solver and reduced model apply unchanged to (M, -b, c) at negated frequencies (``ip_form``).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import hbar as ipbar

einsum = lambda *a: np.einsum(*a, optimize=True)  # noqa: E731


def pairs(v: int):
    return [(a, b) for b in range(v) for a in range(b)]


def dim(o: int, v: int) -> int:
    return v + v * (v - 1) // 2 * o


def unpack(x: np.ndarray, o: int, v: int):
    """Packed [..., D] -> (r1 [..., v], r2 [..., v, v, o] antisymmetric in the virtual pair)."""
    x = np.asarray(x)
    lead = x.shape[:-1]
    r1 = x[..., :v]
    r2 = np.zeros(lead + (v, v, o), dtype=x.dtype)
    body = x[..., v:].reshape(lead + (v * (v - 1) // 2, o))
    for k, (a, b) in enumerate(pairs(v)):
        r2[..., a, b, :] = body[..., k, :]
        r2[..., b, a, :] = -body[..., k, :]
    return r1, r2


def pack(r1: np.ndarray, r2: np.ndarray) -> np.ndarray:
    v = r1.shape[-1]
    o = r2.shape[-1]
    lead = r1.shape[:-1]
    out = np.empty(lead + (dim(o, v),), dtype=np.result_type(r1, r2))
    out[..., :v] = r1
    for k, (a, b) in enumerate(pairs(v)):
        out[..., v + k * o:v + (k + 1) * o] = r2[..., a, b, :]
    return out


def unpack_vvvv(vp: np.ndarray, v: int) -> np.ndarray:
    """Packed [pair(a,b)][pair(c,d)] = <ab||cd> -> full [a,b,c,d], antisymmetric in ab and in cd."""
    out = np.zeros((v, v, v, v))
    pr = pairs(v)
    for k, (a, b) in enumerate(pr):
        for l, (c, d) in enumerate(pr):
            x = vp[k, l]
            out[a, b, c, d] = x
            out[b, a, c, d] = -x
            out[a, b, d, c] = -x
            out[b, a, d, c] = x
    return out


@dataclass
class EaHbar:
    o: int
    v: int
    Fmi: np.ndarray    # [m,i]
    Fme: np.ndarray    # [m,e]
    Fae: np.ndarray    # [a,e]
    Wabef: np.ndarray  # [a,b,e,f]
    Wamef: np.ndarray  # [a,m,e,f]
    Wabej: np.ndarray  # [a,b,e,j]
    Wmbej: np.ndarray  # [m,b,e,j]
    Vmnef: np.ndarray  # [m,n,e,f]
    t2: np.ndarray     # [i,j,a,b]
    sector: str = "ea"


def build(inp, vvvv: np.ndarray | None = None) -> EaHbar:
    """EA H-bar elements; ``vvvv`` = full [v,v,v,v] <ab||cd> (default: from ``inp.vvvv_pairs()``)."""
    o, v = inp.o, inp.v
    ip = ipbar.build(inp)
    t1, t2 = inp.t1, inp.t2
    if vvvv is None:
        vvvv = unpack_vvvv(inp.vvvv_pairs(), v)
    v_oovv = inp.oovv
    v_vovv = -inp.ovvv.transpose(1, 0, 2, 3)          # <am||ef> = -<ma||ef>
    v_ovvo = -inp.ovov.transpose(0, 1, 3, 2)          # <mb||ej> = -<mb||je>
    v_oovo = -inp.ooov.transpose(0, 1, 3, 2)          # <mn||ej> = -<mn||je>
    v_vvvo = -inp.ovvv.transpose(2, 3, 1, 0)          # <ab||ej> = <ej||ab> = -<je||ab>
    tau = t2 + einsum("ia,jb->ijab", t1, t1) - einsum("ib,ja->ijab", t1, t1)

    tmp = einsum("mb,amef->abef", t1, v_vovv)
    Wabef = vvvv - tmp + tmp.transpose(1, 0, 2, 3) + 0.5 * einsum("mnab,mnef->abef", tau, v_oovv)
    Wamef = v_vovv - einsum("na,nmef->amef", t1, v_oovv)

    Wabej = (v_vvvo - einsum("me,mjab->abej", ip.Fme, t2)
             + einsum("jf,abef->abej", t1, Wabef)
             + 0.5 * einsum("mnej,mnab->abej", v_oovo, tau))
    tmp = einsum("mbef,mjaf->abej", inp.ovvv, t2)     # <mb||ef> t_mj^af
    Wabej = Wabej - tmp + tmp.transpose(1, 0, 2, 3)
    X = v_ovvo - einsum("njbf,mnef->mbej", t2, v_oovv)
    tmp = einsum("ma,mbej->abej", t1, X)
    Wabej = Wabej - tmp + tmp.transpose(1, 0, 2, 3)
    return EaHbar(o=o, v=v, Fmi=ip.Fmi, Fme=ip.Fme, Fae=ip.Fae, Wabef=Wabef, Wamef=Wamef, Wabej=Wabej,
                  Wmbej=ip.Wmbej, Vmnef=v_oovv, t2=t2)


def sigma(hb: EaHbar, x: np.ndarray) -> np.ndarray:
    """M x for x of shape [D] or [nvec, D] (real or complex)."""
    o, v = hb.o, hb.v
    single = np.asarray(x).ndim == 1
    X = np.atleast_2d(x)
    r1, r2 = unpack(X, o, v)
    s1 = (einsum("ae,ze->za", hb.Fae, r1)
          + einsum("me,zaem->za", hb.Fme, r2)
          + 0.5 * einsum("amef,zefm->za", hb.Wamef, r2))
    s2 = (einsum("abej,ze->zabj", hb.Wabej, r1)
          - einsum("mj,zabm->zabj", hb.Fmi, r2)
          + 0.5 * einsum("abef,zefj->zabj", hb.Wabef, r2))
    tmp = einsum("ae,zebj->zabj", hb.Fae, r2) + einsum("mbej,zaem->zabj", hb.Wmbej, r2)
    s2 = s2 + tmp - tmp.transpose(0, 2, 1, 3)
    xm = einsum("mnef,zefn->zm", hb.Vmnef, r2)
    s2 = s2 - 0.5 * einsum("zm,mjab->zabj", xm, hb.t2)
    out = pack(s1, s2)
    return out[0] if single else out


def dense_matrix(hb: EaHbar) -> np.ndarray:
    D = dim(hb.o, hb.v)
    return sigma(hb, np.eye(D)).T


def diagonal(hb: EaHbar) -> np.ndarray:
    """Fock part of diag(M): F_aa on 1p, F_aa + F_bb - F_jj on 2p1h (a Jacobi preconditioner only)."""
    o, v = hb.o, hb.v
    fo = np.diag(hb.Fmi)
    fv = np.diag(hb.Fae)
    d2 = np.array([fv[a] + fv[b] - fo for (a, b) in pairs(v)]).reshape(-1)
    return np.concatenate([fv.copy(), d2])


def b_vectors(inp, orbitals=None) -> np.ndarray:
    """Rows b_q (projection of e^{-T} a_q^+ e^{T}|Phi>): b_a = unit 1p vector; b_i[e] = -t_i^e,
    b_i[ef, n] = -t_in^ef."""
    o, v = inp.o, inp.v
    n = o + v
    orbitals = list(range(n)) if orbitals is None else list(orbitals)
    out = []
    for q in orbitals:
        r1 = np.zeros(v)
        r2 = np.zeros((v, v, o))
        if q >= o:
            r1[q - o] = 1.0
        else:
            r1[:] = -inp.t1[q]
            r2[:] = -inp.t2[q].transpose(1, 2, 0)
        out.append(pack(r1, r2))
    return np.array(out)


def c_vectors(inp, orbitals=None) -> np.ndarray:
    """Rows c_p[nu] = <Phi|(1+Lambda) e^{-T} a_p e^{T} R_nu|Phi>:
      c_i[c] = -l_c^i,  c_i[ef, n] = -l_ef^in
      c_a[c] = delta_ac - t_k^a l_c^k - 1/2 t_kl^ad l_cd^kl,
      c_a[ef, n] = delta_ae l_f^n - delta_af l_e^n - t_k^a l_ef^kn."""
    o, v = inp.o, inp.v
    n = o + v
    t1, t2, l1, l2 = inp.t1, inp.t2, inp.l1, inp.l2
    orbitals = list(range(n)) if orbitals is None else list(orbitals)
    out = []
    for p in orbitals:
        r1 = np.zeros(v)
        r2 = np.zeros((v, v, o))
        if p < o:
            i = p
            r1[:] = -l1[i]
            r2[:] = -l2[i].transpose(1, 2, 0)
        else:
            a = p - o
            r1[a] += 1.0
            r1 -= einsum("k,kc->c", t1[:, a], l1)
            r1 -= 0.5 * einsum("kld,klcd->c", t2[:, :, a, :], l2)
            r2[a, :, :] += l1.T
            r2[:, a, :] -= l1.T
            r2 -= einsum("k,knef->efn", t1[:, a], l2)
        out.append(pack(r1, r2))
    return np.array(out)


def dense_solve(M: np.ndarray, B: np.ndarray, omegas, eta: float) -> np.ndarray:
    """Y[w, q, :] = (w + i eta - M)^{-1} b_q by dense LU."""
    D = M.shape[0]
    I = np.eye(D)
    out = np.empty((len(omegas), B.shape[0], D), dtype=complex)
    for k, w in enumerate(omegas):
        out[k] = np.linalg.solve((w + 1j * eta) * I - M, B.T.astype(complex)).T
    return out


def green(C: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """G^EA[w, p, q] = c_p^T Y[w, q]."""
    return np.einsum("pd,wqd->wpq", C, Y)


def ip_form(inp, hb: EaHbar, orbitals=None, read_orbitals=None):
    """(B', C) of the same systems in the IP form (w' - i eta + M) y = b' at w' = -w: B' = -B."""
    return -b_vectors(inp, orbitals), c_vectors(inp, read_orbitals)
