"""IP-GFCCSD sigma vector: the action of Hbar_N on a 1h + 2h1p vector (oracle, FP64).

Test infrastructure: only tests, the smoke check and the CPU baseline use the oracle.

A vector X_p(w) of Eq. xp holds x^i (1h, o entries) and x^{ij}_a for i<j (2h1p, P*v entries,
P = o(o-1)/2). Packed layout: [x^0 .. x^{o-1} | x^{pair(i,j)}_a at o + pair(i,j)*v + a], with
pair(i,j) = j(j-1)/2 + i. Internally the 2h1p part is unpacked into a full array r[i,j,a] that is
antisymmetric in (i,j).

sigma = M r, where M is the matrix of Hbar_N on this space (Eq. xplin):

  s_i     = - F_mi r_m + F_me r_im^e - 1/2 W_mnie r_mn^e
  s_ij^a  = - W_maij r_m + F_ae r_ij^e - P(ij) F_mi r_mj^a + 1/2 W_mnij r_mn^a
            + P(ij) W_maei r_mj^e + 1/2 <mn||ef> r_mn^f t_ij^ae

(summation over repeated indices; P(ij) g_ij = g_ij - g_ji). The transpose (left) action M^T is
also given, for the adjoint systems. Signs and factors are pinned against the brute-force
Fock-space matrix of ``oracle.fockspace``.
"""
from __future__ import annotations

import numpy as np

einsum = lambda *a: np.einsum(*a, optimize=True)  # noqa: E731


def pairs(o: int):
    return [(i, j) for j in range(o) for i in range(j)]


def dim(o: int, v: int) -> int:
    return o + o * (o - 1) // 2 * v


def unpack(x: np.ndarray, o: int, v: int):
    """Packed [..., D] -> (r1 [..., o], r2 [..., o, o, v] antisymmetric in the occupied pair)."""
    x = np.asarray(x)
    lead = x.shape[:-1]
    r1 = x[..., :o]
    r2 = np.zeros(lead + (o, o, v), dtype=x.dtype)
    body = x[..., o:].reshape(lead + (o * (o - 1) // 2, v))
    for k, (i, j) in enumerate(pairs(o)):
        r2[..., i, j, :] = body[..., k, :]
        r2[..., j, i, :] = -body[..., k, :]
    return r1, r2


def pack(r1: np.ndarray, r2: np.ndarray) -> np.ndarray:
    """(r1, r2) -> packed, keeping the i<j entries of r2."""
    o = r1.shape[-1]
    v = r2.shape[-1]
    lead = r1.shape[:-1]
    out = np.empty(lead + (dim(o, v),), dtype=np.result_type(r1, r2))
    out[..., :o] = r1
    for k, (i, j) in enumerate(pairs(o)):
        out[..., o + k * v:o + (k + 1) * v] = r2[..., i, j, :]
    return out


def sigma(hb, x: np.ndarray) -> np.ndarray:
    """M x for x of shape [D] or [nvec, D] (real or complex). An electron-attachment H-bar
    (``oracle.ea.EaHbar``) gives the 1p + 2p1h sigma instead, so that the solvers and the reduced
    model of the oracle run on either space."""
    if getattr(hb, "sector", "ip") == "ea":
        from . import ea
        return ea.sigma(hb, x)
    o, v = hb.o, hb.v
    single = np.asarray(x).ndim == 1
    X = np.atleast_2d(x)
    r1, r2 = unpack(X, o, v)
    s1 = (-einsum("mi,zm->zi", hb.Fmi, r1)
          + einsum("me,zime->zi", hb.Fme, r2)
          - 0.5 * einsum("mnie,zmne->zi", hb.Wmnie, r2))
    s2 = (-einsum("maij,zm->zija", hb.Wmbij, r1)
          + einsum("ae,zije->zija", hb.Fae, r2)
          + 0.5 * einsum("mnij,zmna->zija", hb.Wmnij, r2))
    tmp = -einsum("mi,zmja->zija", hb.Fmi, r2) + einsum("maei,zmje->zija", hb.Wmbej, r2)
    s2 = s2 + tmp - tmp.transpose(0, 2, 1, 3)
    xe = einsum("mnef,zmnf->ze", hb.Vmnef, r2)
    s2 = s2 + 0.5 * einsum("ze,ijae->zija", xe, hb.t2)
    out = pack(s1, s2)
    return out[0] if single else out


def sigma_transpose(hb, y: np.ndarray) -> np.ndarray:
    """M^T y, computed column by column from the explicit matrix (small systems only)."""
    M = dense_matrix(hb)
    Y = np.atleast_2d(y)
    out = Y @ M
    return out[0] if np.asarray(y).ndim == 1 else out


def dense_matrix(hb) -> np.ndarray:
    """M as a dense [D, D] array, by applying sigma to the unit vectors."""
    if getattr(hb, "sector", "ip") == "ea":
        from . import ea
        return ea.dense_matrix(hb)
    D = dim(hb.o, hb.v)
    return sigma(hb, np.eye(D)).T


def diagonal(hb) -> np.ndarray:
    """diag(M) from the one-body elements: -F_ii on 1h, F_aa - F_ii - F_jj on 2h1p.

    Used only as a (Jacobi) preconditioner; it does not change any solution."""
    if getattr(hb, "sector", "ip") == "ea":
        from . import ea
        return ea.diagonal(hb)
    o, v = hb.o, hb.v
    d1 = -np.diag(hb.Fmi).copy()
    fo = np.diag(hb.Fmi)
    fv = np.diag(hb.Fae)
    d2 = np.array([fv - fo[i] - fo[j] for (i, j) in pairs(o)]).reshape(-1)
    return np.concatenate([d1, d2])
