"""Seeded synthetic inputs for the IP-GFCC linear systems (shared by the oracle and the GPU tests).

This module holds only input generation: random numbers and the molecule-shaped recipe
that turns them into orbital energies, antisymmetrised integrals and amplitudes. It holds
none of the Green's-function method's arithmetic, and it imports neither ``oracle`` nor the
CUDA package.

Random numbers are counter-based: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) applied to
``base + (k+1)*gamma`` gives the k-th 64-bit draw of a stream, and Box-Muller turns two draws
into one normal deviate. Every value is a pure function of (seed, stream, index), so any block
of the integral tensor can be generated alone, in any order, on any machine.

Recipe (the paper's molecules and their NWChem amplitudes are not available; these inputs
keep their shapes and structure):

* spin-orbital energies: occupied ~ U[-1.5, -0.3] Ha, virtual ~ U[0.1, 2.0] Ha; the Fock
  matrix of the reference is diag(eps) (normal-ordered H_N, Eq. gfxn1 text).
* two-electron integrals: a real chemist-notation tensor (pq|rs) with the 8-fold permutational
  symmetry of real orbitals, drawn as ``scale * N(0,1)`` once per canonical index; then
  <pq|rs> = (pr|qs) and <pq||rs> = <pq|rs> - <pq|sr>.
* ``scale``: 0.05 at the tiny size o=4, v=8.  ``scale_mode="size_consistent"`` (default)
  scales it as 0.05*sqrt(4*8**2/(o*v**2)) so that the MP2-like correlation shift of the Fock
  diagonal (which grows as scale**2 * o * v**2) stays at the tiny system's ~0.2 Ha and the
  ionisation poles stay in the [-1.2, -0.2] Ha windows; ``"literal"`` keeps 0.05 at every size.
* T1 ~ N(0, 0.01) (standard deviation), T2_ij^ab = <ij||ab> / (e_i + e_j - e_a - e_b).
* Lambda1 = T1, Lambda2 = T2 (same index order).
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)

# stream identifiers (arbitrary distinct constants)
STREAM_EPS_OCC = 1
STREAM_EPS_VIR = 2
STREAM_ERI = 3
STREAM_T1 = 4
STREAM_AUX = 5


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on uint64 arrays (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
        return z ^ (z >> np.uint64(31))


def _base(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.array([(seed & 0xFFFFFFFF) * 0x100000000 + (stream & 0xFFFFFFFF)], dtype=np.uint64)
        return _mix(s * _GAMMA + _GAMMA)[0]


def draw_u64(seed: int, stream: int, idx) -> np.ndarray:
    """k-th SplitMix64 output of stream (seed, stream) for every k in ``idx``."""
    k = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(_base(seed, stream) + (k + np.uint64(1)) * _GAMMA)


def uniform(seed: int, stream: int, idx) -> np.ndarray:
    """Uniform deviates in (0, 1): top 53 bits of the draw, offset by half a unit."""
    z = draw_u64(seed, stream, idx)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, idx) -> np.ndarray:
    """Standard normal deviates by Box-Muller from draws 2k and 2k+1."""
    k = np.asarray(idx, dtype=np.uint64)
    u1 = uniform(seed, stream, k * np.uint64(2))
    u2 = uniform(seed, stream, k * np.uint64(2) + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def _canon_pair(p, q):
    hi = np.maximum(p, q).astype(np.int64)
    lo = np.minimum(p, q).astype(np.int64)
    return hi * (hi + 1) // 2 + lo


def chem_eri(seed: int, scale: float, p, q, r, s) -> np.ndarray:
    """(pq|rs) for broadcastable index arrays, 8-fold symmetric by construction."""
    pq = _canon_pair(np.asarray(p), np.asarray(q))
    rs = _canon_pair(np.asarray(r), np.asarray(s))
    key = _canon_pair(pq, rs)
    return scale * normal(seed, STREAM_ERI, key)


def antisym_block(seed: int, scale: float, P, Q, R, S, chunk: int = 1) -> np.ndarray:
    """<pq||rs> for p in P, q in Q, r in R, s in S (index lists); slices of P are generated in
    parallel threads (NumPy releases the GIL), each value depending only on its indices."""
    P, Q, R, S = (np.asarray(x, dtype=np.int64) for x in (P, Q, R, S))
    out = np.empty((len(P), len(Q), len(R), len(S)), dtype=np.float64)
    q = Q[None, :, None, None]
    r = R[None, None, :, None]
    s = S[None, None, None, :]

    def fill(i0):
        p = P[i0:i0 + chunk, None, None, None]
        out[i0:i0 + chunk] = chem_eri(seed, scale, p, r, q, s) - chem_eri(seed, scale, p, s, q, r)

    starts = list(range(0, len(P), chunk))
    if out.size < (1 << 20) or len(starts) == 1:
        for i0 in starts:
            fill(i0)
    else:
        import concurrent.futures as cf
        with cf.ThreadPoolExecutor(max_workers=min(len(starts), os.cpu_count() or 1)) as ex:
            list(ex.map(fill, starts))
    return out


def pair_lists(k: int) -> tuple[np.ndarray, np.ndarray]:
    """(first, second) index of every pair a < b of range(k), in the packed order
    pair(a, b) = b(b-1)/2 + a."""
    b = np.concatenate([np.full(j, j, dtype=np.int64) for j in range(k)]) if k > 1 else np.zeros(0, np.int64)
    a = np.concatenate([np.arange(j, dtype=np.int64) for j in range(k)]) if k > 1 else np.zeros(0, np.int64)
    return a, b


def antisym_pairs(seed: int, scale: float, P, Q, R, S, chunk: int = 64) -> np.ndarray:
    """out[k, l] = <P[k] Q[k] || R[l] S[l]>: rows and columns run over index pairs (packed
    antisymmetric storage); row chunks are generated in parallel threads."""
    P, Q, R, S = (np.asarray(x, dtype=np.int64) for x in (P, Q, R, S))
    out = np.empty((len(P), len(R)), dtype=np.float64)
    r = R[None, :]
    s = S[None, :]

    def fill(i0):
        p = P[i0:i0 + chunk, None]
        q = Q[i0:i0 + chunk, None]
        out[i0:i0 + chunk] = chem_eri(seed, scale, p, r, q, s) - chem_eri(seed, scale, p, s, q, r)

    starts = list(range(0, len(P), chunk))
    if out.size < (1 << 20) or len(starts) == 1:
        for i0 in starts:
            fill(i0)
    else:
        import concurrent.futures as cf
        with cf.ThreadPoolExecutor(max_workers=min(len(starts), os.cpu_count() or 1)) as ex:
            list(ex.map(fill, starts))
    return out


def integral_scale(o: int, v: int, mode: str = "size_consistent") -> float:
    if mode == "literal":
        return 0.05
    if mode == "size_consistent":
        return 0.05 * math.sqrt(4.0 * 8.0 ** 2 / (o * max(v, 1) ** 2))
    raise ValueError(f"unknown scale mode {mode!r}")


@dataclass
class Inputs:
    """Ground-state inputs of the IP-GFCC linear systems (all real float64, row-major).

    Index blocks of the antisymmetrised integrals <pq||rs> (occupied index range first):
    ``oooo[i,j,k,l]``, ``ooov[i,j,k,a]``, ``oovv[i,j,a,b]``, ``ovov[i,a,j,b]``, ``ovvv[i,a,b,c]``.
    ``t1[i,a]``, ``t2[i,j,a,b]``, ``l1[i,a]`` (lambda^i_a), ``l2[i,j,a,b]`` (lambda^ij_ab).
    """

    o: int
    v: int
    eps: np.ndarray
    oooo: np.ndarray
    ooov: np.ndarray
    oovv: np.ndarray
    ovov: np.ndarray
    ovvv: np.ndarray
    t1: np.ndarray
    t2: np.ndarray
    l1: np.ndarray
    l2: np.ndarray
    seed: int = 0
    scale: float = 0.05
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.o + self.v

    @property
    def npair(self) -> int:
        return self.o * (self.o - 1) // 2

    @property
    def dim(self) -> int:
        return self.o + self.npair * self.v

    def full_antisym(self) -> np.ndarray:
        """Full n^4 <pq||rs> (small systems only; used by brute-force checks)."""
        n = self.n
        idx = np.arange(n)
        return antisym_block(self.seed, self.scale, idx, idx, idx, idx)

    def vvvv_pairs(self) -> np.ndarray:
        """The virtual-virtual block in packed pair form: out[pair(a,b)][pair(c,d)] = <ab||cd> for
        a < b, c < d (virtual indices counted from 0, pair(a,b) = b(b-1)/2 + a). Generated on demand,
        from the same integral tensor as the other blocks (the electron-attachment space needs it)."""
        a, b = pair_lists(self.v)
        a = a + self.o
        b = b + self.o
        return antisym_pairs(self.seed, self.scale, a, b, a, b)


def make_inputs(o: int, v: int, seed: int, scale_mode: str = "size_consistent",
                t1_sd: float = 0.01, with_t: bool = True, with_lambda: bool = True,
                scale: float | None = None) -> Inputs:
    """Generate the synthetic inputs for o occupied and v virtual spin-orbitals."""
    if o < 1 or v < 0:
        raise ValueError("need o >= 1 and v >= 0")
    sc = integral_scale(o, v, scale_mode) if scale is None else float(scale)
    eps_o = -1.5 + 1.2 * uniform(seed, STREAM_EPS_OCC, np.arange(o))
    eps_v = 0.1 + 1.9 * uniform(seed, STREAM_EPS_VIR, np.arange(v))
    eps = np.concatenate([eps_o, eps_v])
    O = np.arange(o)
    V = np.arange(o, o + v)
    oooo = antisym_block(seed, sc, O, O, O, O)
    ooov = antisym_block(seed, sc, O, O, O, V)
    oovv = antisym_block(seed, sc, O, O, V, V)
    ovov = antisym_block(seed, sc, O, V, O, V)
    ovvv = antisym_block(seed, sc, O, V, V, V)
    if with_t:
        t1 = t1_sd * normal(seed, STREAM_T1, np.arange(o * v)).reshape(o, v)
        denom = (eps_o[:, None, None, None] + eps_o[None, :, None, None]
                 - eps_v[None, None, :, None] - eps_v[None, None, None, :])
        t2 = oovv / denom
    else:
        t1 = np.zeros((o, v))
        t2 = np.zeros((o, o, v, v))
    if with_lambda:
        l1 = t1.copy()
        l2 = t2.copy()
    else:
        l1 = np.zeros((o, v))
        l2 = np.zeros((o, o, v, v))
    return Inputs(o=o, v=v, eps=eps, oooo=oooo, ooov=ooov, oovv=oovv, ovov=ovov, ovvv=ovvv,
                  t1=t1, t2=t2, l1=l1, l2=l2, seed=seed, scale=sc,
                  meta={"scale_mode": scale_mode, "t1_sd": t1_sd})


def random_amplitudes(inp: Inputs, seed: int, sd1: float = 0.05, sd2: float = 0.05) -> Inputs:
    """Replace T and Lambda by independent random antisymmetric amplitudes (for pinning tests:
    polynomial identities must hold for any amplitudes, not only MP2-like ones)."""
    o, v = inp.o, inp.v

    def anti(x):
        x = x - x.transpose(1, 0, 2, 3)
        return x - x.transpose(0, 1, 3, 2)

    z = normal(seed, STREAM_AUX, np.arange(2 * o * v + 2 * o * o * v * v))
    k = 0
    t1 = sd1 * z[k:k + o * v].reshape(o, v); k += o * v
    l1 = sd1 * z[k:k + o * v].reshape(o, v); k += o * v
    t2 = anti(sd2 * z[k:k + o * o * v * v].reshape(o, o, v, v)); k += o * o * v * v
    l2 = anti(sd2 * z[k:k + o * o * v * v].reshape(o, o, v, v))
    return Inputs(o=o, v=v, eps=inp.eps, oooo=inp.oooo, ooov=inp.ooov, oovv=inp.oovv,
                  ovov=inp.ovov, ovvv=inp.ovvv, t1=t1, t2=t2, l1=l1, l2=l2,
                  seed=inp.seed, scale=inp.scale, meta=dict(inp.meta, random_amplitudes=seed))


def omega_grid(wmin: float, wmax: float, n: int) -> np.ndarray:
    """Uniform frequency grid including both ends."""
    if n == 1:
        return np.array([0.5 * (wmin + wmax)])
    return np.linspace(wmin, wmax, n)


# Named workloads: (o, v, seed, omega window, n_omega, eta). Sizes follow the molecules the
# method was applied to (CO/cc-pVDZ, butadiene, benzene, adenine) and a tiny brute-force case.
# The attachment window [ea_wmin, ea_wmax] covers the lower part of the virtual orbital energies
# (drawn on [0.1, 2.0] Ha) and the lowest 2p1h satellites.
WORKLOADS = {
    "tiny_o4_v8": dict(o=4, v=8, seed=1001, wmin=-1.0, wmax=0.0, nw=200, eta=0.01, ea_wmin=0.1, ea_wmax=1.1),
    "co_o14_v42": dict(o=14, v=42, seed=1002, wmin=-1.2, wmax=-0.3, nw=500, eta=0.01, ea_wmin=0.1, ea_wmax=1.0),
    "butadiene_o30_v130": dict(o=30, v=130, seed=1003, wmin=-1.0, wmax=-0.2, nw=1000, eta=0.005,
                               ea_wmin=0.1, ea_wmax=0.9),
    "benzene_o42_v186": dict(o=42, v=186, seed=1004, wmin=-1.0, wmax=-0.2, nw=5000, eta=0.01,
                             ea_wmin=0.1, ea_wmax=0.9),
    "adenine_o70_v250": dict(o=70, v=250, seed=1005, wmin=-0.8, wmax=-0.2, nw=2000, eta=0.01,
                             ea_wmin=0.1, ea_wmax=0.7),
}

