"""Thin ctypes binding of libgfcc (include/gfcc.h). Argument marshalling only.

Arrays may be NumPy arrays (host memory) or CUDA torch tensors (device memory); outputs are
allocated here as NumPy arrays unless the caller passes its own buffers. Every computation runs in
the CUDA library: if ``libgfcc.so`` is missing or cannot be loaded, importing this module's
``load()`` raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgfcc.so")

PREC_FP64, PREC_TF32, PREC_BF16, PREC_FP64_TC = 0, 1, 2, 3
PRECISIONS = {"fp64": PREC_FP64, "tf32": PREC_TF32, "bf16": PREC_BF16, "fp64_tc": PREC_FP64_TC}

ERRORS = {-1: "GFCC_ERR_ARG", -2: "GFCC_ERR_NOT_CONVERGED", -3: "GFCC_ERR_RANK", -4: "GFCC_ERR_NONFINITE",
          -5: "GFCC_ERR_OOM", -6: "GFCC_ERR_CUDA", -7: "GFCC_ERR_STATE"}

# exported symbols and their prototypes (kept in one place: the CPU tests check the library
# exports exactly these)
_dp, _ip, _vp = C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_void_p


class VBlocks(C.Structure):
    _fields_ = [("oooo", _vp), ("ooov", _vp), ("oovv", _vp), ("ovov", _vp), ("ovvv", _vp)]


class Opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("restart", C.c_int), ("max_restarts", C.c_int),
                ("precision", C.c_int), ("max_batch", C.c_int), ("drop_tol", C.c_double),
                ("verbose", C.c_int), ("residual_precision", C.c_int), ("deriv_indicator", C.c_int),
                ("mor_guess", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("sigma_calls", C.c_longlong), ("sigma_cols", C.c_longlong),
                ("gmres_iters", C.c_longlong), ("restarts", C.c_longlong),
                ("max_rel_res", C.c_double), ("not_converged", C.c_int)]


PROTOTYPES = {
    "gfcc_default_opts": (C.c_int, [C.POINTER(Opts)]),
    "gfcc_init": (C.c_int, [C.POINTER(_vp), C.c_int, C.c_int, _vp, C.POINTER(VBlocks), _vp, _vp, _vp, _vp,
                            C.POINTER(Opts), _vp]),
    "gfcc_init_ea": (C.c_int, [C.POINTER(_vp), C.c_int, C.c_int, _vp, C.POINTER(VBlocks), _vp, _vp, _vp, _vp,
                               _vp, C.POINTER(Opts), _vp]),
    "gfcc_sector": (C.c_int, [_vp, _ip]),
    "gfcc_dim": (C.c_int, [_vp, _ip]),
    "gfcc_set_opts": (C.c_int, [_vp, C.POINTER(Opts)]),
    "gfcc_sigma": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, C.c_int, C.c_int]),
    "gfcc_vectors": (C.c_int, [_vp, _vp, C.c_int, C.c_int, _vp, C.c_int]),
    "gfcc_solve_full": (C.c_int, [_vp, _vp, C.c_int, C.c_double, _vp, C.c_int, _vp, C.c_int, _vp, _vp, _vp,
                                  C.c_int, C.POINTER(Stats)]),
    "gfcc_green_derivatives": (C.c_int, [_vp, _vp, C.c_int, C.c_double, _vp, C.c_int, _vp, C.c_int, _vp, _vp, _vp]),
    "gfcc_green_grad_t2": (C.c_int, [_vp, _vp, C.c_int, C.c_double, _vp, C.c_int, _vp, C.c_int, _vp, _vp, _vp]),
    "gfcc_mor_build": (C.c_int, [_vp, _vp, C.c_int, C.c_double, _vp, C.c_int, _vp, C.c_int]),
    "gfcc_mor_build_siso": (C.c_int, [_vp, _vp, C.c_int, C.c_double, _vp, C.c_int]),
    "gfcc_mor_build_krylov": (C.c_int, [_vp, C.c_int, C.c_double, _vp, C.c_int, _vp, C.c_int]),
    "gfcc_mor_model_info": (C.c_int, [_vp, C.c_int, _ip, _dp, C.c_int, _ip, _ip]),
    "gfcc_mor_refine": (C.c_int, [_vp, C.c_double, C.c_double, C.c_int, C.c_double, C.c_int, _ip, _dp]),
    "gfcc_mor_eval": (C.c_int, [_vp, _vp, C.c_int, _vp, _vp, _vp]),
    "gfcc_mor_info": (C.c_int, [_vp, _dp, C.c_int, _ip, _ip, _ip, _ip]),
    "gfcc_mor_stats": (C.c_int, [_vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "gfcc_mor_save": (C.c_int, [_vp, C.c_char_p]),
    "gfcc_mor_load": (C.c_int, [_vp, C.c_char_p]),
    "gfcc_spectral": (C.c_int, [_vp, C.c_int, _vp, C.c_int, _vp, C.c_int, _vp, C.c_int, _vp]),
    "gfcc_tc_gemm": (C.c_int, [C.c_int, _vp, _vp, C.c_int, C.c_int, C.c_int, _vp]),
    "gfcc_tc_gemm_noalloc": (C.c_int, [C.c_int, _vp, _vp, C.c_int, C.c_int, C.c_int, _vp, _vp]),
    "gfcc_autotune_info": (C.c_int, [C.c_int, _ip, _ip, _ip, _ip, _ip, _ip, _dp, _dp]),
    "gfcc_release_cached_memory": (C.c_int, []),
    "gfcc_launch_count": (C.c_longlong, []),
    "gfcc_profile": (C.c_int, [C.c_int]),
    "gfcc_profile_read": (C.c_int, [C.c_int, C.POINTER(C.c_longlong), _dp, _dp]),
    "gfcc_last_error": (C.c_char_p, [_vp]),
    "gfcc_free": (None, [_vp]),
}

_LIB = None


def load(path: str | None = None):
    """Load libgfcc.so (raises OSError/RuntimeError if it is missing: there is no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libgfcc.so not found at {p}: build it with paper_1902_06016_gb300.build.build()")
    lib = C.CDLL(p)
    for name, (res, args) in PROTOTYPES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def tc_gemm(A, B, precision="bf16"):
    """C = A B^T on the tensor cores (diagnostic): A [M, K], B [N, K] float64 host arrays."""
    lib = load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    M, K = A.shape
    N = B.shape[0]
    C = np.empty((M, N), dtype=np.float32)
    rc = lib.gfcc_tc_gemm(PRECISIONS[precision], _ptr(A), _ptr(B), M, N, K, _ptr(C))
    if rc != 0:
        raise GfccError(rc, "gfcc_tc_gemm failed")
    return C


def tc_gemm_noalloc(A, B, C, precision="bf16", stream=None):
    """C = A B^T on the tensor cores without any device allocation: A [M, K], B [N, K] float64 and
    C [M, N] float32 must be contiguous CUDA tensors (the library reads A and B as row-major with K
    contiguous and writes M x N floats into C). Raises ValueError/TypeError on anything else; returns
    the library's status code."""
    lib = load()
    for name, t in (("A", A), ("B", B), ("C", C)):
        if not hasattr(t, "is_cuda") or not t.is_cuda:
            raise TypeError(f"tc_gemm_noalloc: {name} must be a CUDA tensor")
        if not t.is_contiguous() or t.dim() != 2:
            raise ValueError(f"tc_gemm_noalloc: {name} must be a contiguous 2-D tensor")
    if str(A.dtype) != "torch.float64" or str(B.dtype) != "torch.float64" or str(C.dtype) != "torch.float32":
        raise TypeError("tc_gemm_noalloc: A and B must be float64, C float32")
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K or tuple(C.shape) != (M, N):
        raise ValueError(f"tc_gemm_noalloc: shapes A {tuple(A.shape)}, B {tuple(B.shape)}, C {tuple(C.shape)} "
                         "do not match C[M, N] = A[M, K] B[N, K]^T")
    return int(lib.gfcc_tc_gemm_noalloc(PRECISIONS[precision], _ptr(A), _ptr(B), M, N, K, _ptr(C), stream))


def spectral(G, orbitals, qorb=None, A=None, stream=None):
    """A(w) = -(1/pi) sum_p Im G_pp(w) from G [nw, np, nq] complex128 (NumPy or contiguous CUDA tensor)."""
    orb = _ints(orbitals)
    q = _ints(qorb) if qorb is not None else None
    nw = G.shape[0]
    if A is None:
        if isinstance(G, np.ndarray):
            A = np.empty(nw)
        else:
            import torch
            A = torch.empty((nw,), dtype=torch.float64, device=G.device)
    rc = load().gfcc_spectral(_ptr(G), nw, _ptr(orb), len(orb), _ptr(q), len(q) if q is not None else 0, _ptr(A), 0,
                              stream)
    if rc != 0:
        raise GfccError(rc, "gfcc_spectral failed")
    return A


def spectral_adjoint(Abar, orbitals, nq, qorb=None, Gbar=None, stream=None):
    """Gbar [nw, np, nq] complex128 = the adjoint of the spectral function applied to Abar [nw]."""
    orb = _ints(orbitals)
    q = _ints(qorb) if qorb is not None else None
    nw = Abar.shape[0]
    if Gbar is None:
        shape = (nw, len(orb), nq)
        if isinstance(Abar, np.ndarray):
            Gbar = np.empty(shape, dtype=np.complex128)
        else:
            import torch
            Gbar = torch.empty(shape, dtype=torch.complex128, device=Abar.device)
    rc = load().gfcc_spectral(_ptr(Gbar), nw, _ptr(orb), len(orb), _ptr(q), len(q) if q is not None else 0,
                              _ptr(Abar), 1, stream)
    if rc != 0:
        raise GfccError(rc, "gfcc_spectral (adjoint) failed")
    return Gbar


def autotune_report():
    """The autotuner's decisions so far: one dict per tuned GEMM shape bucket."""
    lib = load()
    out = []
    i = 0
    while True:
        vals = [C.c_int() for _ in range(6)]
        mb, md = C.c_double(), C.c_double()
        if lib.gfcc_autotune_info(i, *[C.byref(x) for x in vals], C.byref(mb), C.byref(md)) != 0:
            return out
        kind, exact, tm, tn, gm, gmd = (x.value for x in vals)
        out.append({"precision": {PREC_BF16: "bf16", PREC_TF32: "tf32"}[kind], "exact_slices": bool(exact),
                    "tiles_m": tm, "tiles_n_log2": tn, "gm": gm, "gm_default": gmd, "ms_best": mb.value,
                    "ms_default": md.value})
        i += 1


def launch_count():
    return int(load().gfcc_launch_count())


def release_cached_memory():
    """Return the unused reserve of the library's device memory pools to the devices."""
    rc = load().gfcc_release_cached_memory()
    if rc != 0:
        raise GfccError(rc, "gfcc_release_cached_memory failed")


def profile(enable=True):
    load().gfcc_profile(1 if enable else 0)


def profile_read(cls):
    """(launches, ms, flops) of kernel class or phase cls (numbering as in gfcc_profile's comment)."""
    n, ms, fl = C.c_longlong(), C.c_double(), C.c_double()
    rc = load().gfcc_profile_read(int(cls), C.byref(n), C.byref(ms), C.byref(fl))
    if rc != 0:
        raise GfccError(rc, "gfcc_profile_read failed")
    return n.value, ms.value, fl.value


class GfccError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def _ptr(a):
    """Data pointer of a NumPy array or a torch tensor (host or CUDA)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)}")


def _c64(a):
    """float64 contiguous host array, or a contiguous float64 torch tensor passed through as is."""
    if hasattr(a, "data_ptr") and not isinstance(a, np.ndarray):
        if not a.is_contiguous() or str(a.dtype) != "torch.float64":
            raise TypeError("tensor inputs must be contiguous float64")
        return a
    return np.ascontiguousarray(a, dtype=np.float64)


def _ints(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


@dataclass
class SolveStats:
    sigma_calls: int
    sigma_cols: int
    gmres_iters: int
    restarts: int
    max_rel_res: float
    not_converged: int


class Context:
    """One GFCC problem on the current CUDA device (wraps gfcc_t).

    sector="ip" (default): the ionisation half over the 1h + 2h1p space (gfcc_init).
    sector="ea": the electron-attachment half over the 1p + 2p1h space (gfcc_init_ea); ``vvvv`` is the
    packed [V][V] virtual block (default: ``inputs.vvvv_pairs()``). Frequencies are the physical w; the
    G arrays are indexed [w][free-term orbital q][left-vector orbital p] (G^EA_pq)."""

    def __init__(self, inputs, tol=1e-8, restart=30, max_restarts=200, precision="fp64", max_batch=0,
                 drop_tol=1e-10, stream=None, residual_precision=None, deriv_indicator=False, mor_guess=True,
                 verbose=False, sector="ip", vvvv=None):
        lib = load()
        self._lib = lib
        o, v = inputs.o, inputs.v
        self.o, self.v = o, v
        if sector not in ("ip", "ea"):
            raise ValueError("sector must be 'ip' or 'ea'")
        self.sector = sector
        opts = Opts()
        lib.gfcc_default_opts(C.byref(opts))
        opts.tol, opts.restart, opts.max_restarts = tol, restart, max_restarts
        opts.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        opts.max_batch, opts.drop_tol = max_batch, drop_tol
        opts.residual_precision = -1 if residual_precision is None else PRECISIONS[residual_precision]
        opts.deriv_indicator = int(bool(deriv_indicator))
        opts.mor_guess = int(bool(mor_guess))
        opts.verbose = int(bool(verbose))
        self._keep = [_c64(x) for x in (inputs.eps, inputs.oooo, inputs.ooov, inputs.oovv, inputs.ovov,
                                         inputs.ovvv, inputs.t1, inputs.t2, inputs.l1, inputs.l2)]
        eps, oooo, ooov, oovv, ovov, ovvv, t1, t2, l1, l2 = self._keep
        vb = VBlocks(_ptr(oooo), _ptr(ooov), _ptr(oovv), _ptr(ovov), _ptr(ovvv))
        h = C.c_void_p()
        if sector == "ip":
            rc = lib.gfcc_init(C.byref(h), o, v, _ptr(eps), C.byref(vb), _ptr(t1), _ptr(t2), _ptr(l1), _ptr(l2),
                               C.byref(opts), stream)
        else:
            vp = _c64(inputs.vvvv_pairs() if vvvv is None else vvvv)
            self._keep.append(vp)
            rc = lib.gfcc_init_ea(C.byref(h), o, v, _ptr(eps), C.byref(vb), _ptr(vp), _ptr(t1), _ptr(t2), _ptr(l1),
                                  _ptr(l2), C.byref(opts), stream)
        if rc != 0:
            raise GfccError(rc, "gfcc_init failed")
        self._h = h
        self._keep = None
        d = C.c_int()
        lib.gfcc_dim(h, C.byref(d))
        self.D = d.value

    # ---------------------------------------------------------------------------------------
    def _check(self, rc, allow=()):
        if rc != 0 and rc not in allow:
            msg = self._lib.gfcc_last_error(self._h)
            raise GfccError(rc, msg.decode() if msg else "")
        return rc

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gfcc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_opts(self, tol=1e-8, restart=30, max_restarts=200, precision="fp64", max_batch=0, drop_tol=1e-10,
                 deriv_indicator=False, mor_guess=True):
        opts = Opts()
        self._lib.gfcc_default_opts(C.byref(opts))
        opts.deriv_indicator = int(bool(deriv_indicator))
        opts.mor_guess = int(bool(mor_guess))
        opts.tol, opts.restart, opts.max_restarts = tol, restart, max_restarts
        opts.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        opts.max_batch, opts.drop_tol = max_batch, drop_tol
        self._check(self._lib.gfcc_set_opts(self._h, C.byref(opts)))

    # ---------------------------------------------------------------------------------------
    def sigma(self, X, precision="fp64", transpose=False, out=None):
        """Y = M X (or M^T X) for X of shape [nvec, D] complex (NumPy or CUDA torch)."""
        single = False
        if isinstance(X, np.ndarray):
            X = np.ascontiguousarray(X, dtype=np.complex128)
            if X.ndim == 1:
                X = X[None, :]
                single = True
        nvec, ld = X.shape
        if out is None:
            out = np.empty((nvec, ld), dtype=np.complex128) if isinstance(X, np.ndarray) else X.new_empty(X.shape)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self._check(self._lib.gfcc_sigma(self._h, _ptr(X), _ptr(out), nvec, ld, prec, int(bool(transpose))))
        return out[0] if single else out

    def vectors(self, orbitals, left=False):
        orb = _ints(orbitals)
        out = np.empty((len(orb), self.D))
        self._check(self._lib.gfcc_vectors(self._h, _ptr(orb), len(orb), int(left), _ptr(out), self.D))
        return out

    def solve_full(self, omegas, eta, orbitals, qorb=None, want_G=True, want_A=True, want_X=False,
                   G=None, A=None, X=None):
        """Full-dimension solves; returns dict with G [nw, np, nq], A [nw], X [nw, np, D], stats."""
        w = _c64(omegas)
        porb = _ints(orbitals)
        q = _ints(qorb) if qorb is not None else None
        nq = len(q) if q is not None else len(porb)
        nw, npp = len(w), len(porb)
        if want_G and G is None:
            G = np.empty((nw, npp, nq), dtype=np.complex128)
        if want_A and A is None:
            A = np.empty(nw)
        if want_X and X is None:
            X = np.empty((nw, npp, self.D), dtype=np.complex128)
        st = Stats()
        rc = self._lib.gfcc_solve_full(self._h, _ptr(w), nw, float(eta), _ptr(porb), npp, _ptr(q), nq,
                                       _ptr(G), _ptr(A), _ptr(X), self.D, C.byref(st))
        self._check(rc, allow=(-2,))
        stats = SolveStats(st.sigma_calls, st.sigma_cols, st.gmres_iters, st.restarts, st.max_rel_res,
                           st.not_converged)
        return {"G": G, "A": A, "X": X, "stats": stats, "converged": rc == 0}

    def green_derivatives(self, omegas, eta, orbitals, qorb=None):
        """(G, dG/dw, dG/deta), each [nw, np, nq] complex, from forward and adjoint solves."""
        w = _c64(omegas)
        porb = _ints(orbitals)
        q = _ints(qorb) if qorb is not None else None
        nq = len(q) if q is not None else len(porb)
        shape = (len(w), len(porb), nq)
        G = np.empty(shape, dtype=np.complex128)
        dw = np.empty(shape, dtype=np.complex128)
        de = np.empty(shape, dtype=np.complex128)
        self._check(self._lib.gfcc_green_derivatives(self._h, _ptr(w), len(w), float(eta), _ptr(porb), len(porb),
                                                     _ptr(q), nq, _ptr(G), _ptr(dw), _ptr(de)))
        return G, dw, de

    def green_grad_t2(self, omegas, eta, orbitals, Gbar, qorb=None):
        """(G, dL/dt2) for L = Re sum conj(Gbar) G: G [nw, np, nq] complex, dL/dt2 [o, o, v, v]."""
        w = _c64(omegas)
        porb = _ints(orbitals)
        q = _ints(qorb) if qorb is not None else None
        nq = len(q) if q is not None else len(porb)
        Gb = np.ascontiguousarray(Gbar, dtype=np.complex128)
        if Gb.shape != (len(w), len(porb), nq):
            raise ValueError("Gbar must have shape [nw, np, nq]")
        G = np.empty(Gb.shape, dtype=np.complex128)
        g = np.empty((self.o, self.o, self.v, self.v))
        self._check(self._lib.gfcc_green_grad_t2(self._h, _ptr(w), len(w), float(eta), _ptr(porb), len(porb),
                                                 _ptr(q), nq, _ptr(Gb), _ptr(G), _ptr(g)))
        return G, g

    def mor_build(self, seeds, eta, orbitals, qorb=None):
        s = _c64(seeds)
        porb = _ints(orbitals)
        q = _ints(qorb) if qorb is not None else None
        self._check(self._lib.gfcc_mor_build(self._h, _ptr(s), len(s), float(eta), _ptr(porb), len(porb), _ptr(q),
                                             len(q) if q is not None else 0))

    def mor_build_siso(self, seeds, eta, orbitals):
        """One reduced model of G_pp per orbital p (gfcc_mor_build_siso)."""
        s = _c64(seeds)
        porb = _ints(orbitals)
        self._check(self._lib.gfcc_mor_build_siso(self._h, _ptr(s), len(s), float(eta), _ptr(porb), len(porb)))

    def mor_build_krylov(self, nblocks, eta, orbitals, qorb=None):
        """Reduced model on the block Krylov space K_nblocks(M, [b_p]) (gfcc_mor_build_krylov)."""
        porb = _ints(orbitals)
        q = _ints(qorb) if qorb is not None else None
        self._check(self._lib.gfcc_mor_build_krylov(self._h, int(nblocks), float(eta), _ptr(porb), len(porb), _ptr(q),
                                                    len(q) if q is not None else 0))

    def mor_model_info(self, k):
        """{"orbital", "sampled", "m"} of model k of the current set."""
        orb, ns, m = C.c_int(), C.c_int(), C.c_int()
        self._check(self._lib.gfcc_mor_model_info(self._h, int(k), C.byref(orb), None, 0, C.byref(ns), C.byref(m)))
        w = np.empty(max(ns.value, 1))
        self._check(self._lib.gfcc_mor_model_info(self._h, int(k), C.byref(orb), w.ctypes.data_as(_dp), ns.value,
                                                  C.byref(ns), C.byref(m)))
        return {"orbital": orb.value, "sampled": w[:ns.value].copy(), "m": m.value}

    def mor_refine(self, wmin, wmax, ngrid, tol, m_max):
        m = C.c_int()
        e = C.c_double()
        rc = self._lib.gfcc_mor_refine(self._h, float(wmin), float(wmax), int(ngrid), float(tol), int(m_max),
                                       C.byref(m), C.byref(e))
        self._check(rc, allow=(-2,))
        return {"m": m.value, "max_err": e.value, "converged": rc == 0}

    def mor_eval(self, omegas, want_G=True, want_A=True, want_res=False, np_=None, nq=None, G=None, A=None,
                 maxres=None):
        w = _c64(omegas)
        nw = len(w)
        if want_G and G is None:
            info = self.mor_info()
            G = np.empty((nw, info["np"], info["nq"]), dtype=np.complex128)
        if want_A and A is None:
            A = np.empty(nw)
        if want_res and maxres is None:
            maxres = np.empty(nw)
        self._check(self._lib.gfcc_mor_eval(self._h, _ptr(w), nw, _ptr(G), _ptr(A), _ptr(maxres)))
        return {"G": G, "A": A, "maxres": maxres}

    def mor_info(self):
        ns, m, npp, nq = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        self._check(self._lib.gfcc_mor_info(self._h, None, 0, C.byref(ns), C.byref(m), None, None))
        w = np.empty(max(ns.value, 1))
        self._check(self._lib.gfcc_mor_info(self._h, w.ctypes.data_as(_dp), ns.value, C.byref(ns), C.byref(m),
                                            C.byref(npp), C.byref(nq)))
        return {"sampled": w[:ns.value].copy(), "m": m.value, "np": npp.value, "nq": nq.value}

    def mor_stats(self):
        """{"arnoldi_steps", "columns"} of the full solves made by mor_build / mor_refine."""
        a, b = C.c_longlong(), C.c_longlong()
        self._check(self._lib.gfcc_mor_stats(self._h, C.byref(a), C.byref(b)))
        return {"arnoldi_steps": a.value, "columns": b.value}

    def mor_save(self, path):
        self._check(self._lib.gfcc_mor_save(self._h, os.fsencode(path)))

    def mor_load(self, path):
        self._check(self._lib.gfcc_mor_load(self._h, os.fsencode(path)))
