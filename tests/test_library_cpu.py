"""Host-side checks of the C ABI (no GPU): the library builds/loads and exports exactly the entry
points that include/gfcc.h declares, with ctypes prototypes for each."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gfcc.h")


def declared_symbols():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gfcc_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1902_06016_gb300 import build
    try:
        return build.build()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(str(e))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["gfcc_init", "gfcc_sigma", "gfcc_solve_full", "gfcc_mor_build", "gfcc_mor_refine",
                 "gfcc_mor_eval", "gfcc_mor_save", "gfcc_mor_load", "gfcc_last_error", "gfcc_free"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (gfcc_[a-z0-9_]+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_prototypes_cover_the_header(lib_path):
    from paper_1902_06016_gb300 import gfcc
    lib = gfcc.load(lib_path)
    assert sorted(gfcc.PROTOTYPES) == declared_symbols()
    for name in declared_symbols():
        assert hasattr(lib, name)


def test_default_options_without_gpu(lib_path):
    import ctypes
    from paper_1902_06016_gb300 import gfcc
    lib = gfcc.load(lib_path)
    o = gfcc.Opts()
    assert lib.gfcc_default_opts(ctypes.byref(o)) == 0
    assert o.tol == 1e-8 and o.restart == 30 and o.precision == 0
    assert lib.gfcc_default_opts(None) == -1
    # argument errors are caught on the host before any device work
    h = ctypes.c_void_p()
    assert lib.gfcc_init(ctypes.byref(h), 1, 4, None, None, None, None, None, None, None, None) == -1
