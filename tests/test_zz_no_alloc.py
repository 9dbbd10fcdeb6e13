"""The allocation-free tensor-core GEMM entry point (gfcc_tc_gemm_noalloc) against the allocating one
(gfcc_tc_gemm), through the C ABI on a GPU.

It exists for callers that cannot allocate device memory where they call it (a framework that owns
all device memory, a path that must not synchronise the device through cudaMalloc/cudaFree, code that
must not run out of memory after start-up). Its scratch is a fixed array inside the library, shared
by every call, so two calls in a row must each give the right answer (the second one must not see
the first one's leftovers). This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_06016_gb300 import build
    build.build()
    return torch


def _bound(A, B):
    # FP32 accumulation inside the tensor core (the same bound as the allocating entry point's tests)
    return 2.0 ** -17 * (np.abs(A) @ np.abs(B).T) + 1e-6


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_noalloc_matches_allocating_entry_point_twice(torch, prec):
    from paper_1902_06016_gb300.gfcc import tc_gemm, tc_gemm_noalloc
    rng = np.random.default_rng(7 if prec == "bf16" else 8)
    shapes = [(300, 513, 1000), (130, 70, 77)]          # second call: different, smaller shapes
    for M, N, K in shapes:
        A = rng.standard_normal((M, K))
        B = rng.standard_normal((N, K))
        ref = tc_gemm(A, B, prec)
        Ad = torch.from_numpy(A).cuda()
        Bd = torch.from_numpy(B).cuda()
        Cd = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
        assert tc_gemm_noalloc(Ad, Bd, Cd, prec) == 0
        C = Cd.cpu().numpy()
        assert np.all(np.isfinite(C))
        assert np.all(np.abs(C.astype(np.float64) - ref) <= _bound(A, B))


def test_noalloc_rejects_sizes_beyond_its_scratch(torch):
    from paper_1902_06016_gb300.gfcc import tc_gemm_noalloc
    A = torch.zeros((4096, 4096), dtype=torch.float64, device="cuda")
    B = torch.zeros((4096, 4096), dtype=torch.float64, device="cuda")
    C = torch.zeros((4096, 4096), dtype=torch.float32, device="cuda")
    assert tc_gemm_noalloc(A, B, C, "bf16") == -1          # 2 x 32 MiB of bf16 operands > 32 MiB
    small = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    assert tc_gemm_noalloc(A[:8], B[:8], small, "bf16") == 0
