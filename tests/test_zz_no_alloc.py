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


def test_noalloc_rejects_misaligned_output_before_any_launch(torch):
    """The epilogue stores four floats at a time, so an output that does not start on 16 bytes (an
    offset view into a larger buffer) is refused on the host, before anything runs on the device."""
    from paper_1902_06016_gb300.gfcc import launch_count, tc_gemm_noalloc
    M, N, K = 16, 32, 64
    A = torch.zeros((M, K), dtype=torch.float64, device="cuda")
    B = torch.zeros((N, K), dtype=torch.float64, device="cuda")
    big = torch.zeros(M * N + 4, dtype=torch.float32, device="cuda")
    C = big[1:1 + M * N].view(M, N)                  # contiguous, 4 bytes past a 16-byte boundary
    assert C.is_contiguous() and C.data_ptr() % 16 == 4
    n0 = launch_count()
    assert tc_gemm_noalloc(A, B, C, "bf16") == -1
    assert launch_count() == n0
    assert torch.count_nonzero(big).item() == 0


def test_noalloc_wrapper_checks_its_arguments(torch):
    from paper_1902_06016_gb300.gfcc import tc_gemm_noalloc
    A = torch.zeros((8, 16), dtype=torch.float64, device="cuda")
    B = torch.zeros((4, 16), dtype=torch.float64, device="cuda")
    C = torch.zeros((8, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        tc_gemm_noalloc(A, B, torch.zeros((8, 5), dtype=torch.float32, device="cuda"))   # C too small / wrong
    with pytest.raises(ValueError):
        tc_gemm_noalloc(torch.zeros((16, 8), dtype=torch.float64, device="cuda").t(), B, C)   # transposed A
    with pytest.raises(ValueError):
        tc_gemm_noalloc(A, torch.zeros((4, 15), dtype=torch.float64, device="cuda"), C)     # K mismatch
    with pytest.raises(TypeError):
        tc_gemm_noalloc(A.float(), B, C)
    with pytest.raises(TypeError):
        tc_gemm_noalloc(A.cpu(), B, C)
    assert tc_gemm_noalloc(A, B, C) == 0
