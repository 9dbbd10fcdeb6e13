"""Shared helpers of the GPU parity tests (inputs come from synth; expected values from oracle)."""
import functools

import numpy as np
import pytest

import synth


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_06016_gb300 import build
    build.build()
    return torch


@functools.lru_cache(maxsize=None)
def inputs(o, v, seed, scale_mode="size_consistent"):
    return synth.make_inputs(o, v, seed, scale_mode=scale_mode)


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def random_vectors(D, n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, D)) + 1j * rng.standard_normal((n, D))
