"""Shared helpers for the GPU parity tests (no arithmetic of the method)."""
import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_13237_gb300 import build, nne
    build.build()
    nne.load()
    return torch


def rand_c(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)
