"""Helpers shared by the GPU parity tests."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_06216_gb300 import build
    build.build()
    return torch


def rel_l1(x, ref):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.abs(x - ref).sum() / np.abs(ref).sum())
