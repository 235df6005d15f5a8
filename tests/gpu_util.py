"""Helpers for the GPU parity tests: build/load the library, oracle problem setup."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_07632_gb300 import build
    build.build()
    from paper_2011_07632_gb300 import api
    return api


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
