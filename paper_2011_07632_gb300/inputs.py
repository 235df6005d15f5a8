"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds no arithmetic of the method itself: it only draws points, right-hand
sides and the Gaussian sketch matrix with numpy's Philox bit generator (Salmon et al.,
SC'11), so that the GPU path and the CPU oracle see bit-identical inputs.

The workloads mirror the paper's experiments (Sec. 6): points uniform in a unit cube
(or the paper's ball / sphere sets), random right-hand sides, and a standard normal
sketch Omega with r + p columns (Alg. 5.1, step 1).
"""
from __future__ import annotations

import numpy as np


def _gen(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed), int(stream)]))


def uniform_cube(n: int, dim: int, seed: int = 0) -> np.ndarray:
    """n points uniform in [0,1]^dim, row-major (n, dim) float64."""
    return _gen(seed, 0).random((n, dim))


def ball(n: int, seed: int = 0) -> np.ndarray:
    """n points uniform in the 3D ball of radius (3n/(4 pi))^(1/3) (constant density, Sec. 6)."""
    g = _gen(seed, 1)
    rad = (3.0 * n / (4.0 * np.pi)) ** (1.0 / 3.0)
    v = g.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    u = g.random(n) ** (1.0 / 3.0)
    return v * (rad * u)[:, None]


def sphere(n: int, seed: int = 0) -> np.ndarray:
    """n points uniform on the sphere of radius sqrt(n/(4 pi)) (Sec. 6)."""
    g = _gen(seed, 2)
    rad = np.sqrt(n / (4.0 * np.pi))
    v = g.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v * rad


def rhs_uniform(n: int, nrhs: int, seed: int = 1) -> np.ndarray:
    """Right-hand sides with entries uniform on [-0.5, 0.5] (the paper's experiments),
    column-major (n, nrhs) float64 in Fortran order."""
    return np.asfortranarray(_gen(seed, 6).random((n, nrhs)) - 0.5)


def rhs(n: int, nrhs: int, seed: int = 1) -> np.ndarray:
    """Right-hand sides, entries N(0,1), column-major (n, nrhs) float64 in Fortran order."""
    return np.asfortranarray(_gen(seed, 3).standard_normal((n, nrhs)))


def sketch(n: int, s: int, seed: int = 2) -> np.ndarray:
    """Gaussian sketch Omega (n, s), standard normal entries (Alg. 5.1 step 1), Fortran order."""
    return np.asfortranarray(_gen(seed, 4).standard_normal((n, s)))


def log_uniform_sizes(count: int, lo: int, hi: int, seed: int = 3) -> np.ndarray:
    """Problem sizes n drawn log-uniformly in [lo, hi] (multi-instance workloads)."""
    g = _gen(seed, 5)
    return np.floor(np.exp(g.uniform(np.log(lo), np.log(hi), count))).astype(np.int64)
