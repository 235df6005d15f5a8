"""Oracle: kernel functions and the dense shifted kernel matrix.  TEST INFRASTRUCTURE ONLY.

Kernels of Sec. 6, written with a length scale ell that DIVIDES the distance r = |x - y|
(the paper's parameter l multiplies it; l = 1/ell, or 1/ell^2 for the Gaussian and IMQ):

* exponential  exp(-r/ell)                        (Matern-1/2)
* Gaussian     exp(-r^2/ell^2)
* Matern-3/2   (1 + sqrt(3) r/ell) exp(-sqrt(3) r/ell)
* IMQ          1/sqrt(1 + r^2/ell^2)

Every kernel has K(x, x) = 1.  The matrix of Sec. 6.2 is A = sigma I + K(X, X).
"""
from __future__ import annotations

import numpy as np

EXP, GAUSS, MATERN32, IMQ = 0, 1, 2, 3
NAMES = {"exp": EXP, "gauss": GAUSS, "matern32": MATERN32, "imq": IMQ}


def kernel_of_r2(kind: int, r2: np.ndarray, ell: float) -> np.ndarray:
    """K as a function of the squared distance."""
    if kind == EXP:
        return np.exp(-np.sqrt(r2) / ell)
    if kind == GAUSS:
        return np.exp(-r2 / (ell * ell))
    if kind == MATERN32:
        t = np.sqrt(3.0) * np.sqrt(r2) / ell
        return (1.0 + t) * np.exp(-t)
    if kind == IMQ:
        return 1.0 / np.sqrt(1.0 + r2 / (ell * ell))
    raise ValueError(kind)


def sqdist(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Pairwise squared distances, summed coordinate by coordinate."""
    r2 = np.zeros((X.shape[0], Y.shape[0]))
    for a in range(X.shape[1]):
        d = X[:, a][:, None] - Y[:, a][None, :]
        r2 += d * d
    return r2


def kernel_block(kind: int, ell: float, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """K(X, Y) (no shift)."""
    return kernel_of_r2(kind, sqdist(X, Y), ell)


def dense_matrix(kind: int, ell: float, sigma: float, X: np.ndarray) -> np.ndarray:
    """A = sigma I + K(X, X), in the order of the rows of X."""
    A = kernel_block(kind, ell, X, X)
    A[np.diag_indices_from(A)] += sigma
    return A
