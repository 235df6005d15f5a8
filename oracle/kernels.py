"""Oracle: kernel functions and the dense shifted kernel matrix.  TEST INFRASTRUCTURE ONLY.

Kernels of Sec. 6, written with a length scale ell that DIVIDES the distance r = |x - y|
(the paper's parameter l multiplies it; l = 1/ell, or 1/ell^2 for the Gaussian and IMQ):

* exponential  exp(-r/ell)                        (Matern-1/2)
* Gaussian     exp(-r^2/ell^2)
* Matern-3/2   (1 + sqrt(3) r/ell) exp(-sqrt(3) r/ell)
* IMQ          1/sqrt(1 + r^2/ell^2)

Every kernel has K(x, x) = 1.  The matrix of Sec. 6.2 is A = sigma I + K(X, X).

The Rotne-Prager-Yamakawa kernel of Sec. 6 (3D points, particle radius a passed as ell) is
a 3 x 3 tensor: its matrix has three unknowns per point, unknown 3p + c being component c
of point p.  With r = x - y and rr = r r^T / |r|^2:

* r = 0:        (1/a) I
* |r| >= 2a:    3/(4|r|) (I + rr) + 3a^2/(2|r|^3) (I/3 - rr)
* |r| <  2a:    (1/a) (1 - 9|r|/(32a)) I + (1/a) 3|r|/(32a) rr

Reading: the paper prints the last term without the factor 1/a; with it the two branches
agree at |r| = 2a for every a (without it only for a = 1), which is the form taken here.
"""
from __future__ import annotations

import numpy as np

EXP, GAUSS, MATERN32, IMQ, RPY = 0, 1, 2, 3, 4
NAMES = {"exp": EXP, "gauss": GAUSS, "matern32": MATERN32, "imq": IMQ, "rpy": RPY}


def dofs(kind: int) -> int:
    """Unknowns per point."""
    return 3 if kind == RPY else 1


def rpy_tensor(a: float, r: np.ndarray) -> np.ndarray:
    """The 3 x 3 RPY tensor for each difference vector r (shape (m, 3) -> (m, 3, 3))."""
    r = np.asarray(r, dtype=np.float64).reshape(-1, 3)
    d = np.sqrt(np.sum(r * r, axis=1))
    eye = np.broadcast_to(np.eye(3), (len(r), 3, 3))
    out = np.empty((len(r), 3, 3))
    zero = d == 0.0
    out[zero] = eye[zero] / a
    far = ~zero & (d >= 2.0 * a)
    near = ~zero & ~far
    for sel in (far, near):
        if not np.any(sel):
            continue
        ds = d[sel][:, None, None]
        rr = r[sel][:, :, None] * r[sel][:, None, :] / (ds * ds)
        if sel is far:
            out[sel] = 3.0 / (4.0 * ds) * (eye[sel] + rr) + \
                3.0 * a * a / (2.0 * ds ** 3) * (eye[sel] / 3.0 - rr)
        else:
            out[sel] = (1.0 - 9.0 * ds / (32.0 * a)) * eye[sel] / a + \
                3.0 * ds / (32.0 * a) * rr / a
    return out


def rpy_block(a: float, X: np.ndarray, cx: np.ndarray, Y: np.ndarray, cy: np.ndarray) -> np.ndarray:
    """Entries K(x_p, y_q)[cx_p, cy_q] of the RPY tensor for unknowns (x_p, cx_p), (y_q, cy_q)."""
    m, k = X.shape[0], Y.shape[0]
    r = (X[:, None, :] - Y[None, :, :]).reshape(-1, 3)
    T = rpy_tensor(a, r).reshape(m, k, 3, 3)
    ii = np.asarray(cx, dtype=np.int64)[:, None]
    jj = np.asarray(cy, dtype=np.int64)[None, :]
    return T[np.arange(m)[:, None], np.arange(k)[None, :], ii, jj]


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


def kernel_block(kind: int, ell: float, X: np.ndarray, Y: np.ndarray, cx=None, cy=None) -> np.ndarray:
    """K(X, Y) (no shift); for RPY the rows and columns are unknowns: points X, Y with
    their components cx, cy."""
    if kind == RPY:
        return rpy_block(ell, X, cx, Y, cy)
    return kernel_of_r2(kind, sqdist(X, Y), ell)


def unknowns(kind: int, X: np.ndarray):
    """Points and components of the unknowns in their original order (3p + c for RPY)."""
    k = dofs(kind)
    if k == 1:
        return X, None
    return np.repeat(X, k, axis=0), np.tile(np.arange(k), X.shape[0])


def dense_matrix(kind: int, ell: float, sigma: float, X: np.ndarray) -> np.ndarray:
    """A = sigma I + K(X, X), in the order of the rows of X (of its unknowns for RPY)."""
    Xu, cu = unknowns(kind, np.asarray(X, dtype=np.float64))
    A = kernel_block(kind, ell, Xu, Xu, cu, cu)
    A[np.diag_indices_from(A)] += sigma
    return A
