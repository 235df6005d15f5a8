"""Oracle: preconditioned conjugate gradients.  TEST INFRASTRUCTURE ONLY.

Sec. 6.2 solves the kernel systems by PCG with the SPD HSS approximation as the
preconditioner; it fixes only the stopping rule (relative residual).  Reading:
textbook PCG from x_0 = 0, every right-hand side column independent; the recursive
residual is tested after every iteration and, when it passes, the true residual
b - A x is recomputed: the column stops if that passes too, otherwise the recursive
residual is replaced by the true one and the search direction restarts from the
preconditioned residual (beta = 0), so that conjugacy is not assumed across the
replacement.  The iteration count is the number of products with A.
"""
from __future__ import annotations

import numpy as np


def pcg(apply_A, apply_M, b: np.ndarray, tol: float, maxit: int):
    """Returns (x, iters per column, true relative residual per column)."""
    b = np.asarray(b, dtype=np.float64)
    if b.ndim == 1:
        b = b[:, None]
    n, nrhs = b.shape
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = np.linalg.norm(b, axis=0)
    bnorm[bnorm == 0.0] = 1.0
    z = apply_M(r)
    p = z.copy()
    rz = np.einsum("ij,ij->j", r, z)
    iters = np.zeros(nrhs, np.int64)
    done = np.linalg.norm(r, axis=0) / bnorm <= tol
    restart = np.zeros(nrhs, bool)
    for it in range(1, maxit + 1):
        if done.all():
            break
        act = ~done
        q = apply_A(p)
        pq = np.einsum("ij,ij->j", p, q)
        alpha = np.where(act, rz / np.where(pq == 0.0, 1.0, pq), 0.0)
        x += alpha * p
        r -= alpha * q
        iters[act] = it
        rel = np.linalg.norm(r, axis=0) / bnorm
        passed = act & (rel <= tol)
        if passed.any():
            rt = b - apply_A(x)
            trel = np.linalg.norm(rt, axis=0) / bnorm
            for c in np.flatnonzero(passed):
                if trel[c] <= tol:
                    done[c] = True
                else:
                    r[:, c] = rt[:, c]
                    restart[c] = True
        act = ~done
        if not act.any():
            break
        z = apply_M(r)
        rz_new = np.einsum("ij,ij->j", r, z)
        beta = np.where(act & ~restart, rz_new / np.where(rz == 0.0, 1.0, rz), 0.0)
        restart[:] = False
        p = np.where(act, z + beta * p, p)
        rz = np.where(act, rz_new, rz)
    rel = np.linalg.norm(b - apply_A(x), axis=0) / bnorm
    return x, iters, rel
