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


def pcg_mixed(apply_A, apply_A32, apply_M, b: np.ndarray, tol: float, maxit: int,
              refresh: int = 50, restarts: bool = True, switch: bool = True):
    """PCG of the precision mode (Sec. 6.2's PCG with the products inside the iteration taken
    in FP32; the paper fixes no precision).  apply_A32 is the FP32 product (its rounding is
    the caller's), apply_A the FP64 one.  The recursion and the stopping rule are those of
    pcg above; in addition, every `refresh` iterations (while FP32 products are in use) the
    recursive residual of every column is replaced by the FP64 true residual b - A x, and
      - with `restarts`, a column still iterating whose true residual is above twice its
        recursive one restarts its direction (beta = 0): the FP32 recursion no longer
        describes the FP64 residual, and each block of iterations becomes an inner PCG of
        iterative refinement for A d = r;
      - with `switch`, if some column still iterating has a true residual above 0.9 of its
        value at the previous refresh (a block without progress), the products are FP64
        from then on and every column still iterating restarts.
    refresh = 0 gives pcg with apply_A32 in the iteration.  Returns (x, iters per column,
    true relative residual per column, iteration of the switch or None)."""
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
    tprev = np.full(nrhs, np.inf)
    fp32 = True
    switched_at = None
    for it in range(1, maxit + 1):
        if done.all():
            break
        act = ~done
        q = apply_A32(p) if fp32 else apply_A(p)
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
        if fp32 and refresh > 0 and it % refresh == 0:
            rt = b - apply_A(x)
            trel = np.linalg.norm(rt, axis=0) / bnorm
            r = rt
            free = act & ~restart
            if switch and np.any(free & (trel > 0.9 * tprev)):
                fp32 = False
                switched_at = it
                restart |= act
            elif restarts:
                restart |= free & (trel > 2.0 * rel)
            tprev = trel
        z = apply_M(r)
        rz_new = np.einsum("ij,ij->j", r, z)
        beta = np.where(act & ~restart, rz_new / np.where(rz == 0.0, 1.0, rz), 0.0)
        restart[:] = False
        p = np.where(act, z + beta * p, p)
        rz = np.where(act, rz_new, rz)
    rel = np.linalg.norm(b - apply_A(x), axis=0) / bnorm
    return x, iters, rel, switched_at
