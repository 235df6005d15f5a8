"""Oracle: column-pivoted Householder QR.  TEST INFRASTRUCTURE ONLY.

Step 3 of Alg. 5.1 (randomized basis): Psi P = Q R, U = first r columns of Q.  The same
factorization, with a relative stopping threshold, gives the interpolative decomposition
used by the proxy-point H^2 construction (Sec. 6).

Readings (the paper does not fix them):
* the pivot at step j is the remaining column of largest 2-norm, recomputed from the
  updated trailing rows (not downdated); ties go to the lowest column index;
* Householder reflector H = I - tau v v^T with v_0 = 1, beta = -sign(x_0)|x|, sign(0) = +;
* the factorization stops after kmax steps, or before step j when the largest remaining
  column norm is <= rtol times the first pivot norm (|R_jj| <= rtol |R_00|).
"""
from __future__ import annotations

import numpy as np


def pivoted_qr(A: np.ndarray, kmax: int, rtol: float):
    """Returns (k, piv, R, Q): piv is the full column order, R is k x ncols (columns in
    pivot order), Q is m x k with orthonormal columns, A[:, piv[:k]] = Q R[:, :k] and
    A[:, piv] ~= Q R."""
    A = np.array(A, dtype=np.float64, copy=True)
    m, ncol = A.shape
    piv = np.arange(ncol)
    kmax = min(kmax, m, ncol)
    vs, taus = [], []
    first = None
    k = 0
    for j in range(kmax):
        norms = np.sqrt((A[j:, j:] ** 2).sum(axis=0))
        c = int(np.argmax(norms))            # lowest index among equal maxima
        nmax = norms[c]
        if first is None:
            first = nmax
        if nmax == 0.0 or nmax <= rtol * first:
            break
        c += j
        if c != j:
            A[:, [j, c]] = A[:, [c, j]]
            piv[[j, c]] = piv[[c, j]]
        x = A[j:, j].copy()
        alpha = x[0]
        normx = np.sqrt(np.dot(x, x))
        beta = -normx if alpha >= 0.0 else normx
        v = x.copy()
        v[0] = alpha - beta
        if v[0] != 0.0:
            v /= v[0]
        tau = (beta - alpha) / beta
        w = v @ A[j:, j:]
        A[j:, j:] -= tau * np.outer(v, w)
        A[j, j] = beta
        A[j + 1:, j] = 0.0
        vs.append(v)
        taus.append(tau)
        k = j + 1
    R = np.triu(A[:k, :])
    Q = np.zeros((m, k))
    for a in range(k):
        Q[a, a] = 1.0
    for j in range(k - 1, -1, -1):
        v, tau = vs[j], taus[j]
        Q[j:, :] -= tau * np.outer(v, v @ Q[j:, :])
    return k, piv, R, Q
