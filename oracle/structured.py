"""Oracle: the SPD HSS construction of Alg. 5.3 on an H^2 matrix, without forming the
dense matrix.  TEST INFRASTRUCTURE ONLY.

The quadratic oracle (spdhss.py) needs the dense matrix and so stops at a few thousand
points; this one follows Alg. 5.3 on the H^2 representation itself, so that the GPU's
construction can be checked at tens of thousands of points:

* the samples Y^(k) = (A - blkdiag_k A) Omega (Eq. Yk) are summed block by block over the
  H^2 blocks of A: the near blocks K(X_i, X_j) of leaf pairs (plus sigma I on the
  diagonal) and the far blocks U_i B_ij U_j^T of the Type-3 pairs (explicit nested bases,
  Eq. nested); a block (i, j) enters Y^(k) unless i and j lie in the same node of level k;
* leaf level (Alg. 5.3): A_ii + sigma I = S_i S_i^T, Lambda_i Omega = S_i^{-1} Y_i^(1),
  V_i from its column-pivoted QR, Phi_i = V_i^T S_i^{-1} (explicit), U_i = S_i V_i;
* levels k >= 2: bold B_ii from the children's B, (I + bold B_ii)^{+-1/2} by a symmetric
  eigendecomposition (Eq. Si0), Lambda_i Omega = (I + bold B_ii)^{-1/2} [Phi_c Y_c^(k)],
  Vbar_i, Phi_i = Vbar_i^T (I + bold B_ii)^{-1/2} diag(Phi_c) (Eq. phi),
  R_i = (I + bold B_ii)^{1/2} Vbar_i (Eq. Rik);
* B_ij for the pairs the next level needs (Sec. 5.2.2): Type-1 (near) pairs at the leaves
  B_ij = Phi_i K(X_i, X_j) Phi_j^T, above them by the recursion (Eq. Mijk)
  B_ij = Vbar_i^T (I + bold B_ii)^{-1/2} bold B_ij (I + bold B_jj)^{-1/2} Vbar_j, whose
  blocks are the children pairs' B; Type-3 (far) pairs B_ij = (Phi U)_i B^H2_ij (Phi U)_j^T
  with (Phi U)_i = Phi_i U_i (Eq. type3_Mij).  Both are exact identities of
  B_ij = Phi_i A_ij Phi_j^T (Eq. bij_hss).

The result is an spdhss.HSS (D, U, R and B of every computed pair), so assemble_dense and
the ULV oracle apply to it; hss_matvec and h2_matvec apply the two matrices without dense
forms.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import kernels as K
from .h2 import H2, explicit_basis
from .linalg import pivoted_qr
from .spdhss import HSS, RANK_RTOL, _sym_power


def _near_block(h2: H2, i: int, j: int) -> np.ndarray:
    t = h2.tree
    bi, ei, bj, ej = t.begin[i], t.end[i], t.begin[j], t.end[j]
    ci = h2.cs[bi:ei] if h2.cs is not None else None
    cj = h2.cs[bj:ej] if h2.cs is not None else None
    A = K.kernel_block(h2.kind, h2.ell, h2.Xs[bi:ei], h2.Xs[bj:ej], ci, cj)
    if i == j:
        A = A + h2.sigma * np.eye(ei - bi)
    return A


def _bases(h2: H2) -> dict:
    t = h2.tree
    return {i: explicit_basis(h2, i) for i in range(t.num_nodes) if h2.rank(i) > 0}


class H2Apply:
    """The near blocks and explicit bases of an H^2 matrix, kept for repeated products."""

    def __init__(self, h2: H2):
        t = h2.tree
        self.h2 = h2
        self.Ub = _bases(h2)
        self.near = {(int(i), int(j)): _near_block(h2, int(i), int(j))
                     for i in t.nodes_at_depth(t.D) for j in t.near(int(i))}

    def __call__(self, X):
        return h2_matvec(self.h2, X, self.Ub, self.near)


def h2_matvec(h2: H2, X: np.ndarray, Ub: dict = None, near: dict = None) -> np.ndarray:
    """A X for the H^2 matrix A, X in tree order: near blocks of the leaf pairs plus the
    far blocks U_i B_ij U_j^T of every Type-3 pair."""
    t = h2.tree
    X = np.asarray(X, dtype=np.float64)
    vec = X.ndim == 1
    if vec:
        X = X[:, None]
    Ub = _bases(h2) if Ub is None else Ub
    Y = np.zeros_like(X)
    for i in t.nodes_at_depth(t.D):
        bi, ei = t.begin[i], t.end[i]
        for j in t.near(i):
            j = int(j)
            Aij = near[(i, j)] if near is not None else _near_block(h2, i, j)
            Y[bi:ei] += Aij @ X[t.begin[j]:t.end[j]]
    xhat = {j: Ub[j].T @ X[t.begin[j]:t.end[j]] for j in Ub}
    for i in Ub:
        bi, ei = t.begin[i], t.end[i]
        for j in t.far(i):
            j = int(j)
            if j in Ub:
                Y[bi:ei] += Ub[i] @ (h2.B[(i, j)] @ xhat[j])
    return Y[:, 0] if vec else Y


def sample_products_h2(h2: H2, Omega: np.ndarray, Ub: dict = None) -> dict:
    """Y^(k) = (A - blkdiag_k A) Omega for k = 1 .. L-1 (Eq. Yk), block by block over the
    H^2 blocks of A: block (i, j), i and j of depth t, is left out of Y^(k) exactly when
    i and j have the same ancestor at the depth of level k."""
    t = h2.tree
    Ub = _bases(h2) if Ub is None else Ub
    Y = {k: np.zeros_like(Omega) for k in range(1, t.L)}

    def add(i, j, P):
        ti = t.depth(i)
        for k in range(1, t.L):
            dk = t.D + 1 - k
            same = (i == j) if ti <= dk else \
                t.ancestor_at_depth(i, dk) == t.ancestor_at_depth(j, dk)
            if not same:
                Y[k][t.begin[i]:t.end[i]] += P

    for i in t.nodes_at_depth(t.D):
        for j in t.near(i):
            j = int(j)
            add(i, j, _near_block(h2, i, j) @ Omega[t.begin[j]:t.end[j]])
    for i in Ub:
        for j in t.far(i):
            j = int(j)
            if j in Ub:
                P = Ub[i] @ (h2.B[(i, j)] @ (Ub[j].T @ Omega[t.begin[j]:t.end[j]]))
                add(i, j, P)
    return Y


def build_spdhss_h2(h2: H2, Omega: np.ndarray, r: int, rtol: float = RANK_RTOL) -> HSS:
    """Alg. 5.3 on the H^2 matrix h2 with the sketch Omega (tree order, n x (r + p)) and
    rank cap r; Omega's columns and the pivoted QR's stopping rule as in spdhss.build_spdhss."""
    rtol = max(float(rtol), RANK_RTOL)
    t = h2.tree
    hss = HSS(t)
    Lv = t.L
    if Lv == 1:
        hss.D[0] = _near_block(h2, 0, 0)
        return hss
    Ub = _bases(h2)
    Y = sample_products_h2(h2, Omega, Ub)
    PhiU = {}

    def phiu(i):
        if i not in PhiU:
            PhiU[i] = hss.Phi[i] @ Ub[i] if i in Ub else np.zeros((hss.rank[i], 0))
        return PhiU[i]

    def type3(i, j):
        return phiu(i) @ h2.B[(i, j)] @ phiu(j).T if (i in Ub and j in Ub) else \
            np.zeros((hss.rank[i], hss.rank[j]))

    # leaf level
    leaves = [int(i) for i in t.nodes_at_level(1)]
    for i in leaves:
        b, e = t.begin[i], t.end[i]
        Aii = _near_block(h2, i, i)
        hss.D[i] = Aii
        S = np.linalg.cholesky(Aii)
        lam = sla.solve_triangular(S, Y[1][b:e], lower=True)
        k, piv, Rq, V = pivoted_qr(lam, r, rtol)
        hss.S[i] = S
        hss.Vbar[i] = V
        hss.rank[i] = k
        hss.Phi[i] = sla.solve_triangular(S, V, lower=True, trans="T").T   # V^T S^{-1}
        hss.U[i] = S @ V
    for i in leaves:
        for j in t.near(i):
            j = int(j)
            if j != i:
                hss.B[(i, j)] = hss.Phi[i] @ _near_block(h2, i, j) @ hss.Phi[j].T
        for j in t.far(i):
            hss.B[(i, int(j))] = type3(i, int(j))
    # levels 2 .. L-1
    Fmh, kids_of, off_of = {}, {}, {}
    for k in range(2, Lv):
        nodes = [int(i) for i in t.nodes_at_level(k)]
        for i in nodes:
            kids = [int(c) for c in t.children(i)]
            off = np.concatenate([[0], np.cumsum([hss.rank[c] for c in kids])]).astype(int)
            kids_of[i], off_of[i] = kids, off
            m = int(off[-1])
            Bb = np.zeros((m, m))
            for a, ca in enumerate(kids):
                for bb, cb in enumerate(kids):
                    if ca != cb:
                        Bb[off[a]:off[a + 1], off[bb]:off[bb + 1]] = hss.B[(ca, cb)]
            Fh = _sym_power(Bb, 0.5)
            Fmh[i] = _sym_power(Bb, -0.5)
            lam = Fmh[i] @ np.vstack([hss.Phi[c] @ Y[k][t.begin[c]:t.end[c]] for c in kids])
            kk, piv, Rq, Vb = pivoted_qr(lam, r, rtol)
            b, e = t.begin[i], t.end[i]
            PhiStack = np.zeros((m, e - b))
            for a, c in enumerate(kids):
                PhiStack[off[a]:off[a + 1], t.begin[c] - b:t.end[c] - b] = hss.Phi[c]
            hss.Bbold[i] = Bb
            hss.Fhalf[i] = Fh
            hss.Vbar[i] = Vb
            hss.rank[i] = kk
            hss.Phi[i] = Vb.T @ Fmh[i] @ PhiStack
            hss.R[i] = Fh @ Vb
        for i in nodes:
            for j in t.near(i):
                j = int(j)
                if j == i:
                    continue
                ki, oi = kids_of[i], off_of[i]
                kj, oj = kids_of[j], off_of[j]
                Bij = np.zeros((oi[-1], oj[-1]))
                for a, ca in enumerate(ki):
                    for bb, cb in enumerate(kj):
                        Bij[oi[a]:oi[a + 1], oj[bb]:oj[bb + 1]] = hss.B[(ca, cb)]
                hss.B[(i, j)] = hss.Vbar[i].T @ Fmh[i] @ Bij @ Fmh[j] @ hss.Vbar[j]
            for j in t.far(i):
                hss.B[(i, int(j))] = type3(i, int(j))
    return hss


def hss_matvec(hss: HSS, X: np.ndarray) -> np.ndarray:
    """H X for the HSS matrix {D_i, U_i, R_i, B_ij (siblings)}, X in tree order."""
    t = hss.tree
    X = np.asarray(X, dtype=np.float64)
    vec = X.ndim == 1
    if vec:
        X = X[:, None]
    if t.L == 1:
        Y = hss.D[0] @ X
        return Y[:, 0] if vec else Y
    xt = {}
    for k in range(1, t.L):
        for i in t.nodes_at_level(k):
            i = int(i)
            xt[i] = hss.U[i].T @ X[t.begin[i]:t.end[i]] if k == 1 else \
                hss.R[i].T @ np.vstack([xt[int(c)] for c in t.children(i)])
    yt = {i: np.zeros_like(v) for i, v in xt.items()}
    for (i, j), Bij in hss.siblings_B().items():
        yt[i] += Bij @ xt[j]
    for k in range(t.L - 1, 1, -1):
        for i in t.nodes_at_level(k):
            i = int(i)
            z = hss.R[i] @ yt[i]
            o = 0
            for c in t.children(i):
                rc = yt[int(c)].shape[0]
                yt[int(c)] += z[o:o + rc]
                o += rc
    Y = np.zeros_like(X)
    for i in t.nodes_at_level(1):
        i = int(i)
        b, e = t.begin[i], t.end[i]
        Y[b:e] = hss.D[i] @ X[b:e] + hss.U[i] @ yt[i]
    return Y[:, 0] if vec else Y
