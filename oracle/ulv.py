"""Oracle: ULV factorization and solve of a symmetric positive definite HSS matrix.
TEST INFRASTRUCTURE ONLY.

The paper applies the SPD HSS approximation through a ULV decomposition (Sec. 1 and
Sec. 6, citing Xia et al. 2010) without giving it.  The reading used here is the
symmetric (Cholesky) ULV:

for every node i of levels 1 .. L-1, bottom-up, with a dense diagonal block D_i
(leaf: A_ii; above: the children's reduced blocks coupled by U~_a B_ab U~_b^T) and a
basis W_i (leaf: U_i; above: diag(U~_children) R_i), m x r_i:
  W_i = Q_i [U~_i; 0]                       (full Householder QR, Q_i = [Q_par Q_perp])
  Q_i^T D_i Q_i = [[D_pp, D_pq], [D_qp, D_qq]]  (p: first r_i coordinates, q: the rest)
  D_qq = L_q L_q^T,  L_pq = D_pq L_q^{-T},  reduced block  D^_i = D_pp - L_pq L_pq^T
and at the root a dense Cholesky of the block assembled from the children.
Solving is a forward sweep (y_q = L_q^{-1} b_q, b^ = b_p - L_pq y_q) and a backward
sweep (x_q = L_q^{-T} (y_q - L_pq^T x_p), x = Q_i [x_p; x_q]).  Every Cholesky exists
because the HSS matrix is SPD (Sec. 3.2).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .spdhss import HSS


class ULV:
    def __init__(self, hss: HSS):
        self.hss = hss
        tree = hss.tree
        self.f = {}
        Dred, Ured = {}, {}
        if tree.L == 1:
            self.root = np.linalg.cholesky(hss.D[0])
            return
        for k in range(1, tree.L):
            for i in tree.nodes_at_level(k):
                if k == 1:
                    Di = hss.D[i]
                    Wi = hss.U[i]
                else:
                    Di = self._assemble(i, Dred, Ured)
                    Wi = sla.block_diag(*[Ured[int(c)] for c in tree.children(i)]) @ hss.R[i]
                m, r = Wi.shape
                Q, Rw = np.linalg.qr(Wi, mode="complete")
                Dt = Q.T @ Di @ Q
                Lq = np.linalg.cholesky(Dt[r:, r:]) if m > r else np.zeros((0, 0))
                Lpq = sla.solve_triangular(Lq, Dt[r:, :r], lower=True).T if m > r else np.zeros((r, 0))
                Dred[i] = Dt[:r, :r] - Lpq @ Lpq.T
                Ured[i] = Rw[:r, :]
                self.f[i] = (Q, Lq, Lpq, r)
        self.root = np.linalg.cholesky(self._assemble(0, Dred, Ured))

    def _assemble(self, i, Dred, Ured):
        kids = [int(c) for c in self.hss.tree.children(i)]
        rc = [Dred[c].shape[0] for c in kids]
        off = np.concatenate([[0], np.cumsum(rc)])
        D = np.zeros((off[-1], off[-1]))
        for a, ca in enumerate(kids):
            for b, cb in enumerate(kids):
                blk = Dred[ca] if a == b else Ured[ca] @ self.hss.B[(ca, cb)] @ Ured[cb].T
                D[off[a]:off[a + 1], off[b]:off[b + 1]] = blk
        return D

    def solve(self, b: np.ndarray) -> np.ndarray:
        """x = H^{-1} b, b in tree order (n or n x nrhs)."""
        tree = self.hss.tree
        b = np.asarray(b, dtype=np.float64)
        vec = b.ndim == 1
        if vec:
            b = b[:, None]
        if tree.L == 1:
            x = sla.cho_solve((self.root, True), b)
            return x[:, 0] if vec else x
        red, yq = {}, {}
        for k in range(1, tree.L):
            for i in tree.nodes_at_level(k):
                Q, Lq, Lpq, r = self.f[i]
                bi = b[tree.begin[i]:tree.end[i]] if k == 1 else \
                    np.vstack([red[int(c)] for c in tree.children(i)])
                bt = Q.T @ bi
                y = sla.solve_triangular(Lq, bt[r:], lower=True) if Lq.size else bt[r:]
                yq[i] = y
                red[i] = bt[:r] - Lpq @ y
        kids = [int(c) for c in tree.children(0)]
        xr = sla.cho_solve((self.root, True), np.vstack([red[c] for c in kids]))
        xp = {}
        o = 0
        for c in kids:
            r = red[c].shape[0]
            xp[c] = xr[o:o + r]
            o += r
        x = np.zeros_like(b)
        for k in range(tree.L - 1, 0, -1):
            for i in tree.nodes_at_level(k):
                Q, Lq, Lpq, r = self.f[i]
                xq = sla.solve_triangular(Lq, yq[i] - Lpq.T @ xp[i], lower=True, trans="T") \
                    if Lq.size else yq[i]
                xi = Q @ np.vstack([xp[i], xq])
                if k == 1:
                    x[tree.begin[i]:tree.end[i]] = xi
                else:
                    o = 0
                    for c in tree.children(i):
                        rc = red[int(c)].shape[0]
                        xp[int(c)] = xi[o:o + rc]
                        o += rc
        return x[:, 0] if vec else x


def dense_solve(H: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x = H^{-1} b by a dense Cholesky factorization."""
    return sla.cho_solve(sla.cho_factor(H, lower=True), b)
