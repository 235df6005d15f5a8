"""Oracle: SPD HSS construction by scaling-and-compression, quadratic cost.
TEST INFRASTRUCTURE ONLY.

On a dense SPD matrix M (the shifted kernel matrix, or the dense form of an H^2 matrix),
in tree order, with a given sketch Omega (n x (r+p)).  The steps follow Alg. 4.1 (Sec. 4)
with the bases of Sec. 5.2.1 (randomized, Alg. 5.1, applied to Lambda_{ii^c} Omega):

leaf level (k = 1)
  A_ii = S_i S_i^T (Cholesky), Lambda_i Omega = S_i^{-1} Y_i^(1),  Y^(k) = (M - blkdiag_k M) Omega
  V_i = first r_i columns of Q from the pivoted QR of Lambda_i Omega
  Phi_i = V_i^T S_i^{-1} (explicit r_i x |I_i| matrix), U_i = S_i V_i
  B_ij = Phi_i M_ij Phi_j^T for ALL i != j in lvl(1)          (Eq. bij_hss)
levels k = 2 .. L-1
  bold B_ii from the children's B (zero diagonal blocks), (I + bold B_ii)^{+-1/2} by a
  symmetric eigendecomposition (Eq. Si0)
  Lambda_i Omega = (I + bold B_ii)^{-1/2} diag(Phi_children) Y_i^(k)
  Vbar_i from its pivoted QR, Phi_i = Vbar_i^T (I + bold B_ii)^{-1/2} diag(Phi_children) (Eq. phi)
  R_i = (I + bold B_ii)^{1/2} Vbar_i                          (Eq. Rik)
  B_ij = Phi_i M_ij Phi_j^T for ALL i != j in lvl(k)

No Type-1 / Type-3 shortcut is used: B_ij always comes from the matrix itself, so the
accelerated algebra of Sec. 5.2.2 is checked independently.  ``factor="chol"`` replaces
(I + bold B)^{1/2} by its Cholesky factor L (I + bold B = L L^T); the two differ by an
orthogonal factor on the right, which column-pivoted QR absorbs, so the assembled HSS
matrix is the same.  r_i = min(r, rows, numerical rank), the pivoted QR stopping when
the largest remaining column norm is <= 1e-14 times the first.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from .linalg import pivoted_qr
from .tree import Tree

RANK_RTOL = 1e-14


@dataclass
class HSS:
    tree: Tree
    D: dict = field(default_factory=dict)      # leaf -> dense diagonal block A_ii
    U: dict = field(default_factory=dict)      # leaf -> U_i (|I_i| x r_i)
    R: dict = field(default_factory=dict)      # nonleaf (levels 2..L-1) -> R_i (sum r_c x r_i)
    B: dict = field(default_factory=dict)      # (i, j) -> B_ij for every i != j of a level
    Phi: dict = field(default_factory=dict)    # node -> explicit Phi_i (r_i x |I_i|)
    Vbar: dict = field(default_factory=dict)   # leaf: V_i; nonleaf: Vbar_i
    S: dict = field(default_factory=dict)      # leaf -> Cholesky factor S_i
    Bbold: dict = field(default_factory=dict)  # nonleaf -> bold B_ii
    Fhalf: dict = field(default_factory=dict)  # nonleaf -> (I + bold B_ii)^{1/2} or its Cholesky factor
    rank: dict = field(default_factory=dict)

    def siblings_B(self):
        """Coefficient matrices of the final HSS form: sibling pairs only."""
        t = self.tree
        return {(i, j): b for (i, j), b in self.B.items() if t.parent[i] == t.parent[j]}


def build_spdhss_adaptive(tree: Tree, M: np.ndarray, Omega: np.ndarray, rank_cap: int,
                          p: int, rtol: float, r0: int = 64) -> HSS:
    """Tolerance-driven construction with a growing sketch (the extension remarked after
    Alg. 5.3: add vectors to Omega until the truncation at rtol is no longer limited by the
    sketch).  Omega holds at least rank_cap + p columns; an attempt with rank cap r uses its
    first r + p.  Starting from r = min(rank_cap, r0), the cap doubles until every rank is
    below the cap of the attempt (the p extra columns then oversample every kept rank) or
    the cap reaches rank_cap."""
    r = min(rank_cap, r0)
    while True:
        hss = build_spdhss(tree, M, Omega[:, :r + p], r, rtol=rtol)
        if max(hss.rank.values(), default=0) < r or r >= rank_cap:
            hss.sketch_rank = r
            return hss
        r = min(2 * r, rank_cap)


def sample_products(tree: Tree, M: np.ndarray, Omega: np.ndarray):
    """Y^(k) = (M - blkdiag_k(M)) Omega for k = 1 .. L-1 (Eq. Yk), literally."""
    Y = {}
    full = M @ Omega
    for k in range(1, tree.L):
        Yk = full.copy()
        for i in tree.nodes_at_level(k):
            b, e = tree.begin[i], tree.end[i]
            Yk[b:e] -= M[b:e, b:e] @ Omega[b:e]
        Y[k] = Yk
    return Y


def _sym_power(Bb: np.ndarray, p: float) -> np.ndarray:
    lam, Q = np.linalg.eigh(Bb)
    d = 1.0 + lam
    if np.any(d <= 0.0):
        raise np.linalg.LinAlgError("I + bold B_ii is not SPD")
    return (Q * d ** p) @ Q.T


def build_spdhss(tree: Tree, M: np.ndarray, Omega: np.ndarray, r: int, factor: str = "eig",
                 rtol: float = RANK_RTOL) -> HSS:
    """Alg. 5.3.  rtol > RANK_RTOL truncates every basis at the relative tolerance rtol
    (the pivoted QR of the scaled sample stops when the largest remaining column norm is
    <= rtol times the first), with r as the rank cap: the tolerance-driven construction
    with a fixed sketch."""
    rtol = max(float(rtol), RANK_RTOL)
    hss = HSS(tree)
    Y = sample_products(tree, M, Omega)
    Lv = tree.L
    # leaf level
    leaves = list(tree.nodes_at_level(1)) if Lv > 1 else [0]
    for i in leaves:
        b, e = tree.begin[i], tree.end[i]
        Aii = M[b:e, b:e]
        hss.D[i] = Aii.copy()
        if Lv == 1:
            break
        S = np.linalg.cholesky(Aii)
        lam = sla.solve_triangular(S, Y[1][b:e], lower=True)
        k, piv, Rq, V = pivoted_qr(lam, r, rtol)
        hss.S[i] = S
        hss.Vbar[i] = V
        hss.rank[i] = k
        hss.Phi[i] = sla.solve_triangular(S, V, lower=True, trans="T").T   # V^T S^{-1}
        hss.U[i] = S @ V
    if Lv == 1:
        return hss
    _all_pairs_B(hss, M, 1)
    for k in range(2, Lv):
        for i in tree.nodes_at_level(k):
            kids = [int(c) for c in tree.children(i)]
            rc = [hss.rank[c] for c in kids]
            off = np.concatenate([[0], np.cumsum(rc)])
            m = int(off[-1])
            Bb = np.zeros((m, m))
            for a, ca in enumerate(kids):
                for bb, cb in enumerate(kids):
                    if ca != cb:
                        Bb[off[a]:off[a + 1], off[bb]:off[bb + 1]] = hss.B[(ca, cb)]
            b, e = tree.begin[i], tree.end[i]
            PhiStack = np.zeros((m, e - b))
            for a, c in enumerate(kids):
                PhiStack[off[a]:off[a + 1], tree.begin[c] - b:tree.end[c] - b] = hss.Phi[c]
            if factor == "eig":
                Fh = _sym_power(Bb, 0.5)
                Fmh = _sym_power(Bb, -0.5)
            else:
                Fh = np.linalg.cholesky(np.eye(m) + Bb)
                Fmh = sla.solve_triangular(Fh, np.eye(m), lower=True)
            lam = Fmh @ (PhiStack @ Y[k][b:e])
            kk, piv, Rq, Vb = pivoted_qr(lam, r, rtol)
            hss.Bbold[i] = Bb
            hss.Fhalf[i] = Fh
            hss.Vbar[i] = Vb
            hss.rank[i] = kk
            hss.Phi[i] = Vb.T @ Fmh @ PhiStack
            hss.R[i] = Fh @ Vb
        _all_pairs_B(hss, M, k)
    return hss


def _principal_basis(C: np.ndarray, r: int):
    """Orthonormal V with col(V) in col(C) minimizing ||C - V V^T C||_F over r columns:
    the leading left singular vectors (Eckart-Young); singular values <= RANK_RTOL times
    the largest count as zero."""
    if C.shape[0] == 0 or C.shape[1] == 0:
        return 0, np.zeros((C.shape[0], 0))
    Uc, sv, _ = np.linalg.svd(C, full_matrices=False)
    k = int(min(r, np.sum(sv > RANK_RTOL * sv[0]))) if sv[0] > 0 else 0
    return k, Uc[:, :k]


def build_spdhss_deterministic(tree: Tree, M: np.ndarray, r: int, keep: bool = False) -> HSS:
    """Alg. 4.1 as printed, without sketching: the leaf bases V_i minimize
    ||C_ii^c - V_i V_i^T C_ii^c||_F for the explicitly scaled block row
    C_ij = S_i^{-1} A_ij S_j^{-T} (j != i in lvl(1)), and above the leaves Vbar_i minimizes
    ||E_ii^c - Vbar_i Vbar_i^T E_ii^c||_F (Eq. minimization) for
    E_ij = (I + bold B_ii)^{-1/2} bold B_ij (I + bold B_jj)^{-1/2}, j != i in lvl(k), both
    by a truncated SVD.  B_ij, R_i, U_i as in build_spdhss.  It measures what the sketch of
    Sec. 5.2.1 costs in accuracy; keep=True stores every C_ii^c / E_ii^c in hss.target."""
    hss = HSS(tree)
    hss.target = {}
    Lv = tree.L
    leaves = list(tree.nodes_at_level(1)) if Lv > 1 else [0]
    for i in leaves:
        b, e = tree.begin[i], tree.end[i]
        hss.D[i] = M[b:e, b:e].copy()
        if Lv > 1:
            hss.S[i] = np.linalg.cholesky(hss.D[i])
    if Lv == 1:
        return hss
    for i in leaves:
        b, e = tree.begin[i], tree.end[i]
        blocks = []
        for j in leaves:
            if j == i:
                continue
            bj, ej = tree.begin[j], tree.end[j]
            Cij = sla.solve_triangular(hss.S[i], M[b:e, bj:ej], lower=True)
            blocks.append(sla.solve_triangular(hss.S[j], Cij.T, lower=True).T)   # C_ij S_j^{-T}
        C = np.hstack(blocks) if blocks else np.zeros((e - b, 0))
        k, V = _principal_basis(C, r)
        if keep:
            hss.target[i] = C
        hss.Vbar[i] = V
        hss.rank[i] = k
        hss.Phi[i] = sla.solve_triangular(hss.S[i], V, lower=True, trans="T").T
        hss.U[i] = hss.S[i] @ V
    _all_pairs_B(hss, M, 1)
    for k in range(2, Lv):
        nodes = [int(i) for i in tree.nodes_at_level(k)]
        off, Fh, Fmh = {}, {}, {}
        for i in nodes:
            kids = [int(c) for c in tree.children(i)]
            off[i] = (kids, np.concatenate([[0], np.cumsum([hss.rank[c] for c in kids])]).astype(int))
        def bold(i, j):
            ki, oi = off[i]
            kj, oj = off[j]
            Bb = np.zeros((oi[-1], oj[-1]))
            for a, ca in enumerate(ki):
                for bb, cb in enumerate(kj):
                    if ca != cb:
                        Bb[oi[a]:oi[a + 1], oj[bb]:oj[bb + 1]] = hss.B[(ca, cb)]
            return Bb
        for i in nodes:
            Bb = bold(i, i)
            hss.Bbold[i] = Bb
            Fh[i], Fmh[i] = _sym_power(Bb, 0.5), _sym_power(Bb, -0.5)
        for i in nodes:
            blocks = [Fmh[i] @ bold(i, j) @ Fmh[j] for j in nodes if j != i]
            E = np.hstack(blocks) if blocks else np.zeros((off[i][1][-1], 0))
            kk, Vb = _principal_basis(E, r)
            if keep:
                hss.target[i] = E
            kids, oi = off[i]
            b, e = tree.begin[i], tree.end[i]
            PhiStack = np.zeros((oi[-1], e - b))
            for a, c in enumerate(kids):
                PhiStack[oi[a]:oi[a + 1], tree.begin[c] - b:tree.end[c] - b] = hss.Phi[c]
            hss.Fhalf[i] = Fh[i]
            hss.Vbar[i] = Vb
            hss.rank[i] = kk
            hss.Phi[i] = Vb.T @ Fmh[i] @ PhiStack
            hss.R[i] = Fh[i] @ Vb
        _all_pairs_B(hss, M, k)
    return hss


def _all_pairs_B(hss: HSS, M: np.ndarray, k: int) -> None:
    """B_ij = Phi_i M_ij Phi_j^T for every i != j in lvl(k) (Eq. bij_hss)."""
    tree = hss.tree
    nodes = list(tree.nodes_at_level(k))
    for i in nodes:
        bi, ei = tree.begin[i], tree.end[i]
        left = hss.Phi[i] @ M[bi:ei, :]
        for j in nodes:
            if i == j:
                continue
            bj, ej = tree.begin[j], tree.end[j]
            hss.B[(i, j)] = left[:, bj:ej] @ hss.Phi[j].T


def explicit_U(hss: HSS, i: int) -> np.ndarray:
    """Full basis of node i, U_i = diag(U_children) R_i (Eq. nested)."""
    tree = hss.tree
    if i in hss.U:
        return hss.U[i]
    kids = [int(c) for c in tree.children(i)]
    blocks = [explicit_U(hss, c) for c in kids]
    Dg = sla.block_diag(*blocks)
    return Dg @ hss.R[i]


def assemble_dense(hss: HSS) -> np.ndarray:
    """Dense HSS matrix from {A_ii, U_i, R_i, B_ij (siblings)} (Sec. 2, HSS representation)."""
    tree = hss.tree
    n = tree.n
    H = np.zeros((n, n))
    for i, Dii in hss.D.items():
        b, e = tree.begin[i], tree.end[i]
        H[b:e, b:e] = Dii
    cache = {}
    for (i, j), Bij in hss.siblings_B().items():
        for v in (i, j):
            if v not in cache:
                cache[v] = explicit_U(hss, v)
        bi, ei, bj, ej = tree.begin[i], tree.end[i], tree.begin[j], tree.end[j]
        H[bi:ei, bj:ej] = cache[i] @ Bij @ cache[j].T
    return H
