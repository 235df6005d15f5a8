"""Oracle: proxy-point H^2 representation.  TEST INFRASTRUCTURE ONLY.

H^2 form of Sec. 5.1: dense near blocks A_ij (j not in F_i) at the leaf level, and
A_ij = U_i B_ij U_j^T for Type-3 pairs (j in F_i, par j not in F_par i) at every level,
with nested bases U_i = diag(U_children) R_i (Eq. nested).  The paper builds it with the
proxy point method (Sec. 6) to relative error 1e-8 but does not spell the method out;
the reading used here:

* the far field of node i lies outside the cube of half-width 3h around the centre c
  of its cell (half-width h): every point closer than one cell width is in near(i);
* proxy points P_i: T = 6 cube surfaces of half-width h_t = 3h + (H - 3h) (t/(T-1))^2,
  H = max-norm distance from c to the farthest face of the enclosing cube, each face
  carrying a q x q cell-centred grid (q = 8 in 3D; 4 edges of q = 32 points in 2D).
  The node has no far field (and gets an empty basis) iff its cell grown by one cell
  width covers the enclosing cube, an integer test on the cell;
* candidates: the node's points at a leaf, the children's skeleton points (children in
  order) above; row interpolative decomposition K(X_cand, P) ~= U K(X_skel, P) from a
  column-pivoted QR of K(P, X_cand), stopped when |R_kk| <= tol |R_00|;
  U = Pi [I; (R_11^{-1} R_12)^T], skeleton = candidates in pivot order;
* coupling B_ij = K(X_skel_i, X_skel_j) for Type-3 pairs (no shift: off-diagonal blocks).
* a vector-valued kernel (RPY, three unknowns per point) works on unknowns throughout:
  the tree counts unknowns (tree.expand_dofs), every proxy point gives one row per
  component (row 3t + c: component c of proxy point t), and the decomposition picks
  skeleton unknowns.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla

from . import kernels as K
from .tree import Tree, bits_per_dim

PROXY_SHELLS = 6
PROXY_GRID = {3: 8, 2: 32}


def proxy_points(c: np.ndarray, h: float, H: float) -> np.ndarray:
    """Proxy points around a cell of centre c and half-width h (reading above)."""
    dim = len(c)
    if not H > 3.0 * h:
        return np.zeros((0, dim))
    q = PROXY_GRID[dim]
    g = -1.0 + (2.0 * np.arange(q) + 1.0) / q
    out = []
    for t in range(PROXY_SHELLS):
        f = t / (PROXY_SHELLS - 1)
        ht = 3.0 * h + (H - 3.0 * h) * (f * f)
        for a in range(dim):
            others = [b for b in range(dim) if b != a]
            for sgn in (-1.0, 1.0):
                if dim == 3:
                    P = np.zeros((q * q, 3))
                    u = np.repeat(g, q)
                    v = np.tile(g, q)
                    P[:, others[0]] = c[others[0]] + u * ht
                    P[:, others[1]] = c[others[1]] + v * ht
                else:
                    P = np.zeros((q, 2))
                    P[:, others[0]] = c[others[0]] + g * ht
                P[:, a] = c[a] + sgn * ht
                out.append(P)
    return np.vstack(out)


def has_far_field(tree: Tree, i: int) -> bool:
    """Integer test: the cell grown by one cell width does not cover the enclosing cube."""
    wd = tree.width(i)
    top = 1 << bits_per_dim(tree.dim)
    return bool(np.any(tree.cell_lo[i] - wd > 0) or np.any(top - tree.cell_hi[i] - wd > 0))


def node_proxies(tree: Tree, i: int) -> np.ndarray:
    if not has_far_field(tree, i):
        return np.zeros((0, tree.dim))
    blo, side = tree.box(i)
    h = 0.5 * side
    c = blo + h
    H = float(np.max(np.maximum(c - tree.lo, tree.lo + tree.w - c)))
    return proxy_points(c, h, max(H, 3.0 * h * (1.0 + 1e-12)))


@dataclass
class H2:
    tree: Tree
    kind: int
    ell: float
    sigma: float
    Xs: np.ndarray          # points in sorted (tree) order (of every unknown for RPY)
    cs: np.ndarray          # component of every sorted unknown (None: scalar kernel)
    skel: list              # per node: indices into Xs (pivot order)
    U: list                 # per node: leaf basis (|I_i| x k_i) or transfer R_i (sum k_c x k_i)
    B: dict                 # (i, j) -> K(X_skel_i, X_skel_j) for Type-3 pairs

    def rank(self, i: int) -> int:
        return len(self.skel[i])


def build_h2(tree: Tree, X: np.ndarray, kind: int, ell: float, sigma: float, tol: float) -> H2:
    """Proxy-point H^2 (bottom-up ID of every node of depth >= 1)."""
    X = np.asarray(X, dtype=np.float64)
    k_u = tree.dofs
    Xs = X[tree.perm // k_u]
    cs = tree.perm % k_u if k_u > 1 else None
    sub = (lambda idx: cs[idx]) if k_u > 1 else (lambda idx: None)
    nn = tree.num_nodes
    skel = [np.zeros(0, np.int64) for _ in range(nn)]
    U = [np.zeros((0, 0)) for _ in range(nn)]
    for t in range(tree.D, 0, -1):
        for i in tree.nodes_at_depth(t):
            if t == tree.D:
                cand = np.arange(tree.begin[i], tree.end[i])
            else:
                cand = np.concatenate([skel[c] for c in tree.children(i)])
            P = node_proxies(tree, i)
            if len(P) == 0 or len(cand) == 0:
                skel[i] = np.zeros(0, np.int64)
                U[i] = np.zeros((len(cand), 0))
                continue
            cP = None
            if k_u > 1:
                P, cP = np.repeat(P, k_u, axis=0), np.tile(np.arange(k_u), len(P))
            M = K.kernel_block(kind, ell, P, Xs[cand], cP, sub(cand))   # |P| x |cand|
            # column-pivoted QR by LAPACK (dgeqp3), truncated at |R_kk| <= tol |R_00|
            R, piv = sla.qr(M, mode="r", pivoting=True)
            d = np.abs(np.diag(R))
            k = int(np.argmax(d <= tol * d[0])) if np.any(d <= tol * d[0]) else len(d)
            Ui = np.zeros((len(cand), k))
            Ui[piv[:k], :] = np.eye(k)
            if k < len(cand):
                T = sla.solve_triangular(R[:k, :k], R[:k, k:], lower=False)
                Ui[piv[k:], :] = T.T
            skel[i] = cand[piv[:k]]
            U[i] = Ui
    B = {}
    for i in range(nn):
        for j in tree.far(i):
            si, sj = skel[i], skel[int(j)]
            B[(i, int(j))] = K.kernel_block(kind, ell, Xs[si], Xs[sj], sub(si), sub(sj))
    return H2(tree, kind, ell, sigma, Xs, cs, skel, U, B)


def explicit_basis(h2: H2, i: int) -> np.ndarray:
    """The full basis of node i (|I_i| x k_i) from the nested form, Eq. nested."""
    tree = h2.tree
    if tree.depth(i) == tree.D:
        return h2.U[i]
    kids = tree.children(i)
    blocks = [explicit_basis(h2, int(c)) for c in kids]
    rows = sum(b.shape[0] for b in blocks)
    cols = sum(b.shape[1] for b in blocks)
    Dg = np.zeros((rows, cols))
    r0 = c0 = 0
    for b in blocks:
        Dg[r0:r0 + b.shape[0], c0:c0 + b.shape[1]] = b
        r0 += b.shape[0]
        c0 += b.shape[1]
    return Dg @ h2.U[i]


def dense(h2: H2) -> np.ndarray:
    """Dense matrix represented by the H^2 form, in sorted (tree) order, including sigma I."""
    tree = h2.tree
    n = tree.n
    A = np.zeros((n, n))
    for i in tree.nodes_at_depth(tree.D):
        for j in tree.near(i):
            bi, ei, bj, ej = tree.begin[i], tree.end[i], tree.begin[j], tree.end[j]
            ci = h2.cs[bi:ei] if h2.cs is not None else None
            cj = h2.cs[bj:ej] if h2.cs is not None else None
            A[bi:ei, bj:ej] = K.kernel_block(h2.kind, h2.ell, h2.Xs[bi:ei], h2.Xs[bj:ej], ci, cj)
    ub = {}
    for (i, j), Bij in h2.B.items():
        for v in (i, j):
            if v not in ub:
                ub[v] = explicit_basis(h2, v)
        bi, ei, bj, ej = tree.begin[i], tree.end[i], tree.begin[j], tree.end[j]
        A[bi:ei, bj:ej] = ub[i] @ Bij @ ub[j].T
    A[np.diag_indices_from(A)] += h2.sigma
    return A


def matmul_original_order(h2: H2, X: np.ndarray) -> np.ndarray:
    """Y = A_H2 X with X and Y in the original point order."""
    perm = h2.tree.perm
    Xs = X[perm]
    Ys = dense(h2) @ Xs
    Y = np.empty_like(Ys)
    Y[perm] = Ys
    return Y
