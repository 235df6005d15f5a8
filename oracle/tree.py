"""Oracle: cluster tree, permutation and admissibility lists.  TEST INFRASTRUCTURE ONLY.

Follows Sec. 2 (hierarchical index sets I_i, levels, lvl(k)) and the partitioning of
Sec. 6 (a 2^d-ary tree from recursively bisecting every dimension of a box enclosing
the points until boxes are small).  Readings for what the paper leaves open:

* enclosing box: the cube with lower corner lo = coordinate-wise min and side
  w = largest extent; integer cell q = floor((x - lo) * (2^B / w)) clamped to 2^B - 1,
  B = 21 in 3D and 31 in 2D.  One FP64 subtract and one multiply; all later logic is
  integer, so the tree is exact.
* split rule: a box is split iff it holds more than ``leaf_size`` points; empty children
  are dropped; children are ordered by their Morton child index.
* non-perfect trees (Sec. 2 assumes a perfect tree): every leaf shallower than the
  deepest leaf D is padded with a chain of single-child copies down to depth D, so every
  depth partitions I.  A padded copy keeps the cell of its source leaf.
* admissibility ("well separated", Sec. 5.1): cells are integer intervals on the finest
  grid; i and j are admissible iff the max-norm gap between them is at least the wider
  of the two cell widths.  For equal cells this is "not adjacent".
* near(i) = {j at the depth of i : not adm(i, j)} (includes i);
  far(i)  = {j : adm(i, j) and not adm(par i, par j)}  (Type-3 partners, Sec. 5.2.2).

HSS level k (k = 1 leaves ... L root) is depth D + 1 - k.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np


def bits_per_dim(dim: int) -> int:
    if dim == 3:
        return 21
    if dim == 2:
        return 31
    raise ValueError("dim must be 2 or 3")


def enclosing_cube(X: np.ndarray):
    """lo (per-dim min) and w (largest extent) of the enclosing cube (Sec. 6)."""
    lo = X.min(axis=0)
    w = float((X.max(axis=0) - lo).max())
    return lo, w


def quantize(X: np.ndarray):
    """Integer cell coordinates on the finest 2^B grid, shape (n, dim) int64."""
    n, dim = X.shape
    B = bits_per_dim(dim)
    lo, w = enclosing_cube(X)
    if w > 0.0:
        scale = float(2.0 ** B) / w
        q = np.floor((X - lo) * scale)
    else:
        q = np.zeros_like(X)
    q = np.clip(q, 0, 2 ** B - 1).astype(np.int64)
    return q, lo, w


def morton_key(q: np.ndarray) -> np.ndarray:
    """Interleave the bits of the integer cells; dim 0 is the most significant in a group."""
    n, dim = q.shape
    B = bits_per_dim(dim)
    key = np.zeros(n, dtype=np.uint64)
    for b in range(B - 1, -1, -1):
        for a in range(dim):
            key = (key << np.uint64(1)) | ((q[:, a] >> b) & 1).astype(np.uint64)
    return key


@dataclass
class Tree:
    n: int
    dim: int
    leaf_size: int
    lo: np.ndarray
    w: float
    perm: np.ndarray            # sorted position -> original index
    depth_off: np.ndarray       # nodes of depth t are [depth_off[t], depth_off[t+1])
    begin: np.ndarray           # point range [begin, end) in sorted order
    end: np.ndarray
    parent: np.ndarray          # -1 for the root
    child_off: np.ndarray       # children of node i are child_idx[child_off[i]:child_off[i+1]]
    child_idx: np.ndarray
    cell_lo: np.ndarray         # (nn, dim) int64, finest-grid interval [cell_lo, cell_hi)
    cell_hi: np.ndarray
    near_off: np.ndarray
    near_idx: np.ndarray
    far_off: np.ndarray
    far_idx: np.ndarray
    D: int = 0                  # depth of the leaf level
    dofs: int = 1               # unknowns per point (n, perm, begin, end count unknowns)

    @property
    def num_nodes(self) -> int:
        return len(self.begin)

    @property
    def L(self) -> int:
        """Number of levels: leaves are level 1, the root is level L = D + 1."""
        return self.D + 1

    def depth(self, i: int) -> int:
        return int(np.searchsorted(self.depth_off, i, side="right") - 1)

    def level(self, i: int) -> int:
        return self.D + 1 - self.depth(i)

    def nodes_at_depth(self, t: int) -> range:
        return range(int(self.depth_off[t]), int(self.depth_off[t + 1]))

    def nodes_at_level(self, k: int) -> range:
        return self.nodes_at_depth(self.D + 1 - k)

    def children(self, i: int) -> np.ndarray:
        return self.child_idx[self.child_off[i]:self.child_off[i + 1]]

    def near(self, i: int) -> np.ndarray:
        return self.near_idx[self.near_off[i]:self.near_off[i + 1]]

    def far(self, i: int) -> np.ndarray:
        return self.far_idx[self.far_off[i]:self.far_off[i + 1]]

    def size(self, i: int) -> int:
        return int(self.end[i] - self.begin[i])

    def width(self, i: int) -> int:
        return int(self.cell_hi[i, 0] - self.cell_lo[i, 0])

    def ancestor_at_depth(self, i: int, t: int) -> int:
        while self.depth(i) > t:
            i = int(self.parent[i])
        return i

    def lca_level(self, i: int, j: int) -> int:
        """HSS level of the lowest common ancestor of two nodes of equal depth."""
        while i != j:
            i = int(self.parent[i])
            j = int(self.parent[j])
        return self.level(i)

    def box(self, i: int):
        """Real-coordinate cell of node i: (lower corner, side)."""
        B = bits_per_dim(self.dim)
        h = self.w / float(2 ** B)
        return self.lo + self.cell_lo[i] * h, self.width(i) * h


def admissible(lo_i, hi_i, lo_j, hi_j) -> bool:
    """Max-norm gap between the cells is at least the wider cell width."""
    gap = np.maximum(0, np.maximum(lo_j - hi_i, lo_i - hi_j)).max()
    wi = int(hi_i[0] - lo_i[0])
    wj = int(hi_j[0] - lo_j[0])
    return bool(gap >= max(wi, wj))


def build_tree(X: np.ndarray, leaf_size: int) -> Tree:
    X = np.asarray(X, dtype=np.float64)
    n, dim = X.shape
    B = bits_per_dim(dim)
    q, lo, w = quantize(X)
    key = morton_key(q)
    perm = np.argsort(key, kind="stable")
    skey = key[perm]
    sq = q[perm]

    # genuine nodes by depth: (begin, end, parent_pos, is_leaf)
    levels = [[(0, n, -1)]]
    leaf_flags = []
    t = 0
    while True:
        cur = levels[t]
        flags = []
        nxt = []
        for pos, (b, e, _) in enumerate(cur):
            split = (e - b) > leaf_size and t < B
            flags.append(not split)
            if split:
                shift = np.uint64(dim * (B - t - 1))
                pref = skey[b:e] >> shift
                cuts = np.flatnonzero(pref[1:] != pref[:-1]) + 1
                bounds = [0] + cuts.tolist() + [e - b]
                for a in range(len(bounds) - 1):
                    nxt.append((b + bounds[a], b + bounds[a + 1], pos))
        leaf_flags.append(flags)
        if not nxt:
            break
        levels.append(nxt)
        t += 1
    D = len(levels) - 1

    # padded tree: per depth, the genuine nodes of that depth plus a copy of every leaf of
    # the depth above (genuine or itself a copy); entries are (begin, end, cell_lo, cell_hi, leafish)
    per_depth = []
    prev = []
    for t in range(D + 1):
        entries = []
        sh = B - t
        for (b, e, _), leaf in zip(levels[t], leaf_flags[t]):
            clo = (sq[b] >> sh) << sh
            entries.append((b, e, clo, clo + (1 << sh), leaf))
        for (b, e, clo, chi, leaf) in prev:
            if leaf:
                entries.append((b, e, clo, chi, True))
        entries.sort(key=lambda z: z[0])
        per_depth.append(entries)
        prev = entries

    depth_off = np.zeros(D + 2, dtype=np.int64)
    for t in range(D + 1):
        depth_off[t + 1] = depth_off[t] + len(per_depth[t])
    nn = int(depth_off[-1])
    begin = np.zeros(nn, np.int64)
    end = np.zeros(nn, np.int64)
    parent = -np.ones(nn, np.int64)
    cell_lo = np.zeros((nn, dim), np.int64)
    cell_hi = np.zeros((nn, dim), np.int64)
    for t in range(D + 1):
        for a, (b, e, clo, chi, _) in enumerate(per_depth[t]):
            g = int(depth_off[t]) + a
            begin[g], end[g] = b, e
            cell_lo[g], cell_hi[g] = clo, chi
    # parents: the node at depth t-1 whose range contains b
    for t in range(1, D + 1):
        pb = begin[depth_off[t - 1]:depth_off[t]]
        for g in range(int(depth_off[t]), int(depth_off[t + 1])):
            p = int(np.searchsorted(pb, begin[g], side="right") - 1)
            parent[g] = int(depth_off[t - 1]) + p
    counts = np.bincount(parent[parent >= 0], minlength=nn)
    child_off = np.zeros(nn + 1, np.int64)
    child_off[1:] = np.cumsum(counts)
    child_idx = np.zeros(int(child_off[-1]), np.int64)
    fill = child_off[:-1].copy()
    for g in range(nn):
        p = parent[g]
        if p >= 0:
            child_idx[fill[p]] = g
            fill[p] += 1

    tree = Tree(n=n, dim=dim, leaf_size=leaf_size, lo=lo, w=w, perm=perm.astype(np.int64),
                depth_off=depth_off, begin=begin, end=end, parent=parent,
                child_off=child_off, child_idx=child_idx, cell_lo=cell_lo, cell_hi=cell_hi,
                near_off=None, near_idx=None, far_off=None, far_idx=None, D=D)
    _build_lists(tree)
    return tree


def _build_lists(tree: Tree) -> None:
    nn = tree.num_nodes
    near = [[] for _ in range(nn)]
    far = [[] for _ in range(nn)]
    near[0] = [0]
    for t in range(1, tree.D + 1):
        for i in tree.nodes_at_depth(t):
            p = int(tree.parent[i])
            for pj in near[p]:
                for c in tree.children(pj):
                    c = int(c)
                    if admissible(tree.cell_lo[i], tree.cell_hi[i], tree.cell_lo[c], tree.cell_hi[c]):
                        far[i].append(c)
                    else:
                        near[i].append(c)
            near[i].sort()
            far[i].sort()
    for name, lists in (("near", near), ("far", far)):
        off = np.zeros(nn + 1, np.int64)
        off[1:] = np.cumsum([len(x) for x in lists])
        idx = np.array([v for x in lists for v in x], dtype=np.int64)
        setattr(tree, name + "_off", off)
        setattr(tree, name + "_idx", idx)


def expand_dofs(tree: Tree, k: int) -> Tree:
    """The same tree over k unknowns per point (a vector-valued kernel): unknown k*p + c is
    component c of point p, in sorted and in original order alike, so every index range
    and the permutation scale by k and the components of a point stay together."""
    if k == 1:
        return tree
    perm = (tree.perm[:, None] * k + np.arange(k)[None, :]).reshape(-1)
    return dataclasses.replace(tree, n=tree.n * k, perm=perm, begin=tree.begin * k,
                               end=tree.end * k, dofs=k)
