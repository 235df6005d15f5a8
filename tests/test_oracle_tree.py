"""Pins of the oracle cluster tree and admissibility lists (Sec. 2, Sec. 5.1, Sec. 6)."""
import numpy as np
import pytest

from oracle import tree as T
from paper_2011_07632_gb300 import inputs


def test_morton_interleave_closed_form():
    # bit b of coordinate a sits at key bit b*d + (d-1-a): dim 0 most significant
    q = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [2, 0, 0], [3, 3, 3]], dtype=np.int64)
    k = T.morton_key(q)
    assert k.tolist() == [4, 2, 1, 32, 63]
    q2 = np.array([[1, 0], [0, 1], [1, 1], [2, 3]], dtype=np.int64)
    assert T.morton_key(q2).tolist() == [2, 1, 3, 0b1101]


def test_quantize_grid_points():
    # points on the corners of the unit cube map to cells 0 and 2^B - 1
    X = np.array([[0.0, 0.0, 0.0], [1.0, 1.0, 1.0], [0.5, 0.25, 1.0]])
    q, lo, w = T.quantize(X)
    B = 21
    assert w == 1.0
    assert q[0].tolist() == [0, 0, 0]
    assert q[1].tolist() == [2 ** B - 1] * 3
    assert q[2].tolist() == [2 ** (B - 1), 2 ** (B - 2), 2 ** B - 1]


def _check_partition(tr):
    for t in range(tr.D + 1):
        nodes = list(tr.nodes_at_depth(t))
        b = tr.begin[nodes]
        e = tr.end[nodes]
        assert b[0] == 0 and e[-1] == tr.n
        assert np.all(b[1:] == e[:-1]) and np.all(e > b)
    for i in range(1, tr.num_nodes):
        p = tr.parent[i]
        assert tr.begin[p] <= tr.begin[i] and tr.end[i] <= tr.end[p]
    for i in range(tr.num_nodes):
        kids = tr.children(i)
        if len(kids):
            assert tr.begin[kids[0]] == tr.begin[i] and tr.end[kids[-1]] == tr.end[i]


@pytest.mark.parametrize("n,dim,leaf", [(4096, 3, 64), (3000, 2, 32), (500, 3, 16), (1, 3, 8), (7, 2, 8)])
def test_tree_invariants(n, dim, leaf):
    X = inputs.uniform_cube(n, dim, 0)
    tr = T.build_tree(X, leaf)
    q, _, _ = T.quantize(X)
    key = T.morton_key(q)
    sk = key[tr.perm]
    assert np.all(sk[1:] >= sk[:-1])
    # stable: equal keys keep the original order
    eq = sk[1:] == sk[:-1]
    assert np.all(tr.perm[1:][eq] > tr.perm[:-1][eq])
    _check_partition(tr)
    for i in tr.nodes_at_depth(tr.D):
        assert tr.size(i) <= leaf
    # a node with children either holds more than leaf points, or is a padded copy (one child,
    # same range and cell)
    for i in range(tr.num_nodes):
        kids = tr.children(i)
        if len(kids) == 1 and tr.begin[kids[0]] == tr.begin[i] and tr.end[kids[0]] == tr.end[i] \
                and tr.size(i) <= leaf:
            assert np.all(tr.cell_lo[kids[0]] == tr.cell_lo[i])
        elif len(kids):
            assert tr.size(i) > leaf


def _brute_lists(tr):
    near, far = {}, {}
    for t in range(1, tr.D + 1):
        nodes = list(tr.nodes_at_depth(t))
        for i in nodes:
            pi = tr.parent[i]
            near[i] = [j for j in nodes if not T.admissible(tr.cell_lo[i], tr.cell_hi[i], tr.cell_lo[j], tr.cell_hi[j])]
            far[i] = [j for j in nodes
                      if T.admissible(tr.cell_lo[i], tr.cell_hi[i], tr.cell_lo[j], tr.cell_hi[j])
                      and not T.admissible(tr.cell_lo[pi], tr.cell_hi[pi], tr.cell_lo[tr.parent[j]], tr.cell_hi[tr.parent[j]])]
    return near, far


@pytest.mark.parametrize("n,dim,leaf", [(4096, 3, 64), (2000, 2, 16), (300, 3, 8)])
def test_lists_brute_force(n, dim, leaf):
    tr = T.build_tree(inputs.uniform_cube(n, dim, 1), leaf)
    near, far = _brute_lists(tr)
    for i in near:
        assert tr.near(i).tolist() == near[i]
        assert tr.far(i).tolist() == far[i]


@pytest.mark.parametrize("n,dim,leaf", [(2048, 3, 32), (1500, 2, 16)])
def test_blocks_cover_matrix_once(n, dim, leaf):
    """Every pair of leaf-depth nodes is a near pair or lies under exactly one Type-3 pair."""
    tr = T.build_tree(inputs.uniform_cube(n, dim, 2), leaf)
    leaves = list(tr.nodes_at_depth(tr.D))
    anc = {i: [i] for i in leaves}
    for i in leaves:
        while tr.parent[anc[i][-1]] >= 0:
            anc[i].append(int(tr.parent[anc[i][-1]]))
    farset = {(int(i), int(j)) for i in range(tr.num_nodes) for j in tr.far(i)}
    nearset = {(int(i), int(j)) for i in leaves for j in tr.near(i)}
    for i in leaves:
        for j in leaves:
            c = int((i, j) in nearset)
            for a, b in zip(anc[i], anc[j]):
                c += int((a, b) in farset)
            assert c == 1, (i, j)


def test_regular_grid_interaction_counts():
    """Perfect octree on an 8x8x8 grid: interior near lists have 27 cells, interaction
    lists 6^3 - 3^3 = 189 cells (Sec. 5.1, Type-3 blocks)."""
    g = (np.arange(8) + 0.5) / 8.0
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    tr = T.build_tree(X, 1)
    assert tr.D == 3 and tr.num_nodes == 1 + 8 + 64 + 512
    counts_near = [len(tr.near(i)) for i in tr.nodes_at_depth(3)]
    counts_far = [len(tr.far(i)) for i in tr.nodes_at_depth(3)]
    assert max(counts_near) == 27 and min(counts_near) == 8
    assert max(counts_far) == 189
    # depth 1: all 8 cells are mutually adjacent: no Type-3 pair
    assert all(len(tr.far(i)) == 0 for i in tr.nodes_at_depth(1))


def test_expand_dofs_keeps_particles_together():
    """Three unknowns per point: the permutation of unknowns is a permutation, every node
    range covers whole particles, and sorted unknown 3s + c is component c of the point
    the point tree puts at position s."""
    X = inputs.uniform_cube(500, 3, 11)
    t = T.build_tree(X, 16)
    u = T.expand_dofs(t, 3)
    assert u.n == 1500 and u.dofs == 3
    assert np.array_equal(np.sort(u.perm), np.arange(1500))
    assert np.array_equal(u.perm[0::3] // 3, t.perm) and np.all(u.perm % 3 == np.tile([0, 1, 2], 500))
    assert np.array_equal(u.begin, 3 * t.begin) and np.array_equal(u.end, 3 * t.end)
    for d in range(u.D + 1):
        nodes = list(u.nodes_at_depth(d))
        assert u.begin[nodes[0]] == 0 and u.end[nodes[-1]] == 1500
        assert np.array_equal(u.end[nodes[:-1]], u.begin[nodes[1:]])
    assert T.expand_dofs(t, 1) is t
