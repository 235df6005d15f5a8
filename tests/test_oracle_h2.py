"""Pins of the oracle proxy-point H^2 representation (Sec. 5.1, Sec. 6)."""
import numpy as np
import pytest

from oracle import h2 as H
from oracle import kernels as K
from oracle import tree as T
from paper_2011_07632_gb300 import inputs


def _setup(n, dim, leaf, kind, ell, tol, seed=0):
    X = inputs.uniform_cube(n, dim, seed)
    tr = T.build_tree(X, leaf)
    h = H.build_h2(tr, X, kind, ell, 1e-2, tol)
    A = K.dense_matrix(kind, ell, 1e-2, X[tr.perm])
    return tr, h, A


def test_full_rank_h2_is_exact():
    # tolerance 0: every ID keeps all candidates, so the H^2 form reproduces A
    tr, h, A = _setup(1500, 3, 32, K.GAUSS, 0.3, 0.0)
    Ah = H.dense(h)
    assert np.abs(Ah - A).max() <= 1e-13


@pytest.mark.parametrize("kind,ell", [(K.EXP, 1.0), (K.MATERN32, 0.2), (K.GAUSS, 0.2)])
def test_h2_matvec_to_tolerance_2d(kind, ell):
    tr, h, A = _setup(4096, 2, 32, kind, ell, 1e-8, seed=3)
    ranks = [h.rank(i) for i in tr.nodes_at_depth(tr.D - 1)]
    cands = [sum(h.rank(c) for c in tr.children(i)) for i in tr.nodes_at_depth(tr.D - 1)]
    assert sum(ranks) < sum(cands)          # truncation really happens
    x = np.random.default_rng(0).standard_normal((4096, 3))
    err = np.linalg.norm(H.dense(h) @ x - A @ x) / np.linalg.norm(A @ x)
    assert err < 1e-7


def test_h2_error_tracks_tolerance_3d():
    tr, h, A = _setup(2048, 3, 32, K.EXP, 1.0, 1e-4, seed=4)
    x = np.random.default_rng(1).standard_normal((2048, 2))
    err = np.linalg.norm(H.dense(h) @ x - A @ x) / np.linalg.norm(A @ x)
    assert 1e-9 < err < 1e-3


def test_id_structure_and_nesting():
    tr, h, A = _setup(2048, 3, 32, K.EXP, 1.0, 1e-6, seed=5)
    for i in range(1, tr.num_nodes):
        U = h.U[i]
        k = h.rank(i)
        if k == 0:
            continue
        # identity rows at the skeleton positions of the candidate list
        if tr.depth(i) == tr.D:
            cand = np.arange(tr.begin[i], tr.end[i])
        else:
            cand = np.concatenate([h.skel[c] for c in tr.children(i)])
        pos = [int(np.flatnonzero(cand == s)[0]) for s in h.skel[i]]
        assert np.array_equal(U[pos], np.eye(k))
        # skeleton points are points of the node
        assert np.all((h.skel[i] >= tr.begin[i]) & (h.skel[i] < tr.end[i]))


def test_proxy_points_lie_outside_near_field():
    tr, h, A = _setup(2048, 3, 32, K.EXP, 1.0, 1e-6, seed=6)
    for i in range(1, tr.num_nodes):
        P = H.node_proxies(tr, i)
        if len(P) == 0:
            assert not H.has_far_field(tr, i)
            continue
        assert len(P) == 6 * 6 * 64
        blo, side = tr.box(i)
        c = blo + side / 2
        dist = np.abs(P - c).max(axis=1)
        assert dist.min() >= 1.5 * side * (1 - 1e-12)
