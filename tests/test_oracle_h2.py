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


def test_pivoting_on_the_r_factor_gives_the_same_ids():
    """The interpolative decomposition only depends on the proxy matrix through its Gram
    matrix: column-pivoted QR of M and of the triangular factor R of an unpivoted QR of M
    (M = QR) pick the same skeletons and the same |R_kk|, so the ID can be taken from a
    tall-skinny QR of the proxy rows followed by a small pivoted QR.  Checked on every
    node of a 3D exponential and a 2D Matern H^2 construction."""
    import scipy.linalg as sla
    for n, dim, leaf, kind, ell in ((2048, 3, 64, K.EXP, 1.0), (1500, 2, 32, K.MATERN32, 0.2)):
        X = inputs.uniform_cube(n, dim, 7)
        tr = T.build_tree(X, leaf)
        h = H.build_h2(tr, X, kind, ell, 0.0, 1e-8)
        Xs = X[tr.perm]
        checked = 0
        for t in range(tr.D, 0, -1):
            for i in tr.nodes_at_depth(t):
                cand = (np.arange(tr.begin[i], tr.end[i]) if t == tr.D
                        else np.concatenate([h.skel[c] for c in tr.children(i)]))
                P = H.node_proxies(tr, i)
                if len(P) == 0 or len(cand) == 0:
                    continue
                M = K.kernel_block(kind, ell, P, Xs[cand])
                R0 = sla.qr(M, mode="r")[0][:M.shape[1]]
                R2, p2 = sla.qr(R0, mode="r", pivoting=True)
                d = np.abs(np.diag(R2))
                k = int(np.argmax(d <= 1e-8 * d[0])) if np.any(d <= 1e-8 * d[0]) else len(d)
                assert k == h.rank(i)
                assert set(cand[p2[:k]]) == set(h.skel[i])
                checked += 1
        assert checked > 20
