"""Pins of the oracle's Rotne-Prager-Yamakawa kernel (Sec. 6) and of its H^2 form.

The tensor is pinned by facts that do not come from its own formula: the two branches
meet at |r| = 2a and the overlap branch tends to the self term (1/a) I as r -> 0; both
branches are divergence-free (checked by central differences); the far branch is the
Oseen tensor 3/(4|r|)(I + r r^T/|r|^2) plus (a^2/3) times its Laplacian (central
differences again); the matrix of any configuration, overlapping particles included, is
symmetric positive definite."""
import numpy as np
import pytest

from oracle import h2 as H
from oracle import kernels as K
from oracle import tree as T
from paper_2011_07632_gb300 import inputs


def _dirs(m, seed):
    v = np.random.default_rng(seed).standard_normal((m, 3))
    return v / np.linalg.norm(v, axis=1)[:, None]


@pytest.mark.parametrize("a", [0.29, 0.42, 1.7])
def test_branches_meet_at_contact_and_at_zero(a):
    u = _dirs(20, 1)
    lo = K.rpy_tensor(a, u * (2 * a) * (1 - 1e-10))
    hi = K.rpy_tensor(a, u * (2 * a) * (1 + 1e-10))
    assert np.abs(lo - hi).max() < 1e-8 / a
    tiny = K.rpy_tensor(a, u * 1e-12 * a)
    np.testing.assert_allclose(tiny, np.broadcast_to(np.eye(3) / a, tiny.shape), atol=1e-10 / a)
    np.testing.assert_array_equal(K.rpy_tensor(a, np.zeros((1, 3)))[0], np.eye(3) / a)


def _fd_grad(f, r, h):
    """d f / d r_j for every j by central differences (f: (m, 3) -> (m, 3, 3))."""
    out = []
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        out.append((f(r + e) - f(r - e)) / (2 * h))
    return np.stack(out, axis=-1)   # (m, 3, 3, 3): [.., i, k, j]


@pytest.mark.parametrize("scale", [0.4, 1.3, 3.0, 7.0])   # |r| / a: overlap and far branches
def test_divergence_free(scale):
    a = 0.42
    r = _dirs(16, 2) * scale * a
    g = _fd_grad(lambda x: K.rpy_tensor(a, x), r, 1e-5 * a)
    div = np.einsum("mijj->mi", g)          # sum_j d K_ij / d r_j
    assert np.abs(div).max() < 1e-7 / (a * a)


def _oseen(r):
    d = np.linalg.norm(r, axis=1)[:, None, None]
    rr = r[:, :, None] * r[:, None, :] / (d * d)
    return 3.0 / (4.0 * d) * (np.eye(3) + rr)


def test_far_branch_is_oseen_plus_its_laplacian():
    a = 0.29
    r = _dirs(12, 3) * np.linspace(2.1, 9.0, 12)[:, None] * a
    h = 1e-3 * a
    lap = np.zeros((len(r), 3, 3))
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        lap += (_oseen(r + e) - 2 * _oseen(r) + _oseen(r - e)) / (h * h)
    want = _oseen(r) + a * a / 3.0 * lap
    got = K.rpy_tensor(a, r)
    assert np.abs(got - want).max() < 1e-5 * np.abs(got).max()


@pytest.mark.parametrize("a,where", [(0.42, "ball"), (0.29, "sphere"), (0.8, "ball")])
def test_matrix_symmetric_positive_definite(a, where):
    X = inputs.ball(300, 5) if where == "ball" else inputs.sphere(300, 5)
    A = K.dense_matrix(K.RPY, a, 0.0, X)
    assert A.shape == (900, 900)
    assert np.array_equal(A, A.T)
    d = np.sqrt(((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))
    assert np.any((d > 0) & (d < 2 * a))    # overlapping particles are present
    assert np.linalg.eigvalsh(A).min() > 0.0
    # unknown 3p + c is component c of point p
    np.testing.assert_array_equal(A[3 * 4:3 * 5, 3 * 9:3 * 10], K.rpy_tensor(a, X[4:5] - X[9:10])[0])


def test_rpy_h2_to_tolerance():
    X = inputs.ball(700, 6)
    a = 0.42
    tr = T.expand_dofs(T.build_tree(X, 40), 3)
    h = H.build_h2(tr, X, K.RPY, a, 0.0, 1e-8)
    A = K.dense_matrix(K.RPY, a, 0.0, X)[np.ix_(tr.perm, tr.perm)]
    assert tr.n == 2100 and tr.end[0] == 2100
    ranks = [h.rank(i) for i in range(1, tr.num_nodes)]
    assert max(ranks) > 0
    x = np.random.default_rng(0).standard_normal((2100, 3))
    err = np.linalg.norm(H.dense(h) @ x - A @ x) / np.linalg.norm(A @ x)
    assert err < 1e-7
    # full rank reproduces the matrix
    h0 = H.build_h2(tr, X, K.RPY, a, 0.0, 0.0)
    assert np.abs(H.dense(h0) - A).max() <= 1e-13 * np.abs(A).max()
