"""GPU parity: cluster tree, permutation and lists bit-exact against the oracle; H^2
skeletons and products against the oracle's H^2 and the dense kernel matrix."""
import numpy as np
import pytest

from oracle import h2 as OH
from oracle import kernels as OK
from oracle import tree as OT
from paper_2011_07632_gb300 import inputs

from gpu_util import need_gpu, rel

pytestmark = pytest.mark.gpu

CASES = [(4096, 3, 64), (3000, 2, 32), (777, 3, 16), (1, 3, 8), (50, 2, 64), (2500, 3, 5)]


@pytest.mark.parametrize("n,dim,leaf", CASES)
def test_tree_bit_exact(n, dim, leaf):
    api = need_gpu()
    X = inputs.uniform_cube(n, dim, 0)
    h = api.H2(X, "exp", 1.0, 1e-2, leaf, 1e-8)
    g = h.export_tree()
    o = OT.build_tree(X, leaf)
    assert g["D"] == o.D
    np.testing.assert_array_equal(g["perm"], o.perm)
    np.testing.assert_array_equal(g["depth_off"], o.depth_off)
    for k in ("begin", "end", "parent", "cell_lo", "cell_hi", "near_off", "near_idx", "far_off",
              "far_idx"):
        np.testing.assert_array_equal(g[k], getattr(o, k), err_msg=k)


def test_tree_coincident_points():
    api = need_gpu()
    X = np.repeat(inputs.uniform_cube(40, 3, 5), 10, axis=0)   # 10 copies of every point
    h = api.H2(X, "gauss", 0.3, 1e-2, 4, 1e-8)
    g = h.export_tree()
    o = OT.build_tree(X, 4)
    np.testing.assert_array_equal(g["perm"], o.perm)
    np.testing.assert_array_equal(g["begin"], o.begin)
    np.testing.assert_array_equal(g["far_idx"], o.far_idx)


def _pair(n, dim, leaf, kind, ell, tol, seed=0, sigma=1e-2):
    api = need_gpu()
    X = inputs.uniform_cube(n, dim, seed)
    h = api.H2(X, kind, ell, sigma, leaf, tol)
    o = OT.build_tree(X, leaf)
    oh = OH.build_h2(o, X, OK.NAMES[kind], ell, sigma, tol)
    return api, X, h, o, oh


@pytest.mark.parametrize("n,dim,leaf,kind,ell,tol", [
    (4096, 3, 64, "exp", 1.0, 1e-8),
    (4096, 2, 32, "matern32", 0.2, 1e-8),
    (2048, 3, 32, "exp", 1.0, 1e-4),
    (3000, 2, 16, "gauss", 0.2, 1e-6),
])
def test_h2_skeletons_and_matvec(n, dim, leaf, kind, ell, tol):
    api, X, h, o, oh = _pair(n, dim, leaf, kind, ell, tol)
    off, idx = h.export_skeletons()
    same = 0
    for i in range(o.num_nodes):
        gs = idx[off[i]:off[i + 1]]
        if len(gs) == len(oh.skel[i]) and np.array_equal(np.sort(gs), np.sort(oh.skel[i])):
            same += 1
    assert same == o.num_nodes
    rng = np.random.default_rng(1)
    x = rng.standard_normal((n, 3))
    y = h.matmul(x).cpu().numpy()
    yo = OH.matmul_original_order(oh, x)
    assert rel(y, yo) < 1e-12
    A = OK.dense_matrix(OK.NAMES[kind], ell, 1e-2, X)
    assert rel(y, A @ x) < max(50 * tol, 1e-13)


def test_h2_full_rank_is_exact():
    api = need_gpu()
    X = inputs.uniform_cube(1500, 3, 2)
    h = api.H2(X, "gauss", 0.3, 1e-3, 32, 0.0)
    x = np.random.default_rng(2).standard_normal((1500, 2))
    A = OK.dense_matrix(OK.GAUSS, 0.3, 1e-3, X)
    assert rel(h.matmul(x).cpu().numpy(), A @ x) < 1e-13


@pytest.mark.parametrize("nrhs", [1, 5, 8, 17, 64, 70])
def test_h2_matvec_column_counts(nrhs):
    api = need_gpu()
    X = inputs.uniform_cube(3000, 3, 3)
    h = api.H2(X, "matern32", 0.1, 1e-3, 64, 1e-8)
    x = np.random.default_rng(nrhs).standard_normal((3000, nrhs))
    A = OK.dense_matrix(OK.MATERN32, 0.1, 1e-3, X)
    assert rel(h.matmul(x).cpu().numpy(), A @ x) < 1e-7


def test_h2_matvec_large_sampled_rows():
    """n = 200,000 Gaussian (ell = 0.1, shift 1e-4, leaf 128, tol 1e-8): sampled rows of
    the product against exact kernel sums."""
    api = need_gpu()
    n = 200_000
    X = inputs.uniform_cube(n, 3, 0)
    h = api.H2(X, "gauss", 0.1, 1e-4, 128, 1e-8)
    x = inputs.rhs(n, 2, 1)
    y = h.matmul(x).cpu().numpy()
    rows = np.random.default_rng(0).choice(n, 40, replace=False)
    K = OK.kernel_block(OK.GAUSS, 0.1, X[rows], X)
    ye = K @ x + 1e-4 * x[rows]
    err = np.abs(y[rows] - ye).max() / np.abs(ye).max()
    assert err < 1e-7


def test_h2_far_field_below_the_squares_underflow():
    """A Gaussian whose far-field values reach 1e-150 and below (n = 20,000 points of unit
    density in a ball, length scale 1, leaf 400): summed squares of such proxy entries
    underflow, which once made the ID's reflectors overflow (ranks of 1, every product
    entry non-finite).  Each node's proxy matrix is now scaled by a power of two before the
    ID, so the skeletons equal the oracle's (scaled LAPACK norms) and the product matches
    the oracle's H^2 product."""
    from oracle import structured as OSt
    api = need_gpu()
    n, leaf, ell = 20000, 400, 1.0
    X = inputs.ball(n, 0)
    h = api.H2(X, "gauss", ell, 1e-2, leaf, 1e-8)
    tr = OT.build_tree(X, leaf)
    oh = OH.build_h2(tr, X, OK.GAUSS, ell, 1e-2, 1e-8)
    off, idx = h.export_skeletons()
    for i in range(len(off) - 1):
        gs = np.sort(idx[off[i]:off[i + 1]])
        os_ = np.sort(np.asarray(oh.skel[i], dtype=np.int64)) if oh.skel[i] is not None else np.zeros(0, np.int64)
        assert np.array_equal(gs, os_), i
    x = np.random.default_rng(3).standard_normal((n, 2))
    y = h.matmul(x).cpu().numpy()
    assert np.isfinite(y).all()
    yo = np.empty_like(y)
    yo[tr.perm] = OSt.h2_matvec(oh, x[tr.perm])
    assert rel(y, yo) < 1e-12
    assert np.isfinite(h.matmul_mixed(x).cpu().numpy()).all()
