"""GPU parity for the Rotne-Prager-Yamakawa tensor kernel (Sec. 6; three unknowns per
point): tree over unknowns, H^2 skeletons and products against the oracle's H^2 and the
dense matrix, SPD-HSS against the oracle's construction (leaf pair products with many
and with few sketch columns, i.e. both near-field kernels), ULV, PCG, the FP32 product."""
import numpy as np
import pytest

from oracle import h2 as OH
from oracle import kernels as OK
from oracle import pcg as OP
from oracle import spdhss as OS
from oracle import tree as OT
from oracle import ulv as OU
from paper_2011_07632_gb300 import inputs

from gpu_util import need_gpu, rel

pytestmark = pytest.mark.gpu


def _points(n, where, seed):
    return inputs.ball(n, seed) if where == "ball" else inputs.sphere(n, seed)


def _pair(n, where, leaf, a, tol, seed=0):
    api = need_gpu()
    X = _points(n, where, seed)
    h = api.H2(X, "rpy", a, 0.0, leaf, tol)
    o = OT.expand_dofs(OT.build_tree(X, leaf), 3)
    oh = OH.build_h2(o, X, OK.RPY, a, 0.0, tol)
    return api, X, h, o, oh


def _unsort(Hs, perm):
    H = np.empty_like(Hs)
    H[np.ix_(perm, perm)] = Hs
    return H


@pytest.mark.parametrize("n,where,leaf,a,tol", [
    (1500, "ball", 64, 0.42, 1e-8),
    (1200, "sphere", 40, 0.29, 1e-6),
    (50, "ball", 64, 0.42, 1e-8),     # one leaf
    (1, "ball", 8, 0.29, 1e-8),       # one particle: (1/a) I
])
def test_rpy_tree_skeletons_and_matvec(n, where, leaf, a, tol):
    api, X, h, o, oh = _pair(n, where, leaf, a, tol)
    assert h.n == 3 * n and h.info()["n"] == 3 * n
    g = h.export_tree()
    np.testing.assert_array_equal(g["perm"], o.perm)
    np.testing.assert_array_equal(g["begin"], o.begin)
    np.testing.assert_array_equal(g["end"], o.end)
    off, idx = h.export_skeletons()
    for i in range(o.num_nodes):
        gs = idx[off[i]:off[i + 1]]
        assert len(gs) == len(oh.skel[i]) and np.array_equal(np.sort(gs), np.sort(oh.skel[i]))
    x = np.random.default_rng(1).standard_normal((3 * n, 3))
    y = h.matmul(x).cpu().numpy()
    assert rel(y, OH.matmul_original_order(oh, x)) < 1e-12
    A = OK.dense_matrix(OK.RPY, a, 0.0, X)
    assert rel(y, A @ x) < max(50 * tol, 1e-13)


@pytest.mark.parametrize("nrhs", [1, 5, 17, 64])
def test_rpy_matvec_column_counts(nrhs):
    api = need_gpu()
    X = inputs.ball(2000, 3)
    h = api.H2(X, "rpy", 0.42, 1e-3, 64, 1e-8)
    x = np.random.default_rng(nrhs).standard_normal((6000, nrhs))
    A = OK.dense_matrix(OK.RPY, 0.42, 1e-3, X)
    assert rel(h.matmul(x).cpu().numpy(), A @ x) < 1e-7
    if nrhs <= 16:
        assert rel(h.matmul_mixed(x).cpu().numpy(), A @ x) < 1e-5


@pytest.mark.parametrize("r,p", [(30, 10), (4, 10)])   # 40 and 14 sketch columns
def test_rpy_hss_ulv_pcg_match_oracle(r, p):
    n, a, leaf, tol = 1200, 0.42, 48, 1e-8
    api, X, h, o, oh = _pair(n, "ball", leaf, a, tol, seed=4)
    N = 3 * n
    Om = inputs.sketch(N, r + p, 2)
    hs = api.HSS(h, r, p, omega=Om)
    Hg = hs.matmul(np.eye(N)).cpu().numpy()
    M = OH.dense(oh)
    ohss = OS.build_spdhss(o, M, Om[o.perm], r)
    Ho = _unsort(OS.assemble_dense(ohss), o.perm)
    assert rel(Hg, Ho) < 1e-10
    u = api.ULV(hs)
    b = inputs.rhs_uniform(N, 2, 6)
    xs = u.solve(b).cpu().numpy()
    assert rel(xs, np.linalg.solve(Ho, b)) < 1e-9
    # PCG on the H^2 matrix, preconditioned by the ULV solve; the oracle runs the same
    # iteration with its own H^2 matrix and ULV factorization
    x, its, rr = api.pcg_solve(h, u, b, tol=1e-8)
    Mo = _unsort(M, o.perm)
    ou = OU.ULV(ohss)
    perm = o.perm
    for c in range(2):
        def apply_m(v):
            out = np.empty_like(v)
            out[perm] = ou.solve(v[perm])
            return out
        xo, ito, _ = OP.pcg(lambda v: Mo @ v, apply_m, b[:, c], 1e-8, 3000)
        assert abs(int(its[c]) - int(ito[0])) <= 1
        assert rel(x[:, c], xo[:, 0]) < 1e-6
    assert np.all(rr <= 1e-8)


def test_rpy_large_sampled_rows():
    """100,000 particles in the ball (300,000 unknowns), a = 0.29, leaf 400, tol 1e-8:
    sampled rows of the product against exact tensor sums."""
    api = need_gpu()
    n = 100_000
    X = inputs.ball(n, 0)
    h = api.H2(X, "rpy", 0.29, 0.0, 400, 1e-8)
    x = inputs.rhs(3 * n, 2, 1)
    y = h.matmul(x).cpu().numpy()
    rows = np.random.default_rng(0).choice(3 * n, 24, replace=False)
    Xu, cu = OK.unknowns(OK.RPY, X)
    ye = np.vstack([OK.kernel_block(OK.RPY, 0.29, Xu[[q]], Xu, cu[[q]], cu) @ x for q in rows])
    assert np.abs(y[rows] - ye).max() / np.abs(ye).max() < 1e-7


def test_unpreconditioned_cg_matches_oracle():
    """ulv = None: plain CG on the H^2 matrix, against the oracle's iteration with the
    identity preconditioner."""
    api = need_gpu()
    X = inputs.ball(900, 8)
    h = api.H2(X, "rpy", 0.42, 0.0, 64, 1e-8)
    b = inputs.rhs_uniform(h.n, 2, 3)
    x, its, rr = api.pcg_solve(h, None, b, tol=1e-6)
    assert np.all(rr <= 1e-6)
    o = OT.expand_dofs(OT.build_tree(X, 64), 3)
    Mo = _unsort(OH.dense(OH.build_h2(o, X, OK.RPY, 0.42, 0.0, 1e-8)), o.perm)
    xo, ito, _ = OP.pcg(lambda v: Mo @ v, lambda v: v.copy(), b, 1e-6, 3000)
    # plain CG over ~170 iterations (kappa ~ 2800) loses orthogonality at a rate set by
    # rounding: the same iteration takes 166/169 steps in extended precision and 175/179
    # in numpy FP64, so the counts agree to a few percent, not to one step
    assert np.all(np.abs(its - ito) <= np.maximum(1, 0.05 * ito))
    assert rel(x, xo) < 1e-5
