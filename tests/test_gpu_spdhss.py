"""GPU parity: SPD-HSS construction (Alg. 5.3) against the oracle's quadratic
construction on the same matrix and the same sketch; HSS properties at small n."""
import numpy as np
import pytest

from oracle import h2 as OH
from oracle import kernels as OK
from oracle import spdhss as OS
from oracle import tree as OT
from paper_2011_07632_gb300 import inputs

from gpu_util import need_gpu, rel

pytestmark = pytest.mark.gpu


def unsort(Hs, perm):
    H = np.empty_like(Hs)
    H[np.ix_(perm, perm)] = Hs
    return H


def gpu_dense(hs, n):
    return hs.matmul(np.eye(n)).cpu().numpy()


def oracle_dense(X, leaf, kind, ell, sigma, tol, Om, r):
    tr = OT.build_tree(X, leaf)
    if tol == 0.0:
        M = OK.dense_matrix(OK.NAMES[kind], ell, sigma, X[tr.perm])
    else:
        M = OH.dense(OH.build_h2(tr, X, OK.NAMES[kind], ell, sigma, tol))
    hss = OS.build_spdhss(tr, M, Om[tr.perm], r)
    return unsort(OS.assemble_dense(hss), tr.perm), unsort(M, tr.perm)


CASES = [
    # n, dim, leaf, kernel, ell, sigma, H2 tol, r
    (4096, 3, 64, "exp", 1.0, 1e-2, 1e-8, 50),
    (2048, 2, 32, "matern32", 0.2, 1e-3, 1e-8, 20),
    (1000, 3, 16, "gauss", 0.3, 1e-4, 1e-6, 8),
    (1500, 3, 40, "imq", 0.5, 1e-3, 1e-8, 30),
]


@pytest.mark.parametrize("n,dim,leaf,kind,ell,sigma,tol,r", CASES)
def test_hss_matches_oracle(n, dim, leaf, kind, ell, sigma, tol, r):
    api = need_gpu()
    X = inputs.uniform_cube(n, dim, 0)
    Om = inputs.sketch(n, r + 10, 2)
    h = api.H2(X, kind, ell, sigma, leaf, tol)
    hs = api.HSS(h, r, 10, omega=Om)
    Hg = gpu_dense(hs, n)
    Ho, M = oracle_dense(X, leaf, kind, ell, sigma, tol, Om, r)
    assert rel(Hg, Ho) < 1e-10


def test_full_rank_hss_equals_matrix():
    api = need_gpu()
    n = 600
    X = inputs.uniform_cube(n, 3, 4)
    Om = inputs.sketch(n, n + 10, 5)
    h = api.H2(X, "exp", 0.5, 1e-2, 32, 0.0)
    hs = api.HSS(h, n, 10, omega=Om)
    A = OK.dense_matrix(OK.EXP, 0.5, 1e-2, X)
    assert rel(gpu_dense(hs, n), A) < 1e-12


@pytest.mark.parametrize("kind,sigma,r", [("gauss", 1e-6, 4), ("matern32", 1e-5, 10)])
def test_gpu_hss_is_spd(kind, sigma, r):
    api = need_gpu()
    n = 512
    X = inputs.uniform_cube(n, 3, 6)
    h = api.H2(X, kind, 0.2, sigma, 16, 1e-8)
    hs = api.HSS(h, r, 10, seed=11)           # sketch drawn on the device
    Hg = gpu_dense(hs, n)
    Hg = 0.5 * (Hg + Hg.T)
    assert np.linalg.eigvalsh(Hg).min() > 0.0


def test_device_sketch_statistics():
    """With omega=None the library draws Omega from Philox4x32-10: the HSS it yields is
    an approximation of the same quality as with a host-drawn Gaussian sketch."""
    api = need_gpu()
    n = 4096
    X = inputs.uniform_cube(n, 3, 0)
    h = api.H2(X, "exp", 1.0, 1e-2, 64, 1e-8)
    A = OK.dense_matrix(OK.EXP, 1.0, 1e-2, X)
    e_dev = rel(gpu_dense(api.HSS(h, 50, 10, seed=3), n), A)
    e_host = rel(gpu_dense(api.HSS(h, 50, 10, omega=inputs.sketch(n, 60, 2)), n), A)
    assert e_dev < 3 * e_host and e_host < 3 * e_dev


@pytest.mark.parametrize("tau", [1e-1, 1e-2, 1e-5])
def test_tolerance_truncated_hss_matches_oracle(tau):
    """Tolerance-driven bases (spdhss_build_tol): the same truncation as the oracle's on
    the same matrix and sketch, and the result stays SPD."""
    api = need_gpu()
    n, dim, leaf, kind, ell, sigma, tol, r = 1500, 3, 40, "exp", 0.5, 1e-3, 1e-8, 40
    X = inputs.uniform_cube(n, dim, 3)
    Om = inputs.sketch(n, r + 10, 4)
    h = api.H2(X, kind, ell, sigma, leaf, tol)
    hs = api.HSS(h, r, 10, omega=Om, tol=tau)
    Hg = gpu_dense(hs, n)
    tr = OT.build_tree(X, leaf)
    M = OH.dense(OH.build_h2(tr, X, OK.NAMES[kind], ell, sigma, tol))
    hss = OS.build_spdhss(tr, M, Om[tr.perm], r, rtol=tau)
    Ho = unsort(OS.assemble_dense(hss), tr.perm)
    assert rel(Hg, Ho) < 1e-10
    assert hs.info()["max_rank"] == max(hss.rank.values())
    assert np.linalg.eigvalsh(0.5 * (Hg + Hg.T)).min() > 0.0


def test_rank_zero_gives_block_jacobi():
    """rank 0: the GPU SPD-HSS is the block diagonal of the leaf blocks and its ULV solve is
    the block-Jacobi solve."""
    api = need_gpu()
    n, leaf = 1200, 50
    X = inputs.uniform_cube(n, 3, 5)
    h = api.H2(X, "matern32", 0.3, 1e-2, leaf, 1e-8)
    hs = api.HSS(h, 0, 10, seed=1)
    Hg = gpu_dense(hs, n)
    tr = OT.build_tree(X, leaf)
    M = OK.dense_matrix(OK.NAMES["matern32"], 0.3, 1e-2, X[tr.perm])
    B = np.zeros_like(M)
    for i in tr.nodes_at_level(1):
        b, e = tr.begin[i], tr.end[i]
        B[b:e, b:e] = M[b:e, b:e]
    assert rel(Hg, unsort(B, tr.perm)) < 1e-13
    u = api.ULV(hs)
    rhs = inputs.rhs(n, 2, 6)
    x = u.solve(rhs).cpu().numpy()
    assert rel(Hg @ x, rhs) < 1e-11


def test_tolerance_driven_sketch_growth_matches_oracle():
    """spdhss_build_tol grows the sketch (first r + p columns, r doubling from 64) until the
    ranks fit: the same attempts and the same result as the oracle's growing construction."""
    api = need_gpu()
    n, dim, leaf, kind, ell, sigma, tol, cap, p = 3000, 3, 100, "matern32", 0.3, 1e-2, 1e-8, 300, 10
    tau = 1e-3                            # ranks up to 159: the sketch grows 64 -> 128 -> 256
    X = inputs.uniform_cube(n, dim, 7)
    Om = inputs.sketch(n, cap + p, 8)
    h = api.H2(X, kind, ell, sigma, leaf, tol)
    hs = api.HSS(h, cap, p, omega=Om, tol=tau)
    Hg = gpu_dense(hs, n)
    tr = OT.build_tree(X, leaf)
    M = OH.dense(OH.build_h2(tr, X, OK.NAMES[kind], ell, sigma, tol))
    ho = OS.build_spdhss_adaptive(tr, M, Om[tr.perm], cap, p, tau, r0=64)
    assert 64 < ho.sketch_rank < cap      # the sketch grew and stopped below the cap
    Ho = unsort(OS.assemble_dense(ho), tr.perm)
    assert rel(Hg, Ho) < 1e-10
    assert hs.info()["max_rank"] == max(ho.rank.values())
