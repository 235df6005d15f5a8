"""GPU parity: ULV solve and PCG (Sec. 6.2) against the oracle."""
import numpy as np
import pytest

from oracle import h2 as OH
from oracle import kernels as OK
from oracle import pcg as OP
from oracle import spdhss as OS
from oracle import tree as OT
from oracle import ulv as OU
from paper_2011_07632_gb300 import inputs, native

from gpu_util import need_gpu, rel

pytestmark = pytest.mark.gpu


def unsort_vec(xs, perm):
    x = np.empty_like(xs)
    x[perm] = xs
    return x


def setup(n, dim, leaf, kind, ell, sigma, tol, r, seed=0):
    api = need_gpu()
    X = inputs.uniform_cube(n, dim, seed)
    Om = inputs.sketch(n, r + 10, 2)
    h = api.H2(X, kind, ell, sigma, leaf, tol)
    hs = api.HSS(h, r, 10, omega=Om)
    u = api.ULV(hs)
    tr = OT.build_tree(X, leaf)
    oh = OH.build_h2(tr, X, OK.NAMES[kind], ell, sigma, tol)
    Mh = OH.dense(oh)                              # oracle H^2 matrix, tree order
    ohss = OS.build_spdhss(tr, Mh, Om[tr.perm], r)
    return api, X, h, hs, u, tr, Mh, ohss


@pytest.mark.parametrize("n,dim,leaf,kind,ell,sigma,r", [
    (4096, 3, 64, "exp", 1.0, 1e-2, 50),
    (2048, 2, 32, "matern32", 0.2, 1e-3, 20),
    (1000, 3, 100, "gauss", 0.3, 1e-2, 150),
    (300, 3, 400, "exp", 1.0, 1e-2, 10),
])
def test_ulv_solve_matches_oracle(n, dim, leaf, kind, ell, sigma, r):
    api, X, h, hs, u, tr, Mh, ohss = setup(n, dim, leaf, kind, ell, sigma, 1e-8, r)
    b = inputs.rhs(n, 3, 1)
    x = u.solve(b).cpu().numpy()
    Ho = OS.assemble_dense(ohss)
    xo = unsort_vec(OU.dense_solve(Ho, b[tr.perm]), tr.perm)
    lam = np.linalg.eigvalsh(Ho)
    kappa = lam.max() / lam.min()
    assert rel(x, xo) < max(1e-12, 1e-10 * kappa)
    # the ULV solve inverts the HSS matrix it factored
    Hx = hs.matmul(x).cpu().numpy()
    assert rel(Hx, b) < 1e-11


def test_pcg_matches_oracle_iterations():
    n, r = 4096, 50
    api, X, h, hs, u, tr, Mh, ohss = setup(n, 3, 64, "exp", 1.0, 1e-2, 1e-8, r)
    b = inputs.rhs(n, 1, 1)
    x, it, rr = api.pcg_solve(h, u, b, tol=1e-6, maxit=3000)
    ou = OU.ULV(ohss)
    xo, ito, rro = OP.pcg(lambda v: Mh @ v, ou.solve, b[tr.perm], 1e-6, 3000)
    assert abs(int(it[0]) - int(ito[0])) <= 1
    assert rr[0] <= 1e-6
    # residual of the returned solution with the oracle's H^2 matrix
    xs = x.cpu().numpy()[tr.perm]
    assert np.linalg.norm(b[tr.perm] - Mh @ xs) / np.linalg.norm(b) <= 1.01e-6


def test_pcg_tight_tolerance_vs_dense_solve():
    """PCG to relres 1e-10 (above kappa * eps for this system) against a dense solve of the
    same H^2 matrix: the error is bounded by kappa * relres."""
    n, r = 4096, 50
    api, X, h, hs, u, tr, Mh, ohss = setup(n, 3, 64, "exp", 1.0, 1e-2, 1e-8, r)
    b = inputs.rhs(n, 1, 1)
    x, it, rr = api.pcg_solve(h, u, b, tol=1e-10, maxit=3000, raise_on_no_convergence=True)
    assert rr[0] <= 1e-10
    xs = x.cpu().numpy()[tr.perm]
    xd = np.linalg.solve(Mh, b[tr.perm])
    lam = np.linalg.eigvalsh(Mh)
    kappa = lam.max() / lam.min()
    assert rel(xs, xd) <= 2.0 * kappa * 1e-10
    assert rel(xs, xd) < 1e-8
    A = OK.dense_matrix(OK.EXP, 1.0, 1e-2, X)
    xa = np.linalg.solve(A, b)
    assert rel(x.cpu().numpy(), xa) < 1e-5


def test_pcg_multiple_rhs_independent_and_host_buffers():
    api = need_gpu()
    n = 3000
    X = inputs.uniform_cube(n, 3, 7)
    h = api.H2(X, "matern32", 0.1, 1e-3, 64, 1e-8)
    hs = api.HSS(h, 30, 10, seed=5)
    u = api.ULV(hs)
    B = inputs.rhs(n, 4, 9)
    xall, itall, rrall = api.pcg_solve(h, u, B, tol=1e-6)
    for c in range(4):
        xc, itc, rrc = api.pcg_solve(h, u, B[:, c], tol=1e-6)
        assert int(itc[0]) == int(itall[c])
        assert rel(xc.cpu().numpy()[:, 0], xall.cpu().numpy()[:, c]) < 1e-12
    # host buffers in and out (end-to-end path): same answer
    xh, ith, rrh = api.pcg_solve(h, u, np.asfortranarray(B), tol=1e-6)
    assert not xh.is_cuda
    assert rel(xh.numpy(), xall.cpu().numpy()) < 1e-14
    assert np.all(rrall <= 1e-6)


def test_pcg_reports_no_convergence():
    api = need_gpu()
    n = 2000
    X = inputs.uniform_cube(n, 3, 8)
    h = api.H2(X, "exp", 1.0, 1e-3, 64, 1e-8)
    hs = api.HSS(h, 5, 10, seed=1)
    u = api.ULV(hs)
    b = inputs.rhs(n, 1, 2)
    x, it, rr = api.pcg_solve(h, u, b, tol=1e-10, maxit=3)
    assert it[0] == 3 and rr[0] > 1e-10
    with pytest.raises(native.SpdhssError) as e:
        api.pcg_solve(h, u, b, tol=1e-10, maxit=3, raise_on_no_convergence=True)
    assert e.value.status == native.NO_CONVERGENCE


def test_not_spd_is_reported():
    """A negative shift larger than the smallest kernel eigenvalue makes A indefinite? The
    API rejects a negative shift up front; an indefinite leaf block is met with points that
    coincide under a zero shift (singular A_ii): the leaf Cholesky reports NOT_SPD."""
    api = need_gpu()
    X = np.repeat(inputs.uniform_cube(50, 3, 1), 4, axis=0)   # every point four times
    h = api.H2(X, "gauss", 0.5, 0.0, 16, 1e-8)
    with pytest.raises(native.SpdhssError) as e:
        api.HSS(h, 8, 10, seed=1)
    assert e.value.status == native.NOT_SPD


@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("case", ["headline", "long"])
def test_pcg_graph_replay_is_identical(case, mixed, monkeypatch):
    """Steady PCG iterations replay a captured CUDA graph of the same launches; with the
    graphs off (SPDHSS_PCG_GRAPHS=0) every iteration is launched directly.  Iteration
    counts, residuals and solutions are bit-identical, through residual replacements,
    restarts and (mixed) the FP64 refreshes every 50 iterations."""
    api = need_gpu()
    if case == "headline":
        n, kind, ell, sigma, r, nrhs = 4096, "exp", 1.0, 1e-2, 50, 3
    else:
        n, kind, ell, sigma, r, nrhs = 3000, "gauss", 0.2, 1e-4, 10, 2
    X = inputs.uniform_cube(n, 3, 0)
    h = api.H2(X, kind, ell, sigma, 64, 1e-8)
    u = api.ULV(api.HSS(h, r, 10, omega=inputs.sketch(n, r + 10, 2)))
    b = inputs.rhs(n, nrhs, 1)
    import torch
    st = torch.cuda.Stream()   # graphs are captured on the caller's stream (not the legacy one)
    x1, it1, rr1 = api.pcg_solve(h, u, b, tol=1e-6, mixed=mixed, stream=st)
    monkeypatch.setenv("SPDHSS_PCG_GRAPHS", "0")
    x0, it0, rr0 = api.pcg_solve(h, u, b, tol=1e-6, mixed=mixed, stream=st)
    torch.cuda.synchronize()
    assert np.array_equal(np.asarray(it1), np.asarray(it0))
    assert np.array_equal(np.asarray(rr1), np.asarray(rr0))
    assert np.array_equal(x1.cpu().numpy(), x0.cpu().numpy())
    assert int(np.max(it1)) > 3
