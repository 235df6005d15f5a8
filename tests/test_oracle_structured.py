"""Oracle: Alg. 5.3 on the H^2 matrix without its dense form (oracle/structured.py),
pinned against the dense forms and the quadratic construction at sizes where those exist:
the H^2 product against dense(H^2), the blockwise samples against Eq. Yk on the dense
matrix, the HSS product against the assembled HSS, and the whole construction against the
quadratic oracle on the same H^2 matrix and sketch (they differ only in how B_ij is
obtained: the recursion / Type-3 identities against Phi_i M_ij Phi_j^T)."""
import numpy as np
import pytest

from oracle import h2 as OH
from oracle import kernels as OK
from oracle import spdhss as OS
from oracle import structured as SO
from oracle import tree as OT
from paper_2011_07632_gb300 import inputs


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [(1500, 3, 32, "exp", 1.0, 1e-2, 20), (2000, 2, 40, "matern32", 0.2, 1e-3, 16),
         (1200, 3, 24, "gauss", 0.3, 1e-3, 12)]


@pytest.mark.parametrize("n,dim,leaf,kind,ell,sigma,r", CASES)
def test_structured_construction_equals_the_quadratic_one(n, dim, leaf, kind, ell, sigma, r):
    X = inputs.uniform_cube(n, dim, 3)
    Om = inputs.sketch(n, r + 10, 4)
    tr = OT.build_tree(X, leaf)
    h = OH.build_h2(tr, X, OK.NAMES[kind], ell, sigma, 1e-8)
    M = OH.dense(h)
    x = inputs.rhs(n, 3, 5)[tr.perm]
    assert rel(SO.h2_matvec(h, x), M @ x) < 1e-13
    Ys = SO.sample_products_h2(h, Om[tr.perm])
    Yd = OS.sample_products(tr, M, Om[tr.perm])
    for k in Yd:
        assert rel(Ys[k], Yd[k]) < 1e-13
    hs = SO.build_spdhss_h2(h, Om[tr.perm], r)
    hq = OS.build_spdhss(tr, M, Om[tr.perm], r)
    Hs = OS.assemble_dense(hs)
    assert rel(Hs, OS.assemble_dense(hq)) < 1e-10
    assert rel(SO.hss_matvec(hs, x), Hs @ x) < 1e-13
    assert np.linalg.eigvalsh(0.5 * (Hs + Hs.T)).min() > 0.0


def test_structured_full_rank_is_the_matrix():
    """Full rank (sketch wider than every block row): the HSS matrix equals the H^2 one."""
    n = 600
    X = inputs.uniform_cube(n, 3, 8)
    tr = OT.build_tree(X, 40)
    h = OH.build_h2(tr, X, OK.EXP, 0.5, 1e-2, 1e-8)
    hs = SO.build_spdhss_h2(h, inputs.sketch(n, n + 10, 9)[tr.perm], n)
    assert rel(OS.assemble_dense(hs), OH.dense(h)) < 1e-12
