"""GPU parity at a size the dense oracle cannot reach: the GPU's SPD-HSS construction and
PCG at n = 20,000 against the structured oracle (Alg. 5.3 on the oracle's own H^2 matrix,
no dense matrix; oracle/structured.py, pinned against the quadratic oracle at small n).
Compared: HSS products on random vectors, and PCG iteration counts with each side's own
preconditioner and product."""
import numpy as np
import pytest

from oracle import h2 as OH
from oracle import kernels as OK
from oracle import pcg as OP
from oracle import structured as SO
from oracle import tree as OT
from oracle import ulv as OU
from paper_2011_07632_gb300 import inputs

from gpu_util import need_gpu, rel

pytestmark = pytest.mark.gpu


def test_construction_and_pcg_at_n20000_against_the_structured_oracle():
    api = need_gpu()
    n, leaf, r = 20000, 64, 30
    X = inputs.uniform_cube(n, 3, 0)
    Om = inputs.sketch(n, r + 10, 2)
    h = api.H2(X, "exp", 1.0, 1e-2, leaf, 1e-8)
    hs = api.HSS(h, r, 10, omega=Om)
    u = api.ULV(hs)
    tr = OT.build_tree(X, leaf)
    oh = OH.build_h2(tr, X, OK.EXP, 1.0, 1e-2, 1e-8)
    ohs = SO.build_spdhss_h2(oh, Om[tr.perm], r)
    x = inputs.rhs(n, 4, 3)
    yg = hs.matmul(x).cpu().numpy()[tr.perm]
    yo = SO.hss_matvec(ohs, x[tr.perm])
    assert rel(yg, yo) < 1e-10
    b = inputs.rhs(n, 1, 1)
    _, it, rr = api.pcg_solve(h, u, b, tol=1e-6)
    A = SO.H2Apply(oh)
    _, ito, rro = OP.pcg(A, OU.ULV(ohs).solve, b[tr.perm], 1e-6, 3000)
    assert abs(int(it[0]) - int(ito[0])) <= 1 and rr[0] <= 1e-6 and rro[0] <= 1e-6
