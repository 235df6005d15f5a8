"""GPU parity for the fixed-rank iteration sweeps over the kernel parameter (Sec. 6.2, the
table of PCG iterations over l for the Matern-3/2, Gaussian and IMQ kernels): PCG iteration
counts with the SPD-HSS preconditioner (r > 0) and with block Jacobi (r = 0) against the
oracle on the same ball of points, shift 1e-2, the paper's PCG setting (right-hand side
uniform on [-0.5, 0.5], relres 1e-4, at most 3000 iterations).

The paper writes the kernels with a parameter l multiplying the distance (Matern) or the
squared distance (Gaussian, IMQ); the library's length scale is ell = 1/l (Matern) and
ell = 1/sqrt(l) (Gaussian, IMQ)."""
import math

import numpy as np
import pytest

from oracle import h2 as OH
from oracle import kernels as OK
from oracle import pcg as OP
from oracle import spdhss as OS
from oracle import tree as OT
from oracle import ulv as OU
from paper_2011_07632_gb300 import inputs

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def length_scale(kind, l):
    return 1.0 / l if kind == "matern32" else 1.0 / math.sqrt(l)


CASES = [("gauss", 0.001), ("gauss", 0.05), ("gauss", 1.0), ("imq", 0.01), ("imq", 1.0),
         ("imq", 100.0), ("matern32", 0.025)]


@pytest.mark.parametrize("r", [0, 40])
@pytest.mark.parametrize("kind,l", CASES)
def test_sweep_iterations_match_oracle(kind, l, r):
    api = need_gpu()
    n, leaf, sigma, tol = 1500, 100, 1e-2, 1e-8
    ell = length_scale(kind, l)
    X = inputs.ball(n, 3)
    b = inputs.rhs_uniform(n, 1, 1)
    Om = inputs.sketch(n, r + 10, 2)
    h = api.H2(X, kind, ell, sigma, leaf, tol)
    u = api.ULV(api.HSS(h, r, 10, omega=Om))
    x, it, rr = api.pcg_solve(h, u, b, tol=1e-4, maxit=3000)
    tr = OT.build_tree(X, leaf)
    Mh = OH.dense(OH.build_h2(tr, X, OK.NAMES[kind], ell, sigma, tol))
    ou = OU.ULV(OS.build_spdhss(tr, Mh, Om[tr.perm], r))
    xo, ito, rro = OP.pcg(lambda v: Mh @ v, ou.solve, b[tr.perm], 1e-4, 3000)
    # PCG on the block-Jacobi systems that take hundreds of iterations is sensitive to
    # rounding: the oracle itself moves by up to 3% of its count when only the summation
    # order of its product or the last bit of the right-hand side changes (measured on these
    # cases: 605 -> 616, 319 -> 315, 100 -> 97); the tolerance is that spread, at least 1.
    assert abs(int(it[0]) - int(ito[0])) <= max(1, math.ceil(0.03 * int(ito[0])))
    if int(ito[0]) < 3000:
        assert rr[0] <= 1e-4
        xs = x.cpu().numpy()[tr.perm]
        assert np.linalg.norm(b[tr.perm] - Mh @ xs) / np.linalg.norm(b) <= 1.01e-4
