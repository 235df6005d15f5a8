"""Mixed precision: FP32 H^2 products against the FP64 product and the exact kernel matrix;
PCG with the FP32 product reaches the FP64 true-residual tolerance."""
import math

import numpy as np
import pytest

from oracle import kernels as OK
from paper_2011_07632_gb300 import inputs

from gpu_util import need_gpu, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,ell,dim,nrhs", [("exp", 1.0, 3, 1), ("gauss", 0.2, 3, 8),
                                               ("matern32", 0.1, 2, 3), ("imq", 0.5, 3, 16)])
def test_fp32_product_accuracy(kind, ell, dim, nrhs):
    api = need_gpu()
    n = 3000
    X = inputs.uniform_cube(n, dim, 5)
    h = api.H2(X, kind, ell, 1e-3, 64, 1e-8)
    x = inputs.rhs(n, nrhs, 6)
    y64 = h.matmul(x).cpu().numpy()
    y32 = h.matmul_mixed(x).cpu().numpy()
    A = OK.dense_matrix(OK.NAMES[kind], ell, 1e-3, X)
    assert rel(y32, y64) < 2e-5
    assert rel(y32, A @ x) < 2e-5


@pytest.mark.parametrize("nrhs", [1, 4])
def test_mixed_pcg_reaches_fp64_tolerance(nrhs):
    api = need_gpu()
    n = 4096
    X = inputs.uniform_cube(n, 3, 0)
    h = api.H2(X, "exp", 1.0, 1e-2, 64, 1e-8)
    u = api.ULV(api.HSS(h, 50, 10, omega=inputs.sketch(n, 60, 2)))
    b = inputs.rhs(n, nrhs, 1)
    x64, it64, rr64 = api.pcg_solve(h, u, b, tol=1e-6)
    x32, it32, rr32 = api.pcg_solve(h, u, b, tol=1e-6, mixed=True, raise_on_no_convergence=True)
    assert np.all(rr32 <= 1e-6)
    assert np.all(it32 <= 2 * it64 + 10)
    # the FP64 residual of the mixed solution, recomputed with the FP64 product
    r = b - h.matmul(x32).cpu().numpy()
    assert np.all(np.linalg.norm(r, axis=0) / np.linalg.norm(b, axis=0) <= 1.01e-6)


@pytest.mark.parametrize("nrhs,row_block", [(3, None), (8, None), (16, None), (8, "128"),
                                            (13, "512")])
def test_fp32_product_split_rows(nrhs, row_block, monkeypatch):
    """High-rank nodes (ranks and transfer-matrix heights above the 128-512 rows of one
    job): the FP32 product then splits their rows over several jobs and adds the partial
    results in a fixed order.  SPDHSS_SYM_ROW_BLOCK sets the rows per job (default 256)."""
    api = need_gpu()
    if row_block:
        monkeypatch.setenv("SPDHSS_SYM_ROW_BLOCK", row_block)
    n = 60000
    X = inputs.uniform_cube(n, 3, 11)
    h = api.H2(X, "gauss", 0.1, 1e-4, 128, 1e-8)
    off, _ = h.export_skeletons()
    k = np.diff(off)
    assert k.max() > int(row_block or 256) // 2
    x = inputs.rhs(n, nrhs, 12)
    y64 = h.matmul(x).cpu().numpy()
    y32 = h.matmul_mixed(x).cpu().numpy()
    # FP32 rounding against sums with ~1000 significant terms of both signs per row
    assert rel(y32, y64) < 1e-4
    # deterministic: a second product is bit-identical
    assert np.array_equal(h.matmul_mixed(x).cpu().numpy(), y32)


@pytest.mark.parametrize("n,nrhs", [(1, 1), (65, 2), (700, 5), (700, 9), (2500, 16)])
def test_fp32_product_small_and_ragged(n, nrhs):
    """Single points, a single leaf, ragged leaves and right-hand-side counts between the
    kernel's column widths (1, 2, 4, 8, 16) against the exact kernel matrix."""
    api = need_gpu()
    X = inputs.uniform_cube(n, 3, 21)
    h = api.H2(X, "exp", 0.5, 1e-2, 64, 1e-8)
    x = inputs.rhs(n, nrhs, 22)
    y32 = h.matmul_mixed(x).cpu().numpy()
    A = OK.dense_matrix(OK.NAMES["exp"], 0.5, 1e-2, X)
    assert rel(y32, A @ x) < 2e-5


# ---- precision mode of the construction (spdhss_build_precision) ------------------------
# The sampling product runs in FP32 with its GEMMs on the tensor cores (3xTF32, or plain
# TF32); everything after it is FP64.  Bounds from the arithmetic and measured values:
# 3xTF32 carries FP32 rounding (~1e-6 relative) into the samples, which moves the HSS by
# about 1e-5 (measured 6e-6 .. 3e-5 against the FP64 oracle) and leaves its approximation
# error and PCG iteration counts unchanged; plain TF32 products carry ~1e-3 (measured
# 1e-3 .. 7e-3 against the oracle, iterations up to 1.7x on the Matern case).
PREC_CASES = [("exp", 1.0, 1e-2, 3, 3000, 64, 40), ("matern32", 0.2, 1e-3, 2, 2500, 64, 30),
              ("gauss", 0.3, 1e-3, 3, 2000, 64, 30)]


@pytest.mark.parametrize("kind,ell,sigma,dim,n,leaf,r", PREC_CASES)
def test_precision_mode_against_the_oracle(kind, ell, sigma, dim, n, leaf, r):
    api = need_gpu()
    from oracle import h2 as OH
    from oracle import pcg as OP
    from oracle import spdhss as OS
    from oracle import tree as OT
    from oracle import ulv as OU
    X = inputs.uniform_cube(n, dim, 0)
    Om = inputs.sketch(n, r + 10, 2)
    h = api.H2(X, kind, ell, sigma, leaf, 1e-8)
    tr = OT.build_tree(X, leaf)
    Mh = OH.dense(OH.build_h2(tr, X, OK.NAMES[kind], ell, sigma, 1e-8))
    ohss = OS.build_spdhss(tr, Mh, Om[tr.perm], r)
    Ho = OS.assemble_dense(ohss)
    b = inputs.rhs(n, 1, 1)
    _, ito, _ = OP.pcg(lambda v: Mh @ v, OU.ULV(ohss).solve, b[tr.perm], 1e-6, 3000)
    a_oracle = rel(Ho, Mh)   # the oracle's approximation error
    for prec, bound, approx_slack, it_factor in ((1, 1e-4, 1e-3, 1.0), (2, 2e-2, 0.3, 2.0)):
        hs = api.HSS(h, r, 10, omega=Om, precision=prec)
        Hg = hs.matmul(np.eye(n)).cpu().numpy()[np.ix_(tr.perm, tr.perm)]
        assert rel(Hg, Ho) < bound, (prec, rel(Hg, Ho))
        assert rel(Hg, Mh) <= a_oracle * (1 + approx_slack) + 1e-8, (prec, rel(Hg, Mh), a_oracle)
        x, it, rr = api.pcg_solve(h, api.ULV(hs), b, tol=1e-6, raise_on_no_convergence=True)
        assert rr[0] <= 1e-6
        # counts in the hundreds move by up to 3% under rounding-only changes (measured on
        # the oracle: a transposed product or a 1e-15 change of b; the Gaussian case here
        # takes ~500 iterations), so the bound carries that spread
        assert it[0] <= it_factor * math.ceil(1.03 * int(ito[0])) + 1, (prec, int(it[0]), int(ito[0]))


@pytest.mark.parametrize("prec", [1, 2])
def test_precision_mode_is_spd(prec):
    """SPD by a dense eigensolve at n = 512 with tiny shifts (Sec. 3.2): the compression,
    the factors and B_ij stay FP64, so FP32 samples leave the guarantee intact."""
    api = need_gpu()
    n = 512
    X = inputs.uniform_cube(n, 3, 6)
    for kind, sigma, r in (("gauss", 1e-6, 4), ("matern32", 1e-5, 10)):
        h = api.H2(X, kind, 0.2, sigma, 16, 1e-8)
        hs = api.HSS(h, r, 10, seed=11, precision=prec)
        Hg = hs.matmul(np.eye(n)).cpu().numpy()
        assert np.linalg.eigvalsh(0.5 * (Hg + Hg.T)).min() > 0.0


def test_precision_build_then_fp32_products_on_one_handle():
    """The precision-mode build makes some FP32 copies of the H^2 generators (bases,
    source-major couplings); the FP32 product made afterwards on the same handle must still
    make its own (destination-major couplings) and agree with the FP64 product."""
    api = need_gpu()
    n = 3000
    X = inputs.uniform_cube(n, 3, 8)
    h = api.H2(X, "matern32", 0.2, 1e-3, 64, 1e-8)
    hs = api.HSS(h, 30, 10, seed=4, precision=1)
    x = inputs.rhs(n, 2, 9)
    assert rel(h.matmul_mixed(x).cpu().numpy(), h.matmul(x).cpu().numpy()) < 2e-5
    b = inputs.rhs(n, 1, 10)
    _, it, rr = api.pcg_solve(h, api.ULV(hs), b, tol=1e-6, mixed=True,
                              raise_on_no_convergence=True)
    assert rr[0] <= 1e-6
