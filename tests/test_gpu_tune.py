"""Launch-variant autotuning: the tuned kind (columns per CTA of the blocked triangular
solve) leaves the arithmetic unchanged, so the SPD-HSS construction, the ULV factorization
and PCG give bit-identical results with every width forced (SPDHSS_TRSM_COLS), with the
tuner's choices and with tuning off (SPDHSS_TUNE=0); the tuner records one choice per shape
bucket."""
import numpy as np
import pytest

from paper_2011_07632_gb300 import inputs, native

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _run(api):
    n = 3000
    X = inputs.uniform_cube(n, 3, 4)
    h = api.H2(X, "matern32", 0.2, 1e-3, 64, 1e-8)
    hs = api.HSS(h, 40, 10, omega=inputs.sketch(n, 50, 2))
    u = api.ULV(hs)
    b = inputs.rhs(n, 2, 5)
    x, it, rr = api.pcg_solve(h, u, b, tol=1e-8)
    v = inputs.rhs(n, 3, 6)
    return (hs.matmul(v).cpu().numpy(), u.solve(v).cpu().numpy(), x.cpu().numpy(),
            np.asarray(it), np.asarray(rr))


def test_trsm_width_is_arithmetic_neutral(monkeypatch):
    api = need_gpu()
    ref = _run(api)                       # tuned widths
    rep = native.tuning_report()
    assert any("trsm_blk" in k for k in rep) and all(v in (1, 2, 4, 8) for v in rep.values())
    for w in ("1", "2", "4", "8"):
        monkeypatch.setenv("SPDHSS_TRSM_COLS", w)
        got = _run(api)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b), w
    monkeypatch.delenv("SPDHSS_TRSM_COLS")
    monkeypatch.setenv("SPDHSS_TUNE", "0")
    got = _run(api)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
