"""Serving on the GPU: a Poisson stream of mixed requests served concurrently on several
CUDA streams gives, for every request, the same result as serving it alone."""
import numpy as np
import pytest

from gpu_util import need_gpu, rel

pytestmark = pytest.mark.gpu


def test_results_same_alone_and_in_the_mix():
    need_gpu()
    from paper_2011_07632_gb300 import serve
    reqs = serve.synthetic_stream(10, rate=200.0, n_lo=1000, n_hi=6000, seed=4, nrhs_max=4,
                                  rank=30, shift=1e-2, blocks=2)
    alone, st1 = serve.Server(serve.GpuExecutor(1), slots=1).run(
        [serve.Request(**{**r.__dict__, "arrival": 0.0}) for r in reqs])
    mixed, st4 = serve.Server(serve.GpuExecutor(4), slots=4, hbm_budget=40 << 30).run(reqs)
    assert st1["completed"] == 10 and st4["completed"] == 10
    assert st4["max_inflight"] >= 2
    for a, m in zip(alone, mixed):
        assert a.rid == m.rid
        for xa, xm, ra in zip(a.x, m.x, a.relres):
            assert rel(xm, xa) <= 1e-12
            assert np.all(ra <= 1e-6)
