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


def test_waves_same_alone_and_in_the_mix_and_match_the_oracle():
    """The served mixed-precision batched form: requests served in waves (merged
    construction launches with the tensor-core sampling, lockstep PCG) give bit-identical
    results to each request served alone (a wave of one), and two of them match the
    oracle's construction and PCG on the oracle's H^2 matrix."""
    api = need_gpu()
    from oracle import h2 as OH
    from oracle import kernels as OK
    from oracle import pcg as OP
    from oracle import spdhss as OS
    from oracle import tree as OT
    from oracle import ulv as OU
    from paper_2011_07632_gb300 import inputs, serve
    reqs = serve.synthetic_stream(8, rate=400.0, n_lo=1000, n_hi=5000, seed=6, nrhs_max=3,
                                  rank=30, shift=1e-2, blocks=2)
    alone = []
    for r in reqs:
        res, st = serve.Server(None).run_waves([serve.Request(**{**r.__dict__, "arrival": 0.0})],
                                               serve.WaveExecutor(1, precision=1), wave_slots=1)
        assert st["completed"] == 1
        alone.append(res[0])
    mixed, stw = serve.Server(None, hbm_budget=40 << 30).run_waves(
        reqs, serve.WaveExecutor(2, precision=1), wave_slots=2, max_wave=8)
    assert stw["completed"] == 8
    for a, m in zip(alone, mixed):
        assert a.rid == m.rid
        for xa, xm, ia, im in zip(a.x, m.x, a.iters, m.iters):
            assert np.array_equal(xa, xm)
            assert np.array_equal(ia, im)
    # two requests against the oracle (its H^2, quadratic construction, PCG): the served
    # solutions reach the tolerance on the oracle's matrix, iterations within 1 of the
    # oracle's preconditioned CG run with the same sketch drawn on the host
    for k in (0, 1):
        r = reqs[k]
        tr = OT.build_tree(r.points, r.leaf_size)
        Mh = OH.dense(OH.build_h2(tr, r.points, OK.NAMES[r.kernel], r.ell, r.shift, r.tol))
        for b, x, it in zip(r.rhs, mixed[k].x, mixed[k].iters):
            xs = x[tr.perm]
            res = np.linalg.norm(b[tr.perm] - Mh @ xs, axis=0) / np.linalg.norm(b, axis=0)
            assert np.all(res <= 1.01e-6)
        # the same request built with the host sketch, alone, against the oracle
        Om = inputs.sketch(r.n, r.rank + r.oversample, 50 + k)
        h = api.H2(r.points, r.kernel, r.ell, r.shift, r.leaf_size, r.tol)
        hs = api.HSS(h, r.rank, r.oversample, omega=Om, precision=1)
        ohss = OS.build_spdhss(tr, Mh, Om[tr.perm], r.rank)
        Hg = hs.matmul(np.eye(r.n)).cpu().numpy()[np.ix_(tr.perm, tr.perm)]
        assert rel(Hg, OS.assemble_dense(ohss)) < 1e-4
        b = r.rhs[0]
        _, it, rr = api.pcg_solve(h, api.ULV(hs), b, tol=1e-6)
        _, ito, _ = OP.pcg(lambda v: Mh @ v, OU.ULV(ohss).solve, b[tr.perm], 1e-6, 3000)
        assert np.all(np.abs(it - ito) <= 1) and np.all(rr <= 1e-6)
