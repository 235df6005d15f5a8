"""Batched level sweep over independent instances (spdhss_build_batched, pcg_solve_batched):
every instance agrees with its one-instance build and solve, the launches are merged, and
a failing instance leaves the others intact."""
import numpy as np
import pytest

from paper_2011_07632_gb300 import inputs, native

from gpu_util import need_gpu, rel

pytestmark = pytest.mark.gpu

KINDS = [("exp", 1.0), ("gauss", 0.1), ("matern32", 0.1)]


def _instances(count, n_lo=600, n_hi=3000, seed=3):
    sizes = inputs.log_uniform_sizes(count, n_lo, n_hi, seed)
    out = []
    for k in range(count):
        kind, ell = KINDS[k % 3]
        dim = 2 if k % 2 == 0 else 3
        out.append(dict(points=inputs.uniform_cube(int(sizes[k]), dim, 100 + k), kernel=kind,
                        ell=ell, shift=1e-3, leaf_size=64, tol=1e-8, rank=30, oversample=10,
                        seed=k))
    return out


def _single(api, inst):
    h = api.H2(inst["points"], inst["kernel"], inst["ell"], inst["shift"], inst["leaf_size"],
               inst["tol"])
    hs = api.HSS(h, inst["rank"], inst["oversample"], seed=inst["seed"])
    return h, hs, api.ULV(hs)


def test_batched_build_matches_single_builds():
    api = need_gpu()
    insts = _instances(6)
    c0 = native.launch_count()
    built, status, (merged, handed) = api.build_batched(insts)
    c1 = native.launch_count()
    assert status == [native.OK] * len(insts)
    # the hand-overs of all instances went out in fewer launches
    assert 0 < merged < handed
    singles = [_single(api, i) for i in insts]
    c2 = native.launch_count()
    assert c1 - c0 < c2 - c1
    for inst, (h, hs, u), (h1, hs1, u1) in zip(insts, built, singles):
        n = inst["points"].shape[0]
        x = inputs.rhs(n, 3, 7)
        assert h.info()["skeleton_total"] == h1.info()["skeleton_total"]
        assert rel(h.matmul(x).cpu().numpy(), h1.matmul(x).cpu().numpy()) < 1e-12
        assert rel(hs.matmul(x).cpu().numpy(), hs1.matmul(x).cpu().numpy()) < 1e-10
        assert rel(u.solve(x).cpu().numpy(), u1.solve(x).cpu().numpy()) < 1e-8


def test_batched_pcg_matches_single_solves():
    api = need_gpu()
    insts = _instances(5, seed=4)
    built, status, _ = api.build_batched(insts)
    assert status == [native.OK] * len(insts)
    Bs = [inputs.rhs(i["points"].shape[0], 1 + (k % 3), 20 + k) for k, i in enumerate(insts)]
    X, its, rrs, st = api.pcg_solve_batched([b[0] for b in built], [b[2] for b in built], Bs,
                                            tol=1e-6)
    assert st == [native.OK] * len(insts)
    for (h, hs, u), b, x, it, rr in zip(built, Bs, X, its, rrs):
        x1, it1, rr1 = api.pcg_solve(h, u, b, tol=1e-6)
        assert np.all(np.abs(it - it1) <= 1)
        assert np.all(rr <= 1e-6)
        r = b - h.matmul(x).cpu().numpy()
        assert np.all(np.linalg.norm(r, axis=0) / np.linalg.norm(b, axis=0) <= 1.01e-6)


def test_failing_instance_leaves_the_others():
    api = need_gpu()
    insts = _instances(3, seed=5)
    # every point four times and no shift: singular leaf blocks, the leaf Cholesky fails
    insts[1] = dict(points=np.repeat(inputs.uniform_cube(50, 3, 1), 4, axis=0), kernel="gauss",
                    ell=0.5, shift=0.0, leaf_size=16, tol=1e-8, rank=8, oversample=10, seed=1)
    built, status, _ = api.build_batched(insts)
    assert status == [native.OK, native.NOT_SPD, native.OK]
    assert built[1] is None
    for k in (0, 2):
        h, hs, u = built[k]
        h1, hs1, u1 = _single(api, insts[k])
        x = inputs.rhs(insts[k]["points"].shape[0], 2, 9)
        assert rel(hs.matmul(x).cpu().numpy(), hs1.matmul(x).cpu().numpy()) < 1e-10
