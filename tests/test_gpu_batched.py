"""Batched level sweep over independent instances (spdhss_build_batched, pcg_solve_batched,
pcg_solve_batched_mixed, pcg_solve_batched_ex):
every instance's results are bit-identical to its one-instance build and solve, instances
inside a batch match the oracle, the launches are merged, and a failing instance leaves the
others intact."""
import math

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


def test_batched_build_is_bit_identical_to_single_builds():
    """Six instances (2D and 3D, all three kernels): every result of the merged sweep equals
    the one-instance result exactly, since no kernel's per-problem arithmetic depends on the
    other problems of its launch."""
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
        off, idx = h.export_skeletons()
        off1, idx1 = h1.export_skeletons()
        assert np.array_equal(off, off1) and np.array_equal(idx, idx1)
        assert np.array_equal(h.matmul(x).cpu().numpy(), h1.matmul(x).cpu().numpy())
        assert hs.info() == hs1.info()
        assert np.array_equal(hs.matmul(x).cpu().numpy(), hs1.matmul(x).cpu().numpy())
        assert np.array_equal(u.solve(x).cpu().numpy(), u1.solve(x).cpu().numpy())


def test_batched_pcg_is_bit_identical_to_single_solves():
    api = need_gpu()
    insts = _instances(6, seed=4)
    built, status, _ = api.build_batched(insts)
    assert status == [native.OK] * len(insts)
    Bs = [inputs.rhs(i["points"].shape[0], 1 + (k % 3), 20 + k) for k, i in enumerate(insts)]
    X, its, rrs, st = api.pcg_solve_batched([b[0] for b in built], [b[2] for b in built], Bs,
                                            tol=1e-6)
    assert st == [native.OK] * len(insts)
    for (h, hs, u), b, x, it, rr in zip(built, Bs, X, its, rrs):
        x1, it1, rr1 = api.pcg_solve(h, u, b, tol=1e-6)
        assert np.array_equal(it, it1)
        assert np.array_equal(rr, rr1)
        assert np.array_equal(x.cpu().numpy(), x1.cpu().numpy())
        assert np.all(rr <= 1e-6)


@pytest.mark.parametrize("precision", [0, 1])
def test_mixed_batched_pcg_is_bit_identical_to_single_mixed_solves(precision):
    """pcg_solve_batched_mixed (FP32 products of all instances in merged launches) against
    pcg_solve_mixed per instance: solutions, iteration counts and residuals bit-identical.
    Six instances with 1 to 16 columns (FP32 product widths 1, 2, 4, 8, 16) built in FP64 or
    in the precision mode; one low-rank instance iterates past the FP64 residual refresh
    (every 50 iterations) and the others converge earlier, so the merged product is rebuilt
    for a shrinking set of instances."""
    api = need_gpu()
    insts = _instances(6, seed=8)
    insts[5]["rank"] = 2
    for i in insts:
        i["precision"] = precision
    built, status, _ = api.build_batched(insts)
    assert status == [native.OK] * len(insts)
    widths = [1, 3, 16, 5, 8, 2]
    Bs = [inputs.rhs(i["points"].shape[0], w, 50 + k)
          for k, (i, w) in enumerate(zip(insts, widths))]
    X, its, rrs, st = api.pcg_solve_batched([b[0] for b in built], [b[2] for b in built], Bs,
                                            tol=1e-6, mixed=True)
    assert st == [native.OK] * len(insts)
    assert max(int(np.max(v)) for v in its) > 50
    assert len({int(np.max(v)) for v in its}) > 1
    for (h, hs, u), b, x, it, rr in zip(built, Bs, X, its, rrs):
        x1, it1, rr1 = api.pcg_solve(h, u, b, tol=1e-6, mixed=True)
        assert np.array_equal(it, it1)
        assert np.array_equal(rr, rr1)
        assert np.array_equal(x.cpu().numpy(), x1.cpu().numpy())
        assert np.all(rr <= 1e-6)


@pytest.mark.parametrize("mixed", [False, True])
def test_batched_pcg_reports_each_instance_when_it_finishes(mixed):
    """pcg_solve_batched_ex: every instance reported once, in the order its iterations ended
    (non-decreasing counts), with the results of the call without the callback."""
    api = need_gpu()
    insts = _instances(6, seed=10)
    built, status, _ = api.build_batched(insts)
    assert status == [native.OK] * len(insts)
    Bs = [inputs.rhs(i["points"].shape[0], 1 + (k % 4), 90 + k) for k, i in enumerate(insts)]
    hs, us = [b[0] for b in built], [b[2] for b in built]
    X0, its0, rrs0, st0 = api.pcg_solve_batched(hs, us, Bs, tol=1e-6, mixed=mixed)
    seen = []

    def done(k, status, x, it, rr):
        seen.append((k, status, x.cpu().numpy(), it, rr))

    X1, its1, rrs1, st1 = api.pcg_solve_batched(hs, us, Bs, tol=1e-6, mixed=mixed, on_done=done)
    assert st1 == st0 == [native.OK] * len(insts)
    assert sorted(k for k, *_ in seen) == list(range(len(insts)))
    ends = [int(np.max(it)) for _, _, _, it, _ in seen]
    assert ends == sorted(ends)
    for k, status, x, it, rr in seen:
        assert status == native.OK
        assert np.array_equal(x, X0[k].cpu().numpy()) and np.array_equal(x, X1[k].cpu().numpy())
        assert np.array_equal(it, its0[k]) and np.array_equal(rr, rrs0[k])


def test_mixed_pcg_converges_on_ill_conditioned_instances():
    """Gaussian kernels in 2D with small shifts: the FP32 product's error relative to the
    residual is large (x = A^-1 b is dominated by the eigenvectors of the smallest
    eigenvalues), so the mixed solve restarts drifting columns and, where a block of
    iterations makes no progress, switches to FP64 products.  Every column still reaches
    the FP64 tolerance, and the batched solve stays bit-identical to the single ones."""
    api = need_gpu()
    insts = []
    for k, n in enumerate([16000, 9000, 4000]):
        insts.append(dict(points=inputs.uniform_cube(n, 2, 300 + k), kernel="gauss", ell=0.1,
                          shift=1e-3, leaf_size=64, tol=1e-8, rank=50, oversample=10, seed=k))
    built, status, _ = api.build_batched(insts)
    assert status == [native.OK] * len(insts)
    Bs = [inputs.rhs(i["points"].shape[0], 1 + 3 * k, 80 + k) for k, i in enumerate(insts)]
    X, its, rrs, st = api.pcg_solve_batched([b[0] for b in built], [b[2] for b in built], Bs,
                                            tol=1e-6, maxit=3000, mixed=True)
    assert st == [native.OK] * len(insts)
    for (h, hs, u), b, x, it, rr in zip(built, Bs, X, its, rrs):
        _, it64, rr64 = api.pcg_solve(h, u, b, tol=1e-6)
        assert np.all(rr64 <= 1e-6)
        x1, it1, rr1 = api.pcg_solve(h, u, b, tol=1e-6, mixed=True)
        assert np.array_equal(it, it1) and np.array_equal(rr, rr1)
        assert np.array_equal(x.cpu().numpy(), x1.cpu().numpy())
        assert np.all(rr <= 1e-6)
        r = b - h.matmul(x).cpu().numpy()
        assert np.all(np.linalg.norm(r, axis=0) / np.linalg.norm(b, axis=0) <= 1.01e-6)


def test_mixed_batched_instances_match_the_oracle():
    """Two instances of a mixed batched solve against the oracle: iterations within 10% (at
    least 3) of the oracle's FP64 PCG with its own ULV preconditioner on its own H^2 matrix
    (the FP32 products perturb the Krylov recurrence by ~1e-6 relative per product), and the
    FP64 true residual of the returned solution within the tolerance."""
    api = need_gpu()
    from oracle import h2 as OH
    from oracle import kernels as OK
    from oracle import pcg as OP
    from oracle import spdhss as OS
    from oracle import tree as OT
    from oracle import ulv as OU
    insts = _instances(4, n_lo=900, n_hi=1600, seed=9)
    checked = [0, 1]
    for k in checked:
        n = insts[k]["points"].shape[0]
        insts[k]["omega"] = inputs.sketch(n, insts[k]["rank"] + 10, 60 + k)
    built, status, _ = api.build_batched(insts)
    assert status == [native.OK] * len(insts)
    Bs = [inputs.rhs(i["points"].shape[0], 1, 70 + k) for k, i in enumerate(insts)]
    X, its, rrs, st = api.pcg_solve_batched([b[0] for b in built], [b[2] for b in built], Bs,
                                            tol=1e-6, mixed=True)
    assert st == [native.OK] * len(insts)
    for k in checked:
        inst = insts[k]
        P = inst["points"]
        tr = OT.build_tree(P, inst["leaf_size"])
        oh = OH.build_h2(tr, P, OK.NAMES[inst["kernel"]], inst["ell"], inst["shift"], inst["tol"])
        Mh = OH.dense(oh)
        ohss = OS.build_spdhss(tr, Mh, inst["omega"][tr.perm], inst["rank"])
        _, ito, _ = OP.pcg(lambda v: Mh @ v, OU.ULV(ohss).solve, Bs[k][tr.perm], 1e-6, 3000)
        assert abs(int(its[k][0]) - int(ito[0])) <= max(3, math.ceil(0.1 * int(ito[0])))
        r = Bs[k] - built[k][0].matmul(X[k]).cpu().numpy()
        assert np.linalg.norm(r) / np.linalg.norm(Bs[k]) <= 1.01e-6
        assert rrs[k][0] <= 1e-6


def test_batched_instances_match_the_oracle():
    """Two instances built and solved inside a batch (with explicit sketches) against the
    oracle's quadratic construction on its own H^2 matrix: assembled HSS within 1e-10,
    PCG iterations within one of the oracle's PCG with its own ULV preconditioner."""
    api = need_gpu()
    from oracle import h2 as OH
    from oracle import kernels as OK
    from oracle import pcg as OP
    from oracle import spdhss as OS
    from oracle import tree as OT
    from oracle import ulv as OU
    insts = _instances(4, n_lo=900, n_hi=1600, seed=6)
    checked = [0, 1]
    for k in checked:
        n = insts[k]["points"].shape[0]
        insts[k]["omega"] = inputs.sketch(n, insts[k]["rank"] + 10, 30 + k)
    built, status, _ = api.build_batched(insts)
    assert status == [native.OK] * len(insts)
    Bs = [inputs.rhs(i["points"].shape[0], 1, 40 + k) for k, i in enumerate(insts)]
    X, its, rrs, st = api.pcg_solve_batched([b[0] for b in built], [b[2] for b in built], Bs,
                                            tol=1e-6)
    assert st == [native.OK] * len(insts)
    for k in checked:
        inst = insts[k]
        P = inst["points"]
        n = P.shape[0]
        tr = OT.build_tree(P, inst["leaf_size"])
        oh = OH.build_h2(tr, P, OK.NAMES[inst["kernel"]], inst["ell"], inst["shift"], inst["tol"])
        Mh = OH.dense(oh)
        ohss = OS.build_spdhss(tr, Mh, inst["omega"][tr.perm], inst["rank"])
        Ho = OS.assemble_dense(ohss)
        hs = built[k][1]
        Hg = hs.matmul(np.eye(n)).cpu().numpy()[np.ix_(tr.perm, tr.perm)]
        assert rel(Hg, Ho) < 1e-10
        _, ito, _ = OP.pcg(lambda v: Mh @ v, OU.ULV(ohss).solve, Bs[k][tr.perm], 1e-6, 3000)
        assert abs(int(its[k][0]) - int(ito[0])) <= 1
        assert rrs[k][0] <= 1e-6


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
        assert np.array_equal(hs.matmul(x).cpu().numpy(), hs1.matmul(x).cpu().numpy())
