"""Host logic of the serving loop (no GPU): admission order, slot and HBM-budget limits,
latency accounting, failure isolation, percentiles."""
import threading
import time

import numpy as np
import pytest

from paper_2011_07632_gb300 import serve


def _reqs(k, gap=0.002, n=1000):
    return [serve.Request(rid=i, arrival=i * gap, points=np.zeros((n + 10 * i, 3)),
                          rhs=[np.zeros((n + 10 * i, 1))]) for i in range(k)]


def test_percentile_nearest_rank():
    v = list(range(1, 101))
    assert serve.percentile(v, 50) == 50
    assert serve.percentile(v, 99) == 99
    assert serve.percentile([3.0], 99) == 3.0


def test_admission_respects_slots_and_budget():
    live = {"n": 0, "max": 0, "bytes": 0, "max_bytes": 0}
    lock = threading.Lock()
    fp = lambda r: 100 + r.rid          # noqa: E731
    budget = 450

    def execute(req, slot):
        with lock:
            live["n"] += 1
            live["bytes"] += fp(req)
            live["max"] = max(live["max"], live["n"])
            live["max_bytes"] = max(live["max_bytes"], live["bytes"])
        time.sleep(0.01)
        with lock:
            live["n"] -= 1
            live["bytes"] -= fp(req)
        return [np.full((req.n, 1), req.rid)], [np.array([1])], [np.array([0.0])]

    srv = serve.Server(execute, slots=3, hbm_budget=budget, footprint=fp)
    res, st = srv.run(_reqs(20))
    assert st["completed"] == 20 and st["failed"] == 0
    assert live["max"] <= 3 and st["max_inflight"] <= 3
    assert live["max_bytes"] <= budget and st["max_in_use_bytes"] <= budget
    # first come, first served
    adm = [r.admitted for r in sorted(res, key=lambda r: r.rid)]
    assert adm == sorted(adm)
    assert all(r.latency >= 0.0 and r.finished >= r.admitted >= r.arrival - 1e-3 for r in res)
    assert all(r.x[0][0, 0] == r.rid for r in res)


def test_failed_request_frees_its_slot_and_memory():
    def execute(req, slot):
        if req.rid == 2:
            raise RuntimeError("NOT_SPD: injected on the host")
        return [np.zeros((req.n, 1))], [np.array([1])], [np.array([0.0])]

    srv = serve.Server(execute, slots=1, hbm_budget=10**12, footprint=lambda r: 10)
    res, st = srv.run(_reqs(6))
    assert st["completed"] == 5 and st["failed"] == 1
    assert "NOT_SPD" in res[2].error
    assert srv.trace[-1][1] == 0 and srv.trace[-1][2] == 0


def test_oversized_request_is_rejected_not_blocking():
    def execute(req, slot):
        return [np.zeros((req.n, 1))], [np.array([1])], [np.array([0.0])]

    srv = serve.Server(execute, slots=2, hbm_budget=150, footprint=lambda r: 1000 if r.rid == 1 else 100)
    res, st = srv.run(_reqs(4))
    assert res[1].error.startswith("rejected")
    assert st["completed"] == 3


def test_synthetic_stream_shape():
    reqs = serve.synthetic_stream(12, rate=200.0, n_lo=1000, n_hi=4000, seed=1)
    arr = [r.arrival for r in reqs]
    assert arr == sorted(arr) and arr[0] == 0.0
    assert {r.points.shape[1] for r in reqs} == {2, 3}
    assert {r.kernel for r in reqs} == {"exp", "gauss", "matern32"}
    assert all(1000 <= r.n <= 4000 for r in reqs)
    assert all(1 <= r.rhs[0].shape[1] <= 16 for r in reqs)
    assert serve.footprint_bytes(reqs[0]) > 0


def test_footprint_counts_unknowns():
    """An RPY request (three unknowns per point) is sized by its 3n unknowns."""
    X = np.zeros((5000, 3))
    scalar = serve.Request(rid=0, arrival=0.0, points=X, kernel="exp", leaf_size=64)
    rpy = serve.Request(rid=1, arrival=0.0, points=X, kernel="rpy", leaf_size=64)
    assert scalar.unknowns == 5000 and rpy.unknowns == 15000
    assert serve.footprint_bytes(rpy) >= 3 * (serve.footprint_bytes(scalar) - (64 << 20))


def test_waves_batch_arrivals_and_respect_the_budget():
    """Requests admitted while waves run join later waves; at most `wave_slots` waves at a
    time; memory in use never exceeds the budget; every request gets its own result."""
    fp = lambda r: 100 + r.rid          # noqa: E731
    budget = 1000
    seen = {"waves": [], "live": 0, "max_live": 0}
    lock = threading.Lock()

    def execute_wave(reqs, slot):
        with lock:
            seen["waves"].append([r.rid for r in reqs])
            seen["live"] += 1
            seen["max_live"] = max(seen["max_live"], seen["live"])
        time.sleep(0.02)
        with lock:
            seen["live"] -= 1
        return [([np.full((r.n, 1), r.rid)], [np.array([1])], [np.array([0.0])]) for r in reqs]

    srv = serve.Server(None, hbm_budget=budget, footprint=fp)
    res, st = srv.run_waves(_reqs(30, gap=0.003), execute_wave, wave_slots=2, max_wave=6)
    assert st["completed"] == 30 and st["failed"] == 0
    assert seen["max_live"] <= 2
    assert max(len(w) for w in seen["waves"]) <= 6
    assert len(seen["waves"]) < 30            # arrivals were batched
    assert sorted(sum(seen["waves"], [])) == list(range(30))
    assert st["max_in_use_bytes"] <= budget
    assert all(r.x[0][0, 0] == r.rid for r in res)
    # first come, first served into waves
    order = sum(seen["waves"], [])
    assert order == sorted(order)


def test_failed_wave_frees_its_memory():
    calls = {"n": 0}

    def execute_wave(reqs, slot):
        calls["n"] += 1
        if calls["n"] == 1:
            raise RuntimeError("NOT_SPD: injected on the host")
        return [([np.zeros((r.n, 1))], [np.array([1])], [np.array([0.0])]) for r in reqs]

    srv = serve.Server(None, hbm_budget=10**12, footprint=lambda r: 10)
    res, st = srv.run_waves(_reqs(8, gap=0.01), execute_wave, wave_slots=1, max_wave=4)
    assert st["completed"] + st["failed"] == 8 and st["failed"] >= 1
    assert all(r.error is None for r in res if r.rid >= 4)


def test_wave_requests_finish_at_their_own_finish_times():
    """An executor that reports a finish time per request (the batched solve's per-instance
    completion) gives each request that finish, not the wave's return; memory is still
    released when the wave returns."""
    def execute_wave(reqs, slot):
        t = []
        for k, r in enumerate(reqs):
            time.sleep(0.01)
            t.append(time.perf_counter())
        time.sleep(0.05)
        return [([np.zeros((r.n, 1))], [np.array([1])], [np.array([0.0])], t[k])
                for k, r in enumerate(reqs)]

    srv = serve.Server(None, hbm_budget=10**12, footprint=lambda r: 10)
    reqs = [serve.Request(**{**r.__dict__, "arrival": 0.0}) for r in _reqs(4)]
    res, st = srv.run_waves(reqs, execute_wave, wave_slots=1, max_wave=4)
    assert st["completed"] == 4
    fin = [r.finished for r in sorted(res, key=lambda r: r.rid)]
    assert fin == sorted(fin) and fin[-1] - fin[0] >= 0.025
    assert st["wall_s"] - fin[-1] >= 0.04       # the wave returned later
    assert srv.trace[-1][1] == 0
