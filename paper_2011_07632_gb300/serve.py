"""Serving loop: continuous batching of build+solve requests on one GPU.

Two forms share the admission policy.  Server.run gives every admitted request a worker
slot and a CUDA stream of its own (one-request-at-a-time with one slot); Server.run_waves
gathers the requests admitted while earlier waves are on the GPU into the next wave,
served by the batched ABI (merged construction launches in the precision mode, lockstep
PCG with the FP32 H^2 products merged over the wave), with two waves overlapping on the
device.

Requests (points, kernel, shift, HSS rank, one or more blocks of right-hand sides) arrive
over time.  A request is admitted as soon as its arrival time has passed, a worker slot is
free and its estimated device footprint fits the HBM budget (first come, first served; a
request that does not fit waits and later ones wait behind it).  An admitted request runs
h2_build, spdhss_build and ulv_factor on its own CUDA stream, keeps that H^2 / HSS / ULV
state resident while pcg_solve serves each of its right-hand-side blocks, then releases it.
Requests in flight therefore overlap on the device, and every result is the same as when
the request runs alone (the kernels are deterministic and the sketch is seeded).

Latency of a request = time its last solve finished - its arrival time.
"""
from __future__ import annotations

import dataclasses
import threading
import time
from typing import Callable, List, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float                  # seconds from the start of the run
    points: np.ndarray              # (n, dim) float64
    kernel: str = "exp"
    ell: float = 1.0
    shift: float = 1e-2
    leaf_size: int = 64
    tol: float = 1e-8
    rank: int = 50
    oversample: int = 10
    seed: int = 0
    rhs: Sequence[np.ndarray] = ()  # blocks (unknowns, nrhs) solved with the same resident state
    relres: float = 1e-6
    maxit: int = 3000

    @property
    def n(self) -> int:
        return int(self.points.shape[0])

    @property
    def unknowns(self) -> int:
        """Matrix size: three unknowns per point for the RPY tensor kernel."""
        return self.n * (3 if self.kernel == "rpy" else 1)


@dataclasses.dataclass
class Result:
    rid: int
    x: List[np.ndarray]
    iters: List[np.ndarray]
    relres: List[np.ndarray]
    arrival: float
    admitted: float
    finished: float
    footprint: int
    error: Optional[str] = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def footprint_bytes(req: Request) -> int:
    """Upper estimate of the device memory of one request: H^2 generators (couplings of up
    to ~190 far neighbours per leaf at leaf-sized ranks), SPD-HSS and ULV factors, the
    sampling buffers of the construction, and the solve vectors.  Sizes count unknowns
    (a leaf of L points holds 3L unknowns for the RPY kernel, and its ranks scale alike)."""
    k = req.unknowns // max(req.n, 1)
    n, L, r = req.unknowns, req.leaf_size * k, req.rank
    s = r + req.oversample
    nrhs = max((b.shape[1] if b.ndim == 2 else 1) for b in req.rhs) if len(req.rhs) else 1
    h2 = 8 * n * (190 * min(L, 64 * k) + 64)
    hss = 8 * n * (6 * r + 4 * s + 2 * L)
    vec = 8 * n * (8 * s + 16 * nrhs)
    return int(h2 + hss + vec + (64 << 20))


def percentile(values: Sequence[float], q: float) -> float:
    """Nearest-rank percentile (q in [0, 100])."""
    v = sorted(values)
    if not v:
        return float("nan")
    k = max(0, min(len(v) - 1, int(np.ceil(q / 100.0 * len(v))) - 1))
    return float(v[k])


class Server:
    """Admission and worker threads; `execute(request, slot)` does the device work and
    returns (x blocks, iteration arrays, relres arrays)."""

    def __init__(self, execute: Callable, slots: int = 4, hbm_budget: Optional[int] = None,
                 footprint: Callable[[Request], int] = footprint_bytes,
                 clock: Callable[[], float] = time.perf_counter):
        self.execute = execute
        self.slots = int(slots)
        self.hbm_budget = hbm_budget
        self.footprint = footprint
        self.clock = clock
        self.trace = []          # (time, in_use_bytes, inflight) after every admit/finish

    def run(self, requests: Sequence[Request]):
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        t0 = self.clock()
        cv = threading.Condition()
        state = {"inflight": 0, "in_use": 0, "free_slots": list(range(self.slots))}
        results: List[Result] = []
        threads = []

        def worker(req: Request, slot: int, fp: int, admitted: float):
            err = None
            xs, its, rrs = [], [], []
            try:
                xs, its, rrs = self.execute(req, slot)
            except Exception as e:  # a failed request frees its slot and memory
                err = f"{type(e).__name__}: {e}"
            done = self.clock() - t0
            with cv:
                results.append(Result(req.rid, xs, its, rrs, req.arrival, admitted, done, fp, err))
                state["inflight"] -= 1
                state["in_use"] -= fp
                state["free_slots"].append(slot)
                self.trace.append((done, state["in_use"], state["inflight"]))
                cv.notify_all()

        for req in reqs:
            fp = int(self.footprint(req))
            if self.hbm_budget is not None and fp > self.hbm_budget:
                results.append(Result(req.rid, [], [], [], req.arrival, req.arrival, req.arrival,
                                      fp, "rejected: footprint exceeds the HBM budget"))
                continue
            wait = req.arrival - (self.clock() - t0)
            if wait > 0:
                time.sleep(wait)
            with cv:
                while not (state["free_slots"] and
                           (self.hbm_budget is None or state["in_use"] + fp <= self.hbm_budget)):
                    cv.wait()
                slot = state["free_slots"].pop(0)
                state["inflight"] += 1
                state["in_use"] += fp
                admitted = self.clock() - t0
                self.trace.append((admitted, state["in_use"], state["inflight"]))
            th = threading.Thread(target=worker, args=(req, slot, fp, admitted), daemon=True)
            th.start()
            threads.append(th)
        for th in threads:
            th.join()
        wall = self.clock() - t0
        return sorted(results, key=lambda r: r.rid), self._stats(reqs, results, wall)


    def run_waves(self, requests: Sequence[Request], execute_wave: Callable,
                  wave_slots: int = 2, max_wave: int = 16):
        """Continuous batching in waves.  Admission is as in run() (arrival order, HBM
        budget, first come first served); admitted requests queue, and each of
        `wave_slots` wave workers takes every queued request (up to `max_wave`) as one wave
        the moment it is free, so that requests arriving while waves are on the GPU join
        the next wave and two waves overlap on the device.  `execute_wave(requests, slot)`
        returns one (x blocks, iteration arrays, relres arrays[, finish time]) per request;
        a finish time (on this server's clock) makes that the request's finish, else the
        wave's return is.  Memory is released when the wave returns."""
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        t0 = self.clock()
        cv = threading.Condition()
        state = {"in_use": 0, "queue": [], "admitting": True, "busy": 0}
        results: List[Result] = []

        def wave_worker(slot: int):
            while True:
                with cv:
                    while not state["queue"] and state["admitting"]:
                        cv.wait()
                    if not state["queue"]:
                        return
                    wave = state["queue"][:max_wave]
                    del state["queue"][:len(wave)]
                    state["busy"] += 1
                outs, err = None, None
                try:
                    outs = execute_wave([w[0] for w in wave], slot)
                except Exception as e:   # a failed wave frees its requests' memory
                    err = f"{type(e).__name__}: {e}"
                done = self.clock() - t0
                with cv:
                    for k, (req, fp, admitted) in enumerate(wave):
                        out = outs[k] if outs is not None else ([], [], [])
                        xs, its, rrs = out[:3]
                        fin = done
                        if len(out) > 3 and out[3] is not None:
                            fin = min(done, out[3] - t0)
                        results.append(Result(req.rid, xs, its, rrs, req.arrival, admitted, fin,
                                              fp, err))
                        state["in_use"] -= fp
                    state["busy"] -= 1
                    self.trace.append((done, state["in_use"], len(wave)))
                    cv.notify_all()

        workers = [threading.Thread(target=wave_worker, args=(k,), daemon=True)
                   for k in range(wave_slots)]
        for w in workers:
            w.start()
        for req in reqs:
            fp = int(self.footprint(req))
            if self.hbm_budget is not None and fp > self.hbm_budget:
                with cv:
                    results.append(Result(req.rid, [], [], [], req.arrival, req.arrival,
                                          req.arrival, fp, "rejected: footprint exceeds the HBM budget"))
                continue
            wait = req.arrival - (self.clock() - t0)
            if wait > 0:
                time.sleep(wait)
            with cv:
                while not (self.hbm_budget is None or state["in_use"] + fp <= self.hbm_budget):
                    cv.wait()
                state["in_use"] += fp
                admitted = self.clock() - t0
                state["queue"].append((req, fp, admitted))
                self.trace.append((admitted, state["in_use"], len(state["queue"])))
                cv.notify_all()
        with cv:
            state["admitting"] = False
            cv.notify_all()
        for w in workers:
            w.join()
        wall = self.clock() - t0
        return sorted(results, key=lambda r: r.rid), self._stats(reqs, results, wall)

    def _stats(self, reqs, results, wall):
        ok = [r for r in results if r.error is None]
        lat = [r.latency for r in ok]
        return {
            "requests": len(reqs), "completed": len(ok), "failed": len(results) - len(ok),
            "wall_s": wall, "requests_per_s": len(ok) / wall if wall > 0 else float("nan"),
            "p50_latency_s": percentile(lat, 50), "p99_latency_s": percentile(lat, 99),
            "mean_latency_s": float(np.mean(lat)) if lat else float("nan"),
            "max_inflight": max((t[2] for t in self.trace), default=0),
            "max_in_use_bytes": max((t[1] for t in self.trace), default=0),
        }


class GpuExecutor:
    """Runs a request through the C ABI on one CUDA stream per worker slot; points and
    right-hand sides are host arrays (staged by the library), solutions come back to the
    host."""

    def __init__(self, slots: int):
        import torch
        self.torch = torch
        self.streams = [torch.cuda.Stream() for _ in range(slots)]

    def __call__(self, req: Request, slot: int):
        from . import api
        torch = self.torch
        s = self.streams[slot]
        with torch.cuda.stream(s):
            h = api.H2(np.ascontiguousarray(req.points, dtype=np.float64), req.kernel, req.ell,
                       req.shift, req.leaf_size, req.tol, stream=s)
            hs = api.HSS(h, req.rank, req.oversample, seed=req.seed, stream=s)
            u = api.ULV(hs, stream=s)
            xs, its, rrs = [], [], []
            for b in req.rhs:
                x, it, rr = api.pcg_solve(h, u, np.asfortranarray(b), tol=req.relres,
                                          maxit=req.maxit, stream=s)
                xs.append(np.asarray(x).copy())
                its.append(it)
                rrs.append(rr)
            u.close()
            hs.close()
            h.close()
        return xs, its, rrs


class WaveExecutor:
    """Runs a wave of requests through the batched C ABI on one CUDA stream per wave slot:
    spdhss_build_batched (H^2, SPD-HSS in the given precision mode, ULV, with the batched
    kernel launches of all requests of the wave merged step by step), then, for every block
    of right-hand sides, the iterations of all requests in lockstep: in the precision mode
    (precision >= 1) pcg_solve_batched_mixed (FP32 H^2 products, FP64 preconditioner and
    residuals; blocks of at most 16 columns), else pcg_solve_batched.  Every request's
    result equals the one it gets alone (a wave of one).  A request is finished when its
    last block's solution has reached the host, which the batched solve reports per request
    as soon as that request has converged (pcg_solve_batched_ex), not when the wave's
    slowest one has; its finish time (on `clock`, the server's clock) is returned with it.
    The wave's handles are released together at its end."""

    def __init__(self, slots: int, precision: int = 1, clock: Callable[[], float] = time.perf_counter):
        import torch
        self.torch = torch
        self.precision = int(precision)
        self.clock = clock
        self.streams = [torch.cuda.Stream() for _ in range(slots)]

    def __call__(self, reqs: Sequence[Request], slot: int):
        from . import api
        torch = self.torch
        s = self.streams[slot]
        insts = [dict(points=np.ascontiguousarray(r.points, dtype=np.float64), kernel=r.kernel,
                      ell=r.ell, shift=r.shift, leaf_size=r.leaf_size, tol=r.tol, rank=r.rank,
                      oversample=r.oversample, seed=r.seed, precision=self.precision)
                 for r in reqs]
        outs = [([], [], []) for _ in reqs]
        fin = [None] * len(reqs)
        with torch.cuda.stream(s):
            built, status, _ = api.build_batched(insts, stream=s)
            bad = [k for k, v in enumerate(status) if v != 0]
            if bad:
                raise RuntimeError(f"requests {[reqs[k].rid for k in bad]} failed to build")
            nblk = max(len(r.rhs) for r in reqs)
            for j in range(nblk):
                ks = [k for k, r in enumerate(reqs) if j < len(r.rhs)]
                mixed = self.precision > 0 and all(
                    np.asarray(reqs[k].rhs[j]).reshape(reqs[k].unknowns, -1).shape[1] <= 16
                    for k in ks)
                got = {}

                def done(i, status, x, it, rr, ks=ks, j=j):
                    k = ks[i]
                    got[k] = x.cpu().numpy()
                    if j == len(reqs[k].rhs) - 1:
                        fin[k] = self.clock()

                X, its, rrs, st = api.pcg_solve_batched(
                    [built[k][0] for k in ks], [built[k][2] for k in ks],
                    [np.asfortranarray(reqs[k].rhs[j]) for k in ks], tol=reqs[ks[0]].relres,
                    maxit=reqs[ks[0]].maxit, stream=s, mixed=mixed, on_done=done)
                for k, x, it, rr in zip(ks, X, its, rrs):
                    outs[k][0].append(got[k] if k in got else x.cpu().numpy())
                    outs[k][1].append(it)
                    outs[k][2].append(rr)
                    if fin[k] is None and j == len(reqs[k].rhs) - 1:
                        fin[k] = self.clock()
            for h, hs, u in built:
                u.close()
                hs.close()
                h.close()
        return [(xs, its, rrs, fin[k]) for k, (xs, its, rrs) in enumerate(outs)]


def synthetic_stream(count: int, rate: float, n_lo: int, n_hi: int, seed: int = 1,
                     nrhs_max: int = 16, rank: int = 50, shift: float = 1e-3,
                     blocks: int = 1) -> List[Request]:
    """Poisson arrivals (mean `rate` per second), n log-uniform in [n_lo, n_hi], 2D and 3D
    alternating, kernels cycled over {exponential, Gaussian ell=0.1, Matern-3/2 ell=0.1},
    1..nrhs_max right-hand sides N(0,1) per block."""
    from . import inputs
    g = np.random.Generator(np.random.Philox(key=[int(seed), 77]))
    gaps = g.exponential(1.0 / rate, count)
    arrivals = np.cumsum(gaps) - gaps[0]
    sizes = inputs.log_uniform_sizes(count, n_lo, n_hi, seed)
    kinds = [("exp", 1.0), ("gauss", 0.1), ("matern32", 0.1)]
    reqs = []
    for k in range(count):
        dim = 2 if k % 2 == 0 else 3
        kern, ell = kinds[k % 3]
        n = int(sizes[k])
        nrhs = int(g.integers(1, nrhs_max + 1))
        pts = inputs.uniform_cube(n, dim, seed=1000 + k)
        rhs = [inputs.rhs(n, nrhs, seed=2000 + 10 * k + b) for b in range(blocks)]
        reqs.append(Request(rid=k, arrival=float(arrivals[k]), points=pts, kernel=kern, ell=ell,
                            shift=shift, leaf_size=64, tol=1e-8, rank=rank, seed=k, rhs=rhs))
    return reqs
