"""Benchmark: SPD-HSS build + PCG solves per second (relative residual 1e-6).

One step = the whole hot path on one synthetic instance: cluster tree and proxy-point H^2
(h2_build), SPD-HSS construction (spdhss_build, Alg. 5.3), ULV factorization (ulv_factor)
and a PCG solve (pcg_solve) to relative residual 1e-6.

Headline workload: n = 4096 points uniform in [0,1]^3, kernel exp(-|x-y|) plus 1e-2 I, leaf
size 64, H^2 tolerance 1e-8, HSS rank 50, oversampling 10, one RHS ~ N(0,1).
The line also carries measured components of the n = 200,000 Gaussian workload
(exp(-|x-y|^2/0.01) + 1e-4 I, leaf 128, rank 50, 8 RHS): H^2 / SPD-HSS / ULV build times,
the 8-column H^2 product and the cost of one PCG iteration.  PCG on that system does not
reach relres 1e-6 within 3000 iterations (the method's iteration count, not a kernel
limit), so its build+solve rate is not a finite-time benchmark.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  --impl reference times the CPU oracle on the host cores (bounded
sample of the same workload).  Multi-GPU runs (torchrun) are independent replicas.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = dict(workload="spdhss_build_pcg_exp3d_n4096", n=4096, dim=3, kernel="exp", ell=1.0,
                shift=1e-2, leaf_size=64, h2_tol=1e-8, rank=50, oversample=10, nrhs=1,
                relres=1e-6, maxit=3000, points="uniform [0,1]^3 seed 0 (+rank)",
                rhs="N(0,1) seed 1 (+rank)")
AT_SCALE = dict(workload="gauss3d_n200000_components", n=200_000, dim=3, kernel="gauss", ell=0.1,
                shift=1e-4, leaf_size=128, h2_tol=1e-8, rank=50, oversample=10, nrhs=8,
                relres=1e-6, pcg_probe_iters=25)
METRIC = "SPD-HSS build+PCG solves/s at relres 1e-6"
UNIT = "build+solve/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--rank", type=int, default=WORKLOAD["rank"])
    # --problem-size: the same option under a name that torchrun's parser does not take for
    # an abbreviation of its own --nnodes / --nproc-per-node
    ap.add_argument("--n", "--problem-size", dest="n", type=int, default=WORKLOAD["n"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-at-scale", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve", type=int, default=0,
                    help="serving mode: this many Poisson-arriving mixed requests, served one at "
                         "a time and then concurrently; prints a serving JSON line")
    ap.add_argument("--tol-sweep", action="store_true",
                    help="tolerance-driven SPD-HSS on the paper's Matern ball/sphere "
                         "workload: PCG iterations and matvec errors at tau 1e-1 and 1e-2")
    ap.add_argument("--rpy-sweep", type=str, default=None, metavar="N1,N2,...",
                    help="the paper's RPY iteration runs at these particle counts")
    ap.add_argument("--rank-sweep", action="store_true",
                    help="fixed ranks 100 and 200 on the paper's Matern ball/sphere workload")
    ap.add_argument("--sweep-kernel", default="matern32", choices=["matern32", "gauss", "imq"],
                    help="kernel of --kernel-sweep")
    ap.add_argument("--kernel-sweep", action="store_true",
                    help="block Jacobi and SPD-HSS r=100 over the Matern parameter l on the "
                         "paper's 320,000-point ball")
    ap.add_argument("--paper-table", action="store_true",
                    help="the paper's timing-table workload (320,000 points in a ball, three "
                         "kernels, r = 100 and 200) on one GPU")
    ap.add_argument("--batch", type=int, default=0,
                    help="batched level sweep: this many independent instances built and solved "
                         "with merged launches, then one at a time; prints a batching JSON line")
    ap.add_argument("--matvec-case", type=int, default=0,
                    help="profiling case: H2 of the Gaussian workload at this n, then 5 products "
                         "with 8 columns (prints timings, no benchmark line)")
    ap.add_argument("--precision", action="store_true",
                    help="the precision workload (n = 500,000 Matern-3/2, rank 100) as its own line")
    ap.add_argument("--n-precision", type=int, default=500_000)
    ap.add_argument("--mixed", action="store_true",
                    help="with --matvec-case: also 5 FP32 products (mixed precision)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------------------
# CPU oracle leg (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------------------
def oracle_step(n, cfg, seed=0):
    from oracle import h2 as OH
    from oracle import pcg as OP
    from oracle import spdhss as OS
    from oracle import tree as OT
    from oracle import ulv as OU
    from oracle import kernels as OK
    from paper_2011_07632_gb300 import inputs
    X = inputs.uniform_cube(n, 3, seed)
    tr = OT.build_tree(X, cfg["leaf_size"])
    h = OH.build_h2(tr, X, OK.NAMES[cfg["kernel"]], cfg["ell"], cfg["shift"], cfg["h2_tol"])
    M = OH.dense(h)
    Om = inputs.sketch(n, cfg["rank"] + cfg["oversample"], 2)[tr.perm]
    hss = OS.build_spdhss(tr, M, Om, cfg["rank"])
    u = OU.ULV(hss)
    b = inputs.rhs(n, cfg["nrhs"], 1)[tr.perm]
    x, it, rr = OP.pcg(lambda v: M @ v, u.solve, b, cfg["relres"], cfg["maxit"])
    return int(it.max())


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(cfg, steps=3):
    t0 = time.perf_counter()
    its = []
    for s in range(steps):
        its.append(oracle_step(cfg["n"], cfg, seed=s))
    dt = (time.perf_counter() - t0) / steps
    return {"value": 1.0 / dt, "unit": UNIT, "cores": cores(), "kind": "oracle",
            "sample": f"the full workload (n={cfg['n']}), {steps} build+solve passes with point "
                      f"seeds 0..{steps-1}, {dt:.2f} s each, PCG iterations {its}"}


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            return
    cfg = dict(WORKLOAD)
    cfg["n"] = args.n
    for _ in range(max(0, args.warmup)):
        pass   # the oracle has no warm-up state; warm-up steps are not repeated on the CPU
    t0 = time.perf_counter()
    its = []
    for s in range(args.steps):
        its.append(oracle_step(cfg["n"], cfg, seed=s))
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    v = 1.0 / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores(), "kind": "oracle",
                             "sample": f"the full workload (n={cfg['n']}) per step, dense oracle, "
                                       f"PCG iterations {its}"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"spdhss_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}",
                                          f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def roof_hbm(st):
    """HBM roofline of a kernel family from its per-launch algorithmic bytes and time."""
    if not st or st["ms"] <= 0:
        return None
    peak = 6801.7
    try:
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except Exception:
        pass
    gbs = st["bytes"] / (st["ms"] / 1e3) / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "tflops": st["flops"] / (st["ms"] / 1e3) / 1e12}


def roof_product_f32(info, c, ms):
    """HBM roofline of the whole FP32 H^2 product (the public call, permutations and
    conversions included) on its algorithmic bytes: the FP32 generators (bases and every
    coupling once), x and y in FP32, and the coordinates the near field is evaluated from."""
    peak = 6801.7
    try:
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except Exception:
        pass
    nbytes = info["stored_bytes"] / 2 + 4 * 2 * c["n"] * c["nrhs"] + 8 * 3 * c["n"]
    gbs = nbytes / (ms / 1e3) / 1e9
    return {"bound": "hbm", "bytes": nbytes, "ms": ms, "achieved": gbs, "peak": peak,
            "unit": "GB/s", "frac": gbs / peak}


def run_at_scale(api, native, torch, dev, stream, fp64_peak):
    """Components of the n = 200,000 Gaussian workload, each timed with CUDA events."""
    from paper_2011_07632_gb300 import inputs
    c = AT_SCALE
    pts = torch.from_numpy(inputs.uniform_cube(c["n"], 3, 0)).to(dev)
    B = torch.from_numpy(np.ascontiguousarray(inputs.rhs(c["n"], c["nrhs"], 1))).to(dev)

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    h, t_h2 = timed(lambda: api.H2(pts, c["kernel"], c["ell"], c["shift"], c["leaf_size"], c["h2_tol"]))
    hs, t_hss = timed(lambda: api.HSS(h, c["rank"], c["oversample"], seed=7))
    u, t_ulv = timed(lambda: api.ULV(hs))
    h.matmul(B)
    native.lib().spdhss_profile(1)
    reps = 3
    _, t_mv = timed(lambda: [h.matmul(B) for _ in range(reps)])
    prof = native.profile_report()
    native.lib().spdhss_profile(0)
    u.solve(B)
    _, t_us = timed(lambda: [u.solve(B) for _ in range(reps)])
    k = c["pcg_probe_iters"]
    (x, it, rr), t_pcg = timed(lambda: api.pcg_solve(h, u, B, tol=c["relres"], maxit=k))
    # mixed precision: FP32 copy of the H^2 generators, FP64 preconditioner and residuals
    h.matmul_mixed(B)
    native.lib().spdhss_profile(1)
    _, t_mv32 = timed(lambda: [h.matmul_mixed(B) for _ in range(reps)])
    prof32 = native.profile_report()
    native.lib().spdhss_profile(0)
    (x2, it2, rr2), t_pcg32 = timed(lambda: api.pcg_solve(h, u, B, tol=c["relres"], maxit=k, mixed=True))
    info = h.info()
    prec = precision_build_record(api, native, torch, h, hs, c, timed, c["n"])
    # where the construction's time goes: a second, profiled build (library CUDA events)
    u.close(); hs.close(); h.close()
    del u, hs, h
    torch.cuda.synchronize()
    native.lib().spdhss_profile(1)
    h = api.H2(pts, c["kernel"], c["ell"], c["shift"], c["leaf_size"], c["h2_tol"])
    hs = api.HSS(h, c["rank"], c["oversample"], seed=7)
    u = api.ULV(hs)
    torch.cuda.synchronize()
    profb = native.profile_report()
    native.lib().spdhss_profile(0)
    build_kernels = {k2: round(v["ms"], 1) for k2, v in
                     sorted(profb.items(), key=lambda kv: -kv[1]["ms"])[:10]}
    u.close(); hs.close(); h.close()
    cp = prof.get("h2_coupling", {"ms": 0.0, "flops": 0.0, "launches": 1})
    ach = cp["flops"] / max(cp["launches"], 1) / (cp["ms"] / max(cp["launches"], 1) / 1e3) / 1e12
    out = {
        "config": c, "h2_build_ms": t_h2, "spdhss_build_ms": t_hss, "ulv_factor_ms": t_ulv,
        "build_total_ms": t_h2 + t_hss + t_ulv,
        "h2_matmul_8rhs_ms": t_mv / reps, "ulv_solve_8rhs_ms": t_us / reps,
        "pcg_ms_per_iteration": t_pcg / max(int(it.max()), 1), "pcg_probe_iterations": int(it.max()),
        "pcg_relres_after_probe": float(rr.max()),
        "pcg_note": "relres 1e-6 is not reached within 3000 iterations for this system at rank 20, "
                    "50 or 100 (measured); the probe only prices one iteration",
        "build_kernels_ms": build_kernels,
        "h2_stored_gb": info["stored_bytes"] / 1e9, "h2_max_rank": info["max_rank"],
        "h2_coupling_entries": info["coupling_entries"],
        "h2_matmul_gbs": (info["stored_bytes"] + 2 * 8 * c["n"] * c["nrhs"]) / (t_mv / reps / 1e3) / 1e9,
        "roofline_h2_coupling": {"bound": "alu", "achieved": ach, "peak": fp64_peak,
                                 "unit": "TFLOP/s", "frac": ach / fp64_peak,
                                 "share_of_matmul": cp["ms"] / max(sum(v["ms"] for v in prof.values()), 1e-9)},
        "mixed": {
            "h2_matmul_8rhs_fp32_ms": t_mv32 / reps,
            "pcg_ms_per_iteration": t_pcg32 / max(int(it2.max()), 1),
            "pcg_relres_after_probe": float(rr2.max()),
            "roofline_h2_coupling_f32": roof_hbm(prof32.get("h2_coupling_f32")),
            "roofline_h2_product_f32": roof_product_f32(info, c, t_mv32 / reps),
            "kernels": {k2: round(v["ms"] / reps, 3) for k2, v in prof32.items()},
        },
        "precision_build": prec,
    }
    u.close(); hs.close(); h.close()
    del pts, B
    torch.cuda.empty_cache()
    return out


def tf32_peak():
    """Dense TF32 tensor peak: the measured bf16 figure times TF32's nominal ratio (1/2)."""
    pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    return pk["bf16_tflops"] / 2.0, "measured bf16 x 1/2 (nominal TF32:BF16 dense ratio)"


def precision_build_record(api, native, torch, h, hs64, c, timed, n):
    """The precision mode of the construction on an H^2 matrix already built: the sampling
    product in FP32 with tensor-core (3xTF32) GEMMs, FP64 afterwards.  Its build time next
    to the FP64 one, where the time goes, the tensor-core coupling GEMM against the TF32
    peak, and the difference of the two HSS matrices on random vectors."""
    from paper_2011_07632_gb300 import inputs
    hs1, t1 = timed(lambda: api.HSS(h, c["rank"], c["oversample"], seed=7, precision=1))
    hs1.close()
    native.lib().spdhss_profile(1)
    hs1, t1b = timed(lambda: api.HSS(h, c["rank"], c["oversample"], seed=7, precision=1))
    prof = native.profile_report()
    native.lib().spdhss_profile(0)
    x = inputs.rhs(n, 4, 21)
    y64 = hs64.matmul(x).cpu().numpy()
    y1 = hs1.matmul(x).cpu().numpy()
    hs1.close()
    diff = float(np.linalg.norm(y1 - y64) / np.linalg.norm(y64))
    tc = prof.get("h2_coupling_sample_tc", {"ms": 0.0, "flops": 0.0})
    peak, src = tf32_peak()
    ach = tc["flops"] / max(tc["ms"], 1e-9) / 1e9   # algorithmic TFLOP/s (FP32-accurate products)
    return {"spdhss_build_ms": t1, "spdhss_build_profiled_ms": t1b,
            "hss_product_rel_diff_vs_fp64": diff,
            "kernels_ms": {k: round(v["ms"], 2) for k, v in
                           sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:8]},
            "roofline_coupling_tc": {"bound": "tensor", "kernel": "k_gemm_tf32 (3xTF32)",
                                     "achieved": ach, "achieved_tf32_mma": 3 * ach,
                                     "peak": peak, "peak_source": src, "unit": "TFLOP/s",
                                     "frac": 3 * ach / peak}}


def run_precision(args):
    """The precision workload: n = 500,000 points uniform in [0,1]^3, Matern-3/2 (ell 0.1)
    + 1e-3 I, leaf 128, H^2 tol 1e-8, rank 100, one RHS N(0,1); a step is h2_build +
    spdhss_build in the precision mode (FP32 sampling, tensor-core GEMMs) + ulv_factor +
    FP64 PCG to relres 1e-6, inputs resident on the device.  Also once, outside the timed
    steps, the FP64 construction of the same H^2 matrix for comparison."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_07632_gb300 import api, inputs, native
    c = dict(workload="precision_matern3d_n%d" % args.n_precision, n=args.n_precision, dim=3,
             kernel="matern32", ell=0.1, shift=1e-3, leaf_size=128, h2_tol=1e-8, rank=100,
             oversample=10, nrhs=1, relres=1e-6, maxit=3000, precision="fp32 sampling (3xTF32 "
             "tensor-core GEMMs), fp64 compression / factors / PCG",
             points="uniform [0,1]^3 seed 0", rhs="N(0,1) seed 1", l2="inputs larger than L2")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    pts = torch.from_numpy(inputs.uniform_cube(c["n"], 3, 0)).to(dev)
    b = torch.from_numpy(np.ascontiguousarray(inputs.rhs(c["n"], 1, 1))).to(dev)

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    def step():
        e0 = ev()
        h = api.H2(pts, c["kernel"], c["ell"], c["shift"], c["leaf_size"], c["h2_tol"])
        e1 = ev()
        hs = api.HSS(h, c["rank"], c["oversample"], seed=7, precision=1)
        e2 = ev()
        u = api.ULV(hs)
        e3 = ev()
        x, it, rr = api.pcg_solve(h, u, b, tol=c["relres"], maxit=c["maxit"])
        e4 = ev()
        torch.cuda.synchronize()
        parts = [e0.elapsed_time(e1), e1.elapsed_time(e2), e2.elapsed_time(e3), e3.elapsed_time(e4)]
        u.close(); hs.close(); h.close()
        return parts, int(it[0]), float(rr[0])

    for _ in range(args.warmup):
        step()
    mon = ClockSampler(0)
    parts_all, its = [], []
    with mon:
        torch.cuda.synchronize()
        t0 = ev()
        for _ in range(args.steps):
            parts, it, rr = step()
            parts_all.append(parts)
            its.append(it)
        t1 = ev()
        torch.cuda.synchronize()
    total = t0.elapsed_time(t1)
    # the FP64 construction of the same matrix, once (context for the precision mode)
    h = api.H2(pts, c["kernel"], c["ell"], c["shift"], c["leaf_size"], c["h2_tol"])
    e0 = ev()
    hs64 = api.HSS(h, c["rank"], c["oversample"], seed=7)
    e1 = ev()
    torch.cuda.synchronize()
    t64 = e0.elapsed_time(e1)

    def timed(fn):
        a = ev()
        out = fn()
        z = ev()
        torch.cuda.synchronize()
        return out, a.elapsed_time(z)

    prec = precision_build_record(api, native, torch, h, hs64, c, timed, c["n"])
    hs64.close(); h.close()
    ms = total / args.steps
    mean = np.mean(np.array(parts_all), axis=0)
    print(json.dumps({
        "metric": METRIC, "value": 1e3 / ms, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32/tf32", "data": "synthetic", "config": c,
        "components_ms": {"h2_build": mean[0], "spdhss_build_precision": mean[1],
                          "ulv_factor": mean[2], "pcg": mean[3]},
        "pcg_iters": its, "pcg_relres": rr, "spdhss_build_fp64_ms": t64,
        "precision_build": prec, "clocks": mon.summary()}))


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of a kernel family on
# the n = 4096 workload, from one ncu capture.  Each entry names the source files of the
# family's kernels and a fingerprint of their text at the time of the capture: when the
# files have changed since, the bench reports the traffic as null (stale capture).
DRAM_TRAFFIC = {
    # k_proxy_qr (profiles/launches_headline_exp3d_n4096.md): leaf level 0.324 MB read +
    # 0.022 MB written, depth 2 0.343 MB + 0.375 MB; the family's two launches per step
    "qr_h2_id_blocks": {"bytes": (324352 + 22016 + 343040 + 375040) // 2,
                        "sources": ["csrc/keval.cu", "csrc/keval.cuh", "csrc/common.cuh",
                                    "csrc/dense.cuh"],
                        "sha16": "e9ccf92b8878d5d0"},
}


def source_fingerprint(files):
    """First 16 hex digits of the SHA-256 of the given package source files, in order."""
    import hashlib
    hsh = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2011_07632_gb300", f), "rb") as fh:
            hsh.update(fh.read())
    return hsh.hexdigest()[:16]


def measured_traffic(family):
    """Per-launch DRAM bytes of a family from the capture table, or None when there is no
    capture or the kernels' sources changed after it."""
    e = DRAM_TRAFFIC.get(family)
    if not e:
        return None
    try:
        if source_fingerprint(e["sources"]) != e["sha16"]:
            return None
    except OSError:
        return None
    return e["bytes"]


def family_table(prof, fp64_peak):
    """Per kernel family of the timed steps (library event timing): total ms, launches and,
    where the family records its algorithmic FP64 flops, the achieved TFLOP/s and its
    fraction of the FP64 peak; largest time first."""
    out = {}
    for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"]):
        row = {"ms": round(v["ms"], 3), "launches": v["launches"]}
        if v.get("flops", 0.0) > 0.0 and v["ms"] > 0.0:
            tf = v["flops"] / (v["ms"] / 1e3) / 1e12
            row["tflops"] = round(tf, 4)
            row["fp64_frac"] = round(tf / fp64_peak, 4)
        out[k] = row
    return out


def replica_throughput(total_ms, steps, world, dist=None, device=None):
    """Whole-job throughput of `world` independent replicas that each ran `steps` steps in
    `total_ms` of their own device time: the job lasts as long as the slowest rank (max over
    ranks), and its value is all ranks' steps over that time.  Returns (job ms, steps/s)."""
    if dist is not None:
        import torch
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    return total_ms, (steps * world) / (total_ms / 1e3)


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_07632_gb300 import api, inputs, native

    cfg = dict(WORKLOAD)
    cfg["n"], cfg["rank"] = args.n, args.rank
    n, nrhs = cfg["n"], cfg["nrhs"]
    dev = torch.device("cuda", torch.cuda.current_device())
    # the step runs on a stream of its own (the library captures steady PCG iterations as
    # CUDA graphs on a caller stream; the legacy default stream cannot be captured)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    pts_h = inputs.uniform_cube(n, 3, 0 + rank)
    b_h = inputs.rhs(n, nrhs, 1 + rank)
    pts = torch.from_numpy(pts_h).to(dev)
    B = torch.from_numpy(np.ascontiguousarray(b_h)).to(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    native.lib().spdhss_profile(0)

    def step(pts_in, B_in):
        h = api.H2(pts_in, cfg["kernel"], cfg["ell"], cfg["shift"], cfg["leaf_size"], cfg["h2_tol"])
        hs = api.HSS(h, cfg["rank"], cfg["oversample"], seed=7)
        u = api.ULV(hs)
        x, it, rr = api.pcg_solve(h, u, B_in, tol=cfg["relres"], maxit=cfg["maxit"])
        info = h.info()
        hinfo = hs.info()
        u.close(); hs.close(); h.close()
        return x, it, rr, info, hinfo

    for _ in range(args.warmup):
        step(pts, B)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = native.launch_count()
    native.lib().spdhss_profile(1)
    ev = []
    iters = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x, it, rr, info, hinfo = step(pts, B)
            e1.record(stream)
            ev.append((e0, e1))
            iters.append(int(it.max()))
        torch.cuda.synchronize()
    launches = native.launch_count() - launches0
    prof = native.profile_report()
    native.lib().spdhss_profile(0)
    times = [a.elapsed_time(b) for a, b in ev]
    total_ms, value = replica_throughput(float(sum(times)), args.steps, world, dist, dev)
    torch.cuda.synchronize()

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if args.e2e_steps > 0:
        # inputs in pinned host memory; the library copies them in and the solution out
        pts_host = torch.from_numpy(np.ascontiguousarray(pts_h)).pin_memory()
        b_host = torch.from_numpy(np.ascontiguousarray(b_h)).pin_memory()
        tot = 0.0
        for _ in range(args.e2e_steps):
            flush.zero_()                 # L2 flushed between steps, outside the timing
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = api.H2(pts_host, cfg["kernel"], cfg["ell"], cfg["shift"], cfg["leaf_size"], cfg["h2_tol"])
            hs = api.HSS(h, cfg["rank"], cfg["oversample"], seed=7)
            u = api.ULV(hs)
            xh, ith, rrh = api.pcg_solve(h, u, b_host, tol=cfg["relres"], maxit=cfg["maxit"])
            torch.cuda.synchronize()
            tot += time.perf_counter() - t0
            u.close(); hs.close(); h.close()
        dt = tot / args.e2e_steps
        e2e = {"value": world / dt, "unit": UNIT, "h2d_bytes_per_step": int(pts_h.nbytes + b_h.nbytes),
               "d2h_bytes_per_step": int(b_h.nbytes)}
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel family (FP64 ALU bound; peak from the FMA unit count)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    fp64_peak = 152 * 2 * 2 * (peaks.get("sm_max_mhz", 2070.0) * 1e6) / 1e12   # TFLOP/s
    top = max(prof, key=lambda k: prof[k]["ms"]) if prof else None
    if top is not None and prof[top]["flops"] <= 0:
        with_flops = [k for k in prof if prof[k]["flops"] > 0]
        top = max(with_flops, key=lambda k: prof[k]["ms"]) if with_flops else top
    roof = None
    if top is not None:
        st = prof[top]
        per_launch_ms = st["ms"] / max(st["launches"], 1)
        achieved = (st["flops"] / max(st["launches"], 1)) / (per_launch_ms / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": top, "achieved": achieved, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                "traffic": measured_traffic(top),
                "peak_source": "FP64 FMA units: 152 SMs x 2 FMA/clk x 2 flop x max SM clock",
                "share_of_step": st["ms"] / max(total_ms, 1e-9),
                "launches_per_step": st["launches"] / args.steps}
    at_scale = None if args.no_at_scale else run_at_scale(api, native, torch, dev, stream, fp64_peak)
    serving = None if args.no_serving or rank != 0 else serving_comparison(args.serve_requests)
    cb = None
    if not args.no_cpu_baseline:
        cb = cpu_baseline(cfg, steps=3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(cfg, parallelism=f"replicas{world}" if world > 1 else "single",
                       l2="256 MB buffer written between timed steps"),
        "p50_ms": float(np.percentile(times, 50)), "p99_ms": float(np.percentile(times, 99)),
        "rhs_solves_per_s": value * nrhs, "pcg_iters": iters,
        "h2": {k: info[k] for k in ("nodes", "D", "max_rank", "stored_bytes", "coupling_entries",
                                    "near_kernel_entries")},
        "hss": hinfo,
        "gpu_launches": int(launches), "roofline": roof, "cpu_baseline": cb, "e2e": e2e,
        "at_scale": at_scale, "serving": serving,
        "clocks": clk.summary(), "kernels": family_table(prof, fp64_peak),
        "tuning": native.tuning_report(),
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_matvec_case(n, mixed=False):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_07632_gb300 import api, inputs
    c = AT_SCALE
    pts = torch.from_numpy(inputs.uniform_cube(n, 3, 0)).cuda()
    B = torch.from_numpy(np.ascontiguousarray(inputs.rhs(n, c["nrhs"], 1))).cuda()
    h = api.H2(pts, c["kernel"], c["ell"], c["shift"], c["leaf_size"], c["h2_tol"])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h.matmul(B)
    e0.record()
    for _ in range(5):
        h.matmul(B)
    e1.record()
    torch.cuda.synchronize()
    out = {"case": "h2_matmul_8rhs", "n": n, "ms": e0.elapsed_time(e1) / 5, "h2": h.info()}
    if mixed:
        h.matmul_mixed(B)
        e0.record()
        for _ in range(5):
            h.matmul_mixed(B)
        e1.record()
        torch.cuda.synchronize()
        out["fp32_ms"] = e0.elapsed_time(e1) / 5
    print(json.dumps(out))


SERVE_WORKLOAD = "poisson200_n1000-16000_2d3d_exp-gauss-matern_rank50_rhs1-16"


def serving_comparison(count, waves_only_stats=False):
    """The serving workload (Poisson arrivals at 200 requests/s, seed 1; n log-uniform in
    [1000, 16000]; 2D and 3D alternating; kernels cycled {exp, Gaussian ell=0.1, Matern-3/2
    ell=0.1}; shift 1e-3; rank 50; 1..16 right-hand sides) served two ways on the same GPU:
    plain FP64, one request at a time; and the served mixed-precision batched form (waves
    of the requests admitted meanwhile, merged construction launches with the tensor-core
    sampling, lockstep PCG with the FP32 H^2 products merged over the wave, two waves
    overlapping).  Latency = arrival to last solution on the host."""
    import torch
    from paper_2011_07632_gb300 import serve
    reqs = serve.synthetic_stream(count, rate=200.0, n_lo=1000, n_hi=16000, seed=1)
    warm = [serve.Request(**{**r.__dict__, "arrival": 0.0}) for r in reqs[:3]]
    serve.Server(serve.GpuExecutor(1), slots=1).run(warm)
    serve.Server(None).run_waves(warm, serve.WaveExecutor(1, precision=1), wave_slots=1)
    free = torch.cuda.mem_get_info()[0]
    one, st1 = serve.Server(serve.GpuExecutor(1), slots=1).run(reqs)
    wav, stw = serve.Server(None, hbm_budget=int(0.6 * free)).run_waves(
        reqs, serve.WaveExecutor(2, precision=1), wave_slots=2, max_wave=16)
    diff = max(float(np.linalg.norm(xw - xo) / max(np.linalg.norm(xo), 1e-300))
               for a, b in zip(one, wav) for xo, xw in zip(a.x, b.x))
    keys = ("requests", "completed", "failed", "wall_s", "requests_per_s", "p50_latency_s",
            "p99_latency_s", "max_inflight")
    return {"workload": SERVE_WORKLOAD, "requests": count,
            "fp64_one_at_a_time": {k: st1[k] for k in keys},
            "mixed_batched_waves": {k: stw[k] for k in keys},
            "speedup_requests_per_s": stw["requests_per_s"] / st1["requests_per_s"],
            "p99_ratio": stw["p99_latency_s"] / st1["p99_latency_s"],
            "max_rel_diff_mixed_vs_fp64_solutions": diff,
            "pcg_iters_fp64": [int(np.max(r.iters[0])) for r in one if r.iters],
            "pcg_iters_mixed": [int(np.max(r.iters[0])) for r in wav if r.iters]}


def run_serve(count):
    """--serve N: the serving comparison over N requests, plus 4 concurrent single-request
    streams (FP64) for context."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_07632_gb300 import serve
    out = serving_comparison(count)
    reqs = serve.synthetic_stream(count, rate=200.0, n_lo=1000, n_hi=16000, seed=1)
    free = torch.cuda.mem_get_info()[0]
    _, st4 = serve.Server(serve.GpuExecutor(4), slots=4, hbm_budget=int(0.6 * free)).run(reqs)
    out["fp64_concurrent_4_streams"] = st4
    print(json.dumps({"metric": "served build+solve requests/s, p50/p99 latency", **out,
                      "dtype": "f64 (+ fp32/tf32 sampling in the batched form)",
                      "data": "synthetic"}))


def batch_instances(count, seed=3):
    """Independent instances: n = floor(exp(U[ln 2000, ln 32000])), 2D and 3D alternating,
    kernels cycled over {exp, Gaussian ell=0.1, Matern-3/2 ell=0.1}, shift 1e-3, leaf 64,
    H^2 tol 1e-8, rank 50, one N(0,1) right-hand side each."""
    from paper_2011_07632_gb300 import inputs
    sizes = inputs.log_uniform_sizes(count, 2000, 32000, seed)
    kinds = [("exp", 1.0), ("gauss", 0.1), ("matern32", 0.1)]
    out = []
    for k in range(count):
        kind, ell = kinds[k % 3]
        dim = 2 if k % 2 == 0 else 3
        n = int(sizes[k])
        out.append(dict(points=inputs.uniform_cube(n, dim, 1000 + k), kernel=kind, ell=ell,
                        shift=1e-3, leaf_size=64, tol=1e-8, rank=50, oversample=10, seed=k,
                        rhs=inputs.rhs(n, 1, 5000 + k)))
    return out


def run_batch(count):
    """Batched level sweep (spdhss_build_batched + pcg_solve_batched) against the same
    instances built and solved one at a time on the same stream; then the batched solve
    with FP32 products (pcg_solve_batched_mixed) on the same construction."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_07632_gb300 import api, native
    insts = batch_instances(count)
    dev = [dict(i, points=torch.from_numpy(i["points"]).cuda(),
                rhs=torch.from_numpy(np.ascontiguousarray(i["rhs"])).cuda()) for i in insts]
    torch.cuda.synchronize()

    def batched(ins, mixed=False):
        t0 = time.perf_counter()
        built, st, stats = api.build_batched(ins)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        X, its, rrs, st2 = api.pcg_solve_batched([b[0] for b in built], [b[2] for b in built],
                                                 [i["rhs"] for i in ins], tol=1e-6, mixed=mixed)
        torch.cuda.synchronize()
        return built, st, stats, X, its, st2, t1 - t0, time.perf_counter() - t1

    def single(ins):
        xs, its, tb, ts = [], [], 0.0, 0.0
        for i in ins:
            t0 = time.perf_counter()
            h = api.H2(i["points"], i["kernel"], i["ell"], i["shift"], i["leaf_size"], i["tol"])
            hs = api.HSS(h, i["rank"], i["oversample"], seed=i["seed"])
            u = api.ULV(hs)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            x, it, rr = api.pcg_solve(h, u, i["rhs"], tol=1e-6)
            xs.append(x.cpu().numpy())
            ts += time.perf_counter() - t1
            tb += t1 - t0
            its.append(int(it[0]))
            u.close(); hs.close(); h.close()
        torch.cuda.synchronize()
        return xs, its, tb, ts

    batched(dev[:4])                     # warm-up
    single(dev[:2])
    c0 = native.launch_count()
    t0 = time.perf_counter()
    built, st, stats, X, its_b, st2, tb_b, ts_b = batched(dev)
    t_b = time.perf_counter() - t0
    c1 = native.launch_count()
    xb = [x.cpu().numpy() for x in X]
    del built, X
    torch.cuda.synchronize()
    c2 = native.launch_count()
    t0 = time.perf_counter()
    xs, its_s, tb_s, ts_s = single(dev)
    t_s = time.perf_counter() - t0
    c3 = native.launch_count()
    diff = max(float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)) for a, b in zip(xb, xs))
    batched(dev[:4], mixed=True)         # warm-up of the FP32 plans' first use
    c4 = native.launch_count()
    built_m, st_m, _, X_m, its_m, st2_m, tb_m, ts_m = batched(dev, mixed=True)
    c5 = native.launch_count()
    xm = [x.cpu().numpy() for x in X_m]
    del built_m, X_m
    diff_m = max(float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
                 for a, b in zip(xm, xb))
    im = [int(v[0]) for v in its_m]
    # device time of the batched kernels (library CUDA events), one more batched pass
    native.lib().spdhss_profile(1)
    res = batched(dev)
    prof = native.profile_report()
    native.lib().spdhss_profile(0)
    del res
    busy = sum(v["ms"] for v in prof.values()) / 1e3
    top = sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:8]
    ib = [int(v[0]) for v in its_b]
    print(json.dumps({
        "metric": "SPD-HSS build+PCG solves/s over independent instances",
        "workload": f"batch{count}_n2000-32000_mixed", "instances": count,
        "batched": {"wall_s": t_b, "instances_per_s": count / t_b, "build_s": tb_b,
                    "solve_s": ts_b, "gpu_launches": c1 - c0,
                    "build_merged_launches": stats[0], "build_hand_overs": stats[1],
                    "status_ok": sum(v == native.OK for v in st),
                    "converged": sum(v == native.OK for v in st2)},
        "one_at_a_time": {"wall_s": t_s, "instances_per_s": count / t_s, "build_s": tb_s,
                          "solve_s": ts_s, "gpu_launches": c3 - c2},
        "pcg_iters": {"batched_max": max(ib), "single_max": max(its_s),
                      "max_abs_diff": max(abs(a - b) for a, b in zip(ib, its_s))},
        "max_rel_diff_batched_vs_single": diff,
        "batched_mixed_pcg": {"solve_s": ts_m, "build_s": tb_m, "gpu_launches": c5 - c4,
                              "converged": sum(v == native.OK for v in st2_m),
                              "iters_max": max(im),
                              "iters_max_abs_diff_vs_fp64": max(abs(a - b) for a, b in zip(im, ib)),
                              "max_rel_diff_vs_fp64_solutions": diff_m},
        "batched_kernel_s": busy,
        "batched_top_kernels_ms": {k: round(v["ms"], 1) for k, v in top},
        "n_total": int(sum(i["points"].shape[0] for i in insts)),
        "dtype": "f64", "data": "synthetic"}))


def run_rank_sweep():
    """The paper's fixed-rank runs on the same Matern (l = 0.25) ball/sphere workload:
    r = 100 and 200, oversampling 10, and r = 0 (the block-Jacobi preconditioner of the
    paper's comparisons); the paper's PCG setting: right-hand side uniform on [-0.5, 0.5],
    relres 1e-4."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_07632_gb300 import api, inputs
    rows = []
    for pset in ("ball", "sphere"):
        for n in (40000, 80000):
            X = inputs.ball(n, 0) if pset == "ball" else inputs.sphere(n, 0)
            pts = torch.from_numpy(X).cuda()
            b = torch.from_numpy(np.ascontiguousarray(inputs.rhs_uniform(n, 1, 1))).cuda()
            h = api.H2(pts, "matern32", 4.0, 1e-2, 400, 1e-8)
            for r in (0, 100, 200):
                hs = api.HSS(h, r, 10, seed=2)
                u = api.ULV(hs)
                x, it, rr = api.pcg_solve(h, u, b, tol=1e-4, maxit=3000)
                rows.append({"points": pset, "n": n, "rank": r, "pcg_iters": int(it.max()),
                             "relres": float(rr.max())})
                u.close(); hs.close()
            h.close()
    print(json.dumps({"metric": "PCG iterations with fixed-rank SPD-HSS",
                      "workload": "matern32_l0.25_ball_sphere_n40k-80k", "rows": rows,
                      "dtype": "f64", "data": "synthetic"}))


def run_rpy_sweep(sizes):
    """The paper's RPY runs: particles of radius a = 0.29 and 0.42 (volume fractions about
    0.1 and 0.3 at the unit density of the ball of radius (3N/4pi)^(1/3); the sphere of
    radius (N/4pi)^(1/2) has unit surface density), 3N unknowns, no shift, H^2 tolerance
    1e-8, leaf boxes of up to 400 particles; no preconditioner, block Jacobi (rank 0) and
    SPD-HSS with r = 100 and 200 (oversampling 10); PCG to relres 1e-4 with a right-hand
    side uniform on [-0.5, 0.5]; also the H^2 and SPD-HSS construction times."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_07632_gb300 import api, inputs
    rows = []
    for pset in ("ball", "sphere"):
        for n in sizes:
            X = inputs.ball(n, 0) if pset == "ball" else inputs.sphere(n, 0)
            pts = torch.from_numpy(X).cuda()
            b = torch.from_numpy(np.ascontiguousarray(inputs.rhs_uniform(3 * n, 1, 1))).cuda()
            for a in (0.29, 0.42):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                h = api.H2(pts, "rpy", a, 0.0, 400, 1e-8)
                torch.cuda.synchronize()
                t_h2 = time.perf_counter() - t0
                row = {"points": pset, "n": n, "unknowns": 3 * n, "a": a,
                       "h2_build_s": round(t_h2, 3), "h2_max_rank": h.info()["max_rank"]}
                if n <= 40000:
                    x, it, rr = api.pcg_solve(h, None, b, tol=1e-4, maxit=3000)
                    row["none"] = int(it.max())
                for r in (0, 100, 200):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    hs = api.HSS(h, r, 10, seed=2)
                    u = api.ULV(hs)
                    torch.cuda.synchronize()
                    t_b = time.perf_counter() - t0
                    x, it, rr = api.pcg_solve(h, u, b, tol=1e-4, maxit=3000)
                    key = "bj" if r == 0 else "r%d" % r
                    row[key] = int(it.max())
                    if r:
                        row[key + "_build_s"] = round(t_b, 3)
                    assert float(rr.max()) <= 1e-4
                    u.close(); hs.close()
                rows.append(row)
                print(json.dumps(row), file=sys.stderr, flush=True)
                h.close()
                torch.cuda.empty_cache()
    print(json.dumps({"metric": "PCG iterations for RPY kernel matrices",
                      "workload": "rpy_a0.29-0.42_ball_sphere", "rows": rows,
                      "dtype": "f64", "data": "synthetic"}))


SWEEP_L = {"matern32": (0.001, 0.01, 0.1, 1.0),
           "gauss": (0.0001, 0.001, 0.01, 0.1, 1.0),
           "imq": (0.001, 0.01, 0.1, 1.0, 10.0, 100.0)}


def run_kernel_sweep(kind="matern32"):
    """The paper's parameter sweep: kernel matrices sigma I + K_l on 320,000 points in a
    ball (constant density), sigma 1e-2, leaf boxes of up to 400 points; block Jacobi
    (rank 0) and SPD-HSS with r = 100; PCG to relres 1e-4 with a right-hand side uniform on
    [-0.5, 0.5].  The paper's l multiplies the distance (Matern-3/2: length scale 1/l) or
    the squared distance (Gaussian, IMQ: length scale 1/sqrt(l))."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_07632_gb300 import api, inputs
    n = 320000
    pts = torch.from_numpy(inputs.ball(n, 0)).cuda()
    b = torch.from_numpy(np.ascontiguousarray(inputs.rhs_uniform(n, 1, 1))).cuda()
    rows = []
    for l in SWEEP_L[kind]:
        ell = 1.0 / l if kind == "matern32" else 1.0 / math.sqrt(l)
        h = api.H2(pts, kind, ell, 1e-2, 400, 1e-8)
        for r in (0, 100):
            hs = api.HSS(h, r, 10, seed=2)
            u = api.ULV(hs)
            x, it, rr = api.pcg_solve(h, u, b, tol=1e-4, maxit=3000)
            rows.append({"l": l, "rank": r, "pcg_iters": int(it.max()), "relres": float(rr.max())})
            u.close(); hs.close()
        h.close()
        torch.cuda.empty_cache()
    print(json.dumps({"metric": f"PCG iterations over the {kind} kernel parameter",
                      "workload": f"{kind}_ball_n320k_l{SWEEP_L[kind][0]}-{SWEEP_L[kind][-1]}",
                      "rows": rows, "dtype": "f64", "data": "synthetic"}))


def run_paper_table():
    """The paper's timing table setting: 320,000 points in a ball of radius (3N/4pi)^(1/3),
    shift 1e-2, H^2 tolerance 1e-8, leaf boxes of up to 400 points, oversampling 10; the
    Matern-3/2 kernel with l = 0.025, the Gaussian with l = 0.01 and the IMQ with l = 1
    (the paper's l; here length scales 40, 10 and 1); SPD-HSS with r = 100 and 200; PCG to
    relres 1e-4 with a right-hand side uniform on [-0.5, 0.5].  Times with CUDA events."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_07632_gb300 import api, inputs
    n = 320000
    pts = torch.from_numpy(inputs.ball(n, 0)).cuda()
    b = torch.from_numpy(np.ascontiguousarray(inputs.rhs_uniform(n, 1, 1))).cuda()

    def timed(fn, reps=1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        out = None
        for _ in range(reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / reps

    rows = []
    for kern, ell, lp in (("matern32", 40.0, 0.025), ("gauss", 10.0, 0.01), ("imq", 1.0, 1.0)):
        h, t_h2 = timed(lambda: api.H2(pts, kern, ell, 1e-2, 400, 1e-8))
        h.matmul(b)
        _, t_mv = timed(lambda: h.matmul(b), reps=5)
        info = h.info()
        row = {"kernel": kern, "paper_l": lp, "h2_build_s": t_h2 / 1e3, "h2_matvec_s": t_mv / 1e3,
               "h2_gb": info["stored_bytes"] / 1e9}
        for r in (100, 200):
            def build():
                hs = api.HSS(h, r, 10, seed=2)
                return hs, api.ULV(hs)
            (hs, u), t_b = timed(build)
            u.solve(b)
            _, t_s = timed(lambda: u.solve(b), reps=5)
            x, it, rr = api.pcg_solve(h, u, b, tol=1e-4, maxit=3000)
            row[f"r{r}"] = {"build_incl_ulv_s": t_b / 1e3, "apply_s": t_s / 1e3,
                            "hss_gb": hs.info()["stored_bytes"] / 1e9, "pcg_iters": int(it.max())}
            u.close(); hs.close()
        rows.append(row)
        h.close()
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "the paper's timing table on one GB300",
                      "workload": "ball_n320k_matern_gauss_imq", "rows": rows,
                      "dtype": "f64", "data": "synthetic"}))


def run_tol_sweep():
    """The paper's relative-tolerance experiment (Matern-3/2 with l = 0.25, i.e. length scale
    4, shift 1e-2, ball and sphere point sets of constant density): bases truncated at
    tau = 1e-1 and 1e-2 (largest ranks 200 and 600, the sketch growing from 64 + 10 columns
    as needed, oversampling 10), leaf boxes of up to 400
    points, H^2 tolerance 1e-8; PCG iterations to relres 1e-4 with a right-hand side uniform
    on [-0.5, 0.5] (the paper's setting) and the average relative error of the SPD-HSS
    product against the H^2 product over 4 random vectors."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_07632_gb300 import api, inputs
    rows = []
    for pset in ("ball", "sphere"):
        for n in (40000, 80000, 160000):
            X = inputs.ball(n, 0) if pset == "ball" else inputs.sphere(n, 0)
            pts = torch.from_numpy(X).cuda()
            b = torch.from_numpy(np.ascontiguousarray(inputs.rhs_uniform(n, 1, 1))).cuda()
            xr = torch.from_numpy(np.ascontiguousarray(inputs.rhs(n, 4, 3))).cuda()
            h = api.H2(pts, "matern32", 4.0, 1e-2, 400, 1e-8)
            yh = h.matmul(xr)
            for tau, cap in ((1e-1, 200), (1e-2, 600)):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                hs = api.HSS(h, cap, 10, seed=2, tol=tau)
                u = api.ULV(hs)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                x, it, rr = api.pcg_solve(h, u, b, tol=1e-4)
                torch.cuda.synchronize()
                t2 = time.perf_counter()
                ys = hs.matmul(xr)
                err = float(((ys - yh).norm(dim=0) / yh.norm(dim=0)).mean())
                rows.append({"points": pset, "n": n, "tol": tau, "rank_cap": cap,
                             "max_rank": hs.info()["max_rank"], "pcg_iters": int(it.max()),
                             "relres": float(rr.max()), "matvec_err": err,
                             "build_ms": (t1 - t0) * 1e3, "solve_ms": (t2 - t1) * 1e3})
                u.close(); hs.close()
            h.close()
            del pts, b, xr, yh
            torch.cuda.empty_cache()
    print(json.dumps({"metric": "PCG iterations with tolerance-truncated SPD-HSS bases",
                      "workload": "matern32_l0.25_ball_sphere_n40k-160k", "rows": rows,
                      "dtype": "f64", "data": "synthetic"}))


def main():
    args = parse()
    if args.tol_sweep:
        run_tol_sweep()
        return
    if args.rpy_sweep:
        run_rpy_sweep([int(v) for v in args.rpy_sweep.split(",")])
        return
    if args.rank_sweep:
        run_rank_sweep()
        return
    if args.kernel_sweep:
        run_kernel_sweep(args.sweep_kernel)
        return
    if args.paper_table:
        run_paper_table()
        return
    if args.batch:
        run_batch(args.batch)
        return
    if args.serve:
        run_serve(args.serve)
        return
    if args.precision:
        run_precision(args)
        return
    if args.matvec_case:
        run_matvec_case(args.matvec_case, args.mixed)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
