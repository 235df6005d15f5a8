"""The multi-GPU bench path is replicas only (independent instances per rank, no data-path
collective): the job time is the slowest rank's and the value counts every rank's steps.
Checked here with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took 100 (r + 1) ms for its 4 steps
    ms, value = bench.replica_throughput(100.0 * (rank + 1), 4, world, dist, "cpu")
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_two_replicas_max_time_and_total_steps():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == pytest.approx(200.0)          # the slowest rank
        assert value == pytest.approx(8 / 0.2)     # 2 ranks x 4 steps in 0.2 s


def test_single_replica_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_throughput(250.0, 5, 1) == (250.0, pytest.approx(20.0))


def test_replicas_draw_different_inputs():
    from paper_2011_07632_gb300 import inputs
    a = inputs.uniform_cube(64, 3, 0 + 0)
    b = inputs.uniform_cube(64, 3, 0 + 1)
    assert not (a == b).all()


def test_reference_arm_under_torchrun_prints_once():
    """bench.py --impl reference launched like the GPU arm with two ranks (gloo on the CPU):
    rank 0 alone times the oracle and prints one JSON line; the other rank exits 0."""
    import json
    import subprocess
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--problem-size", "300"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0


def test_family_table_reports_fp64_fraction():
    sys.path.insert(0, ROOT)
    import bench
    prof = {"a": {"ms": 10.0, "launches": 2, "flops": 6.0e9},
            "b": {"ms": 30.0, "launches": 3, "flops": 0.0}}
    t = bench.family_table(prof, 1.2)
    assert list(t) == ["b", "a"]
    assert t["a"]["tflops"] == pytest.approx(0.6) and t["a"]["fp64_frac"] == pytest.approx(0.5)
    assert "tflops" not in t["b"] and t["b"]["launches"] == 3
