"""The launch merger of the batched level sweep (csrc/merge.cu) on the host: a C++ harness
linked against libspdhss.so runs instances on threads whose hand-overs only record their
members (no GPU): lockstep merging in instance order, instances of uneven depth leaving
early, an instance that runs ahead waiting for the earliest step, empty launcher calls
keeping steps aligned, and an error reaching every member of a failed merged launch."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_merger_policy(tmp_path):
    from paper_2011_07632_gb300 import build
    lib = build.build()
    pkg = os.path.dirname(lib)
    exe = str(tmp_path / "merger_harness")
    cmd = [build._nvcc(), *build.ARCH, "-O1", "-std=c++17", "-I" + os.path.join(ROOT, "include"),
           "-I" + os.path.join(pkg, "csrc"), os.path.join(ROOT, "tests", "merger_harness.cu"),
           "-o", exe, "-L" + pkg, "-lspdhss", "-Xlinker", "-rpath=" + pkg, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0 and out.stdout.strip().endswith("OK"), out.stdout + out.stderr
