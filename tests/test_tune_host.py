"""The launch-variant tuner (csrc/tune.cu) on the host: a C++ harness linked against
libspdhss.so gives it host timing functions (no GPU): the fastest candidate kept and
cached per key, failed candidates skipped, the fallback when tuning is off or every
timing failed, one timing under concurrent first requests, and the report's format."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tuner_policy(tmp_path):
    from paper_2011_07632_gb300 import build
    lib = build.build()
    pkg = os.path.dirname(lib)
    exe = str(tmp_path / "tune_harness")
    cmd = [build._nvcc(), *build.ARCH, "-O1", "-std=c++17", "-I" + os.path.join(ROOT, "include"),
           "-I" + os.path.join(pkg, "csrc"), os.path.join(ROOT, "tests", "tune_harness.cu"),
           "-o", exe, "-L" + pkg, "-lspdhss", "-Xlinker", "-rpath=" + pkg, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    env = dict(os.environ)
    env.pop("SPDHSS_TUNE", None)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60, env=env)
    assert out.returncode == 0 and out.stdout.strip().endswith("OK"), out.stdout + out.stderr
