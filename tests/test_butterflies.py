"""Theorems 1-4 (and Algorithm 5's bound) for the library's own butterfly code,
compiled for the host from csrc/modarith.cuh: exhaustive at beta = 2^8, sampled
with edge values at beta = 2^16, 2^32 and 2^64.  CPU only."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_butterfly_theorems(tmp_path):
    exe = tmp_path / "butterfly_check"
    src = os.path.join(ROOT, "tests", "butterfly_check.cpp")
    inc = os.path.join(ROOT, "paper_1205_2926_gb300", "csrc")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", inc, src, "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "failures 0" in r.stdout
