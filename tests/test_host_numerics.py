"""The library's host numerics (planner.cpp: Jacobi SVD, register-blocked rank-k update,
symmetric eigensolver) compiled with a small C++ driver and checked against their defining
properties (no GPU)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2202_03655_gb300", "csrc")


def test_planner_host_numerics():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "planner_checks")
        subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "host", "planner_checks.cpp"),
                        os.path.join(CSRC, "planner.cpp"), "-o", exe, "-lpthread"], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    lines = out.stdout.strip().splitlines()
    assert out.returncode == 0, "\n".join(l for l in lines if l.startswith("FAIL"))
    assert len(lines) >= 30 and all(l.startswith("ok") for l in lines)
