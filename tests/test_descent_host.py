"""The autotuner's coordinate descent (csrc/gi_descent.h, host-only) on
synthetic cost models with known optima: separable knobs, a pair move, invalid
values, the 1% threshold, error propagation and the pass limit.  Compiled with
the host compiler and run on the CPU; no GPU is needed."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_descent_on_synthetic_models():
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    os.makedirs(os.path.join(HERE, "_build"), exist_ok=True)
    exe = os.path.join(HERE, "_build", "descent_probe")
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-I" + os.path.join(ROOT, "paper_2506_01576_gb300", "csrc"),
                        os.path.join(HERE, "descent_probe.cpp"), "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count(" ok") == 7, r.stdout
