"""Pointer classification of the C ABI (csrc/gi_ptr.h), on the CPU.

Device memory of the index's own device and managed memory are used in place,
host memory is staged, and device memory of another device is refused with
GI_ERR_INVALID: a kernel launched on the index's device must never be handed a
foreign device address (without peer access that is an illegal-address fault).
The rule is a pure function of what the runtime reports for the pointer, so it
is compiled with the host compiler and checked here without a GPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_pointer_classes():
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    os.makedirs(os.path.join(HERE, "_build"), exist_ok=True)
    exe = os.path.join(HERE, "_build", "ptr_class_probe")
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-I" + os.path.join(ROOT, "paper_2506_01576_gb300", "csrc"),
                        os.path.join(HERE, "ptr_class_probe.cpp"), "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count(": ok") == 9, r.stdout
    assert "another device: ok" in r.stdout
