"""The C ABI library loads and exports every function that include/gi.h declares.

No GPU is needed: the library is compiled here (nvcc cross-compiles sm_103a) and
loaded with ctypes; no function that touches the device is called.
"""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2506_01576_gb300 as gi
from paper_2506_01576_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)  # drop comments
        for m in re.finditer(r"\b(gi_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    return _build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("gi_build", "gi_point_lookup", "gi_range_lookup", "gi_destroy"):
        assert f in names


def test_header_is_plain_c():
    # the boundary is a C ABI: the header compiles as strict C99, with no C++
    build = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build")
    os.makedirs(build, exist_ok=True)
    src = os.path.join(build, "header_c99.c")
    with open(src, "w") as f:
        f.write('#include "gi.h"\nint main(void) { gi_info i; gi_tune_result r; (void)i; (void)r; return 0; }\n')
    include = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I" + include,
                        "-c", src, "-o", src + ".o"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_library_exports_every_declared_function(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    missing = declared_functions() - exported
    assert not missing, "declared but not exported: %s" % sorted(missing)


def test_library_loads_and_binding_covers_it(lib_path):
    lib = gi.load()
    for f in declared_functions():
        assert hasattr(lib, f)
        assert hasattr(gi, f), "binding lacks %s" % f
    # host-only calls that need no device
    assert lib.gi_last_error() == b""
    assert gi.gi_launch_count() >= 0
    assert lib.gi_footprint_bytes(None) == 0


def test_host_side_argument_checks_need_no_gpu(lib_path):
    lib = gi.load()
    out = ctypes.c_void_p()
    # bad layout / bad k / NULL out are rejected before any device call
    assert lib.gi_build(None, None, 0, 7, 0, ctypes.byref(out)) == gi.GI_ERR_INVALID
    assert b"layout" in lib.gi_last_error()
    assert lib.gi_build(None, None, 0, gi.GI_EYTZINGER_KARY, 40, ctypes.byref(out)) == gi.GI_ERR_INVALID
    assert lib.gi_build(None, None, 10, gi.GI_SORTED, 0, ctypes.byref(out)) == gi.GI_ERR_INVALID
    assert lib.gi_build(None, None, 0, gi.GI_SORTED | 0x200, 0, ctypes.byref(out)) == gi.GI_ERR_INVALID
    assert lib.gi_build(None, None, 0, gi.GI_SORTED, 0, None) == gi.GI_ERR_INVALID
    assert lib.gi_point_lookup(None, None, 1, None) == gi.GI_ERR_INVALID
    assert lib.gi_range_lookup(None, None, None, 1, None, None) == gi.GI_ERR_INVALID
    assert lib.gi_sync(None) == gi.GI_ERR_INVALID
    lib.gi_destroy(None)  # no-op
    # the autotuner rejects a NULL index or batch before any device call; its table
    # lives on the host
    assert lib.gi_tune(None, None, 1, 0, gi.GI_TUNE_APPLY, None) == gi.GI_ERR_INVALID
    assert lib.gi_batch_tune(None, None, None, 1, 0, None) == gi.GI_ERR_INVALID
    gi.gi_tune_table_clear()
    assert gi.gi_tune_table_get(gi.GI_EYTZINGER_KARY | gi.GI_KEY_U64, 5, 1 << 20) is None
    assert lib.gi_tune_table_get(0, 0, 1, None, None) == gi.GI_ERR_INVALID
    assert gi.gi_tune_table_layout(gi.GI_KEY_U64, 1 << 20) is None
    out = ctypes.c_void_p()
    assert lib.gi_build_tuned(None, None, 0, gi.GI_KEY_U64, None, 1, 0, 0, None, None) == gi.GI_ERR_INVALID
    assert lib.gi_build_tuned(None, None, 0, gi.GI_KEY_U64 | gi.GI_EYTZINGER, None, 1, 0, 0,
                              ctypes.byref(out), None) == gi.GI_ERR_INVALID


def test_binding_fails_loudly_without_library(monkeypatch):
    import importlib
    monkeypatch.setattr(gi, "_lib", None)
    # a path that does not exist (nothing is created)
    monkeypatch.setattr(gi, "lib_path", os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                     "_build", "no-such-dir", "missing.so"))
    with pytest.raises(ImportError):
        gi.load()
