"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle/oracle.cpp (a dropped term, a
reversed tie-break, a wrong index or bound), builds it with g++ under
tests/_build/, and runs the pin tests (test_oracle_pins.py) against it through
GI_ORACLE_LIB: every mutant must fail at least one pin, and the unmodified copy
must pass all of them.  The oracle itself is never modified.  No GPU is needed.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "oracle.cpp")
OUT = os.path.join(HERE, "_build", "mutants")

# (name, text in oracle.cpp, replacement): one plausible mistake each
MUTANTS = [
    ("ties_reversed", "v[j] = {keys[j], j};", "v[j] = {keys[j], n - 1 - j};"),
    ("upper_bound_for_points", "const K* p = std::lower_bound(skeys, skeys + n, q[i]);",
     "const K* p = std::upper_bound(skeys, skeys + n, q[i]);"),
    ("no_key_check", "out[i] = (r < n && skeys[r] == q[i]) ? srows[r] : kMiss;",
     "out[i] = (r < n) ? srows[r] : kMiss;"),
    ("miss_value", "const uint32_t kMiss = 0xFFFFFFFFu;", "const uint32_t kMiss = 0u;"),
    ("exclusive_upper_bound_count", "while (r + c < n && skeys[r + c] <= hi[i]) ++c;",
     "while (r + c < n && skeys[r + c] < hi[i]) ++c;"),
    ("exclusive_upper_bound_fill", "while (r < n && skeys[r] <= hi[i]) out[o++] = srows[r++];",
     "while (r < n && skeys[r] < hi[i]) out[o++] = srows[r++];"),
    ("equal_bounds_empty", "      if (lo[i] > hi[i]) {\n        cnt[i] = 0;",
     "      if (lo[i] >= hi[i]) {\n        cnt[i] = 0;"),
    ("inclusive_scan", "    offsets[i] = run;\n    run += cnt[i];", "    run += cnt[i];\n    offsets[i] = run;"),
    ("child_index_off_by_one", "visit(node * k + 1 + c);", "visit(node * k + c + (c ? 0 : 1));"),
    ("node_width_k", "uint64_t first = node * (k - 1);", "uint64_t first = node * k;"),
    ("slot_before_child", """      visit(node * k + 1 + c);
      if (c + 1 < k) {
        uint64_t s = first + c;
        if (s < n) slot_rank[s] = next++;
      }""", """      if (c + 1 < k) {
        uint64_t s = first + c;
        if (s < n) slot_rank[s] = next++;
      }
      visit(node * k + 1 + c);"""),
]


def _build(name, text):
    d = os.path.join(OUT, name)
    os.makedirs(d, exist_ok=True)
    src = os.path.join(d, "oracle.cpp")
    lib = os.path.join(d, "liboracle.so")
    with open(src, "w") as f:
        f.write(text)
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", src, "-o", lib, "-pthread"])
    return lib


def _pins_pass(lib):
    env = dict(os.environ, GI_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(HERE, "test_oracle_pins.py"),
                        "-q", "-x", "-p", "no:cacheprovider"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    return r.returncode == 0, r.stdout[-1500:]


def test_every_planted_mistake_fails_a_pin():
    original = open(SRC).read()
    jobs = [("unmodified", original)]
    for name, old, new in MUTANTS:
        assert original.count(old) == 1, name  # the mutation still applies to the current source
        jobs.append((name, original.replace(old, new)))
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        libs = list(ex.map(lambda j: _build(*j), jobs))
        results = list(ex.map(_pins_pass, libs))
    ok, log = results[0]
    assert ok, "the unmodified oracle must pass its pins:\n" + log
    survivors = [jobs[i][0] for i in range(1, len(jobs)) if results[i][0]]
    assert not survivors, "mistakes no pin catches: %s" % survivors
