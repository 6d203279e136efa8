"""The bounds-checked build (libul_check.so, -DUL_CHECK): every link offset, neighbour
site and accumulator index of the update, measurement, plaquette and slab-resident kernels
is checked before its access, and an index out of range is recorded instead of faulting.
On 2^4, 4^4 and 6^3x4 lattices, every estimator and launch form records nothing and
matches the oracle (FP64).  It runs in a child process, which loads the checked library
in place of libul.so."""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def test_checked_build_records_no_out_of_range_index():
    from paper_1208_0166_gb300 import build

    build.build(check=True)
    env = dict(os.environ, UL_LIBRARY="check")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "check_build_run.py")], capture_output=True,
                       text=True, timeout=900, env=env, cwd=ROOT)
    print(p.stdout[-3000:])
    assert p.returncode == 0, p.stdout[-3000:] + p.stderr[-3000:]
    assert "CHECK-BUILD-OK" in p.stdout
