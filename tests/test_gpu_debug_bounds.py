"""The bounds-checked build (-DTC_DEBUG_BOUNDS) in a process of its own:
every index the count, gather and dense-core kernels take from graph data
is checked against its array while the whole path runs on small graphs
(n <= 4096) under every strategy, dense core, count mode, sharding and
batching; no check may fail and every result must equal the oracle's.  A
failed check is recorded in an error word and the access skipped, so the
test can fail but never fault the GPU."""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bounds_checked_build_runs_clean():
    out = subprocess.run([sys.executable, os.path.join(HERE, "debug_bounds_worker.py")],
                         capture_output=True, text=True, timeout=1200)
    assert out.returncode == 0, out.stdout[-3000:] + out.stderr[-3000:]
    assert out.stdout.strip().splitlines()[-1].startswith("ok ")
