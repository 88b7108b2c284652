"""Bounded waits that run out leave the heap safe to use.

A test build of the library with DSOA_SPIN_LIMIT = 1 makes every look-back wait
and every blocking bitmap update give up at its first unsuccessful poll.  The
workloads run in a subprocess on that library (``spin_limit_worker.py``); this
test asserts on what it reports:

* an enumeration whose look-back gave up raises DSOA_DEV_SPIN and publishes an
  empty snapshot (r = 0), so no method runs on, or later reuses, a block list
  with misplaced entries; every entry of R stays below the block count;
* an enumeration that did not give up equals the allocated-block bitmap;
* the microbench, Wa-Tor, game of life and traffic run to the end with only
  the library's documented error bits set, the device checker runs, and a new
  heap works afterwards in the same process.

No kernel is made to fault or hang: every wait is bounded and the methods check
the instance and cell indices they read from object fields.
"""
import json
import os
import subprocess
import sys

import pytest

from gpu_common import gpu_ready

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def report():
    gpu_ready()
    from paper_1810_11765_gb300 import build
    lib = build.build(extra_flags=["-DDSOA_SPIN_LIMIT=1"],
                      out_lib=os.path.join(build.OUT, "libdsoa_spin1.so"))
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, os.path.join(HERE, "spin_limit_worker.py"), lib],
                       capture_output=True, text=True, timeout=900, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


@pytest.mark.parametrize("mode", ["one_tile_per_cta", "several_tiles_per_cta", "tickets"])
def test_enumeration_that_gives_up_publishes_an_empty_snapshot(report, mode):
    e = report["enumeration"][mode]
    assert e["blocks"] > 4096 and e["M"] > 4096 * 64          # many level-1 tiles
    assert e["gave_up"] > 0, e                                # the bound was reached
    assert all(n == 0 for n in e["r_when_gave_up"]), e
    assert e["R_in_bounds"], e
    assert e["other_bits"] == 0 and e["mismatch"] == 0, e


@pytest.mark.parametrize("name", ["micro", "wator", "gol", "traffic"])
def test_workloads_finish_with_documented_errors_only(report, name):
    w = report["workloads"][name]
    assert w["unknown_bits"] == 0 and w["check_ran"], w


def test_context_usable_afterwards(report):
    assert 0 < report["after"]["count"] <= 1000
