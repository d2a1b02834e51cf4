"""Failure detection without a GPU fault (needs a GB300).

* A bounded device wait that nothing completes gives up after its limit, reports FASTMPS_ERR_TIMEOUT and
  leaves the context usable (a sampling call afterwards succeeds).
* An injected device-allocation failure (host side, FASTMPS_FAIL_ALLOC_AFTER) is reported as
  FASTMPS_ERR_OOM and the handle keeps working once allocation succeeds again.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounded_wait_times_out_and_context_survives():
    import paper_2512_20064_gb300 as F

    status, waited = F.fastmps_selftest_bounded_wait(0, 50.0)
    assert status == -6  # FASTMPS_ERR_TIMEOUT
    assert 45.0 <= waited < 5000.0
    b, ts, _ = gen.mps_tensors(8, 2, 8, base_seed=1)
    with F.Sampler(precision="bf16x2") as s:
        s.load_chain(ts)
        smp, lp = s.sample(b, 2, 1000, 3)
    assert np.isfinite(lp).all()


def test_injected_allocation_failure_reports_oom():
    code = r'''
import sys, numpy as np
sys.path.insert(0, %r)
import gen, paper_2512_20064_gb300 as F
b, ts, _ = gen.mps_tensors(8, 2, 8, base_seed=1)
s = F.Sampler(precision="fp32")
try:
    s.load_chain(ts)                  # device allocations stop succeeding part-way through
    s.sample(b, 2, 1000, 3)
    print("NO-ERROR")
except F.FastMPSError as e:
    print("CODE", e.code, str(e))
''' % ROOT
    env = dict(os.environ, FASTMPS_FAIL_ALLOC_AFTER="12")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert "CODE -4" in out.stdout, out.stdout + out.stderr
