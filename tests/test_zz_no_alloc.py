"""fastmps_sample_noalloc -- sampling that allocates nothing -- against fastmps_sample_ex (needs a GB300).

Some callers cannot allocate device memory while they sample: runtimes whose memory belongs to their
own caching allocator or a fixed budget, services that allocate only at start-up.  The no-alloc entry
point takes every per-call buffer from a static 64 MiB device array, so it must give the same samples
and log-probabilities as the allocating entry point.  Two calls in a row check that the array's
leftover contents from the first call do not leak into the second.  Calls with more rows than one
micro-batch of scratch holds walk the micro-batch loop.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "bf16x2": 1e-4}


def _noalloc(F, s, b, d, n0, N, seed):
    import torch

    M = len(b) - 1
    out_s = torch.empty((N, M), dtype=torch.uint8, device="cuda")
    out_l = torch.empty(N, dtype=torch.float64, device="cuda")
    F.fastmps_sample_noalloc(s.h, M, d, b, n0, N, seed, 0, out_s, out_l)
    return out_s.cpu().numpy(), out_l.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp32", "bf16x2"])
def test_noalloc_matches_allocating_entry_point_on_two_calls(precision):
    import paper_2512_20064_gb300 as F

    w = gen.WORKLOADS["tiny"]
    b, ts, _ = gen.mps_tensors(w.M, w.d, w.chi, base_seed=w.base_seed, skew=w.skew)
    with F.Sampler(precision=precision) as s:
        s.load_chain(ts)
        for (n0, N, seed) in ((0, 3000, 42), (5000, 1000, 7)):
            ref_s, ref_l = s.sample(b, w.d, N, seed, n0=n0)
            got_s, got_l = _noalloc(F, s, b, w.d, n0, N, seed)
            # identical kernels on identical inputs: outcomes agree; log-probabilities within the
            # first-order bound of the conditional-probability tolerance
            assert np.array_equal(ref_s, got_s), (precision, n0, N)
            assert np.abs(ref_l - got_l).max() <= TOL[precision] * w.M, (precision, n0, N)


def test_noalloc_rejects_oversize_and_host_outputs_then_still_works():
    import torch

    import paper_2512_20064_gb300 as F

    w = gen.WORKLOADS["plain"]
    b, ts, _ = gen.mps_tensors(40, w.d, w.chi, base_seed=5, skew=w.skew, dtype=np.complex64)
    with F.Sampler(precision="fp32") as s:
        s.load_chain(ts)
        M = len(b) - 1
        big = 1 << 16
        out_s = torch.empty((big, M), dtype=torch.uint8, device="cuda")
        out_l = torch.empty(big, dtype=torch.float64, device="cuda")
        with pytest.raises(F.FastMPSError) as e:
            F.fastmps_sample_noalloc(s.h, M, w.d, b, 0, big, 1, 0, out_s, out_l)
        assert e.value.code == -1 and "MiB" in str(e.value)
        with pytest.raises(F.FastMPSError) as e:
            F.fastmps_sample_noalloc(s.h, M, w.d, b, 0, 10, 1, 0, np.empty((10, M), np.uint8), None)
        assert e.value.code == -1
        ref_s, ref_l = s.sample(b, w.d, 500, 3)
        got_s, got_l = _noalloc(F, s, b, w.d, 0, 500, 3)
        assert np.array_equal(ref_s, got_s)
        assert np.abs(ref_l - got_l).max() <= TOL["fp32"] * M


@pytest.mark.parametrize("precision", ["fp32", "bf16x2"])
def test_noalloc_several_microbatches_match_bitwise(precision):
    """M=40 sites at chi=256, d=4: 6000 and 9000 rows need two and three micro-batches of the 64 MiB scratch (the
    contraction scratch Y and the sums of squares P are carved per micro-batch); bitwise equal to
    the allocating entry point, on two calls in a row."""
    import paper_2512_20064_gb300 as F

    w = gen.WORKLOADS["plain"]
    b, ts, _ = gen.mps_tensors(40, w.d, w.chi, base_seed=11, skew=w.skew, dtype=np.complex64)
    with F.Sampler(precision=precision) as s:
        s.load_chain(ts)
        for (n0, N, seed) in ((0, 6000, 21), (777, 9000, 22)):
            ref_s, ref_l = s.sample(b, w.d, N, seed, n0=n0)
            got_s, got_l = _noalloc(F, s, b, w.d, n0, N, seed)
            assert np.array_equal(ref_s, got_s), (precision, n0, N)
            assert np.array_equal(ref_l, got_l), (precision, n0, N)
