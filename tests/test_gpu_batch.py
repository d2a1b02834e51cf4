"""Batched sampling of independent MPS of different shapes in one persistent launch (needs a GB300).

Each job's result from fastmps_sample_batch must equal, bitwise, the same job sampled alone with
fastmps_sample_ex (the persistent kernel does the same arithmetic per tile and per row); a second call
replays the captured CUDA graph and must give the same result again.  Jobs split into several chunks
exercise the per-m-tile step counters across chunk boundaries; a stalled dependency (test hook) makes
the kernel's bounded waits run out and the call report FASTMPS_ERR_TIMEOUT, after which the runner
works again.
"""
import os

import numpy as np
import pytest

import gen
import parity
from oracle import quant

pytestmark = pytest.mark.gpu

SHAPES = [  # (M, d, chi, N, skew)
    (12, 3, 16, 1000, None),
    (20, 2, 32, 3000, 1.5),
    (16, 4, 64, 500, 1.5),
    (10, 6, 24, 2000, 1.5),
    (30, 3, 128, 700, 1.5),
]


def _chains(F, precision, shapes, seed0=500):
    chains, jobs, refs = [], [], []
    for i, (M, d, chi, N, skew) in enumerate(shapes):
        b, ts, _ = gen.mps_tensors(M, d, chi, base_seed=seed0 + 37 * i, skew=skew)
        s = F.Sampler(precision=precision)
        s.load_chain(ts)
        chains.append((s, b, ts))
        refs.append(s.sample(b, d, N, 100 + i, n0=11 * i, job=i))
        jobs.append({"chain": s.h, "bonds": b, "d": d, "N": N, "seed": 100 + i, "n0": 11 * i, "job": i,
                     "out_samples": np.empty((N, M), np.uint8), "out_logprob": np.empty(N, np.float64)})
    return chains, jobs, refs


def _check(jobs, refs, what):
    for j, (ref_s, ref_l) in zip(jobs, refs):
        assert np.array_equal(j["out_samples"], ref_s), what
        assert np.array_equal(j["out_logprob"], ref_l), what


@pytest.mark.parametrize("precision", ["bf16x2", "bf16x3l"])
def test_batch_equals_separate_runs(precision):
    import paper_2512_20064_gb300 as F

    chains, jobs, refs = [], [], []
    for i, (M, d, chi, N, skew) in enumerate(SHAPES):
        b, ts, _ = gen.mps_tensors(M, d, chi, base_seed=500 + 37 * i, skew=skew)
        s = F.Sampler(precision=precision)
        s.load_chain(ts)
        chains.append((s, b, ts))
        refs.append(s.sample(b, d, N, 100 + i, n0=11 * i, job=i))
        jobs.append({"chain": s.h, "bonds": b, "d": d, "N": N, "seed": 100 + i, "n0": 11 * i, "job": i,
                     "out_samples": np.empty((N, M), np.uint8), "out_logprob": np.empty(N, np.float64)})
    with F.Sampler(precision=precision) as runner:
        for call in range(2):
            for j in jobs:
                j["out_samples"][:] = 255
                j["out_logprob"][:] = np.nan
            F.fastmps_sample_batch(runner.h, jobs)
            for j, (ref_s, ref_l) in zip(jobs, refs):
                assert np.array_equal(j["out_samples"], ref_s), call
                assert np.array_equal(j["out_logprob"], ref_l), call
        st = runner.stats()
        print(precision, {k: st[k] for k in ("ms_total", "ms_contract", "launches", "contract_launches")})
        assert st["contract_launches"] == 1
    # oracle parity of one job of the batch
    s, b, ts = chains[2]
    M, d, chi, N, _ = SHAPES[2]
    rep = parity.check(b, [quant.dequant_bf16(A, 1) for A in ts], 102, np.arange(11 * 2, 11 * 2 + N),
                       jobs[2]["out_samples"], jobs[2]["out_logprob"], 1e-4, job=2)
    print(rep)
    for s, _, _ in chains:
        s.close()


def test_batch_rejects_mismatched_precision():
    import paper_2512_20064_gb300 as F

    b, ts, _ = gen.mps_tensors(8, 2, 8, base_seed=1)
    with F.Sampler(precision="fp32") as chain, F.Sampler(precision="bf16x2") as runner:
        chain.load_chain(ts)
        with pytest.raises(F.FastMPSError) as e:
            F.fastmps_sample_batch(runner.h, [{"chain": chain.h, "bonds": b, "d": 2, "N": 10, "seed": 1}])
        assert e.value.code == -1


def test_autotuner_picks_a_width_caches_it_and_stays_correct(tmp_path, monkeypatch):
    """autotune=1 times the candidate n-tile widths and measurement modes (two-pass, single-pass cluster)
    per site shape, records the choice (bn + 10000 * mode) in the JSON cache file, and the sampler stays
    within tolerance of the oracle with the chosen layout and mode."""
    import json

    import paper_2512_20064_gb300 as F

    cache = tmp_path / "tune.json"
    monkeypatch.setenv("FASTMPS_TUNE_CACHE", str(cache))
    b, ts, _ = gen.mps_tensors(24, 4, 256, base_seed=9, skew=1.5, dtype=np.complex64)
    with F.Sampler(precision="bf16x2", autotune=True) as s:
        s.load_chain(ts)
        smp, lp, tr = s.sample(b, 4, 4096, 5, trace_rows=64)
    table = json.loads(cache.read_text())
    code = table["1:256:4:256"]
    assert code % 10000 in (64, 128, 256) and code // 10000 in (0, 2)
    print("tuned widths", table)
    rep = parity.check(b, [quant.dequant_bf16(A, 1) for A in ts], 5, np.arange(64), smp[:64], lp[:64], 1e-4,
                       dev_trace=tr, trace_rows=64)
    print(rep)


def test_batch_several_chunks_per_job_and_uneven_shapes():
    """Jobs of 3 to 9 chunks of 1024 rows (the runner's micro-batch cap): a task of chunk c+1 reuses the
    scratch rows of chunk c and waits for their last measurement; site-varying widths within a job."""
    import paper_2512_20064_gb300 as F

    shapes = [(14, 4, 256, 5000, 1.5), (22, 3, 100, 9000, 1.5), (9, 6, 48, 3100, 1.5), (17, 2, 200, 2049, None)]
    chains, jobs, refs = _chains(F, "bf16x2", shapes, seed0=900)
    with F.Sampler(precision="bf16x2", max_microbatch=1024) as runner:
        for call in range(2):
            F.fastmps_sample_batch(runner.h, jobs)
            _check(jobs, refs, call)
        st = runner.stats()
        assert st["contract_launches"] == 1
        print({k: st[k] for k in ("ms_contract", "launches", "contract_launches")})
    for s, _, _ in chains:
        s.close()


def test_batch_stalled_dependency_times_out_then_runner_recovers(monkeypatch):
    """Test hook FASTMPS_TEST_STALL_DEPENDENCY=1: every task waits for one measurement more than ever
    happens; the bounded wait (100 ms) runs out, the kernel records the error and returns, and the call
    reports FASTMPS_ERR_TIMEOUT.  Without the hook the same runner then gives the exact results."""
    import paper_2512_20064_gb300 as F

    chains, jobs, refs = _chains(F, "bf16x2", SHAPES[:3], seed0=700)
    with F.Sampler(precision="bf16x2") as runner:
        monkeypatch.setenv("FASTMPS_TEST_STALL_DEPENDENCY", "1")
        with pytest.raises(F.FastMPSError) as e:
            F.fastmps_sample_batch(runner.h, jobs)
        assert e.value.code == -6  # FASTMPS_ERR_TIMEOUT
        monkeypatch.delenv("FASTMPS_TEST_STALL_DEPENDENCY")
        F.fastmps_sample_batch(runner.h, jobs)
        _check(jobs, refs, "after the timeout")
    for s, _, _ in chains:
        s.close()
