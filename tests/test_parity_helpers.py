"""Host helpers of the full-size parity test, checked without a GPU: the replayed-row selection and the
fast dequantisation of the binary16 stores."""
import numpy as np
import pytest

import gen
import test_gpu_full_size as fs
from oracle import quant


@pytest.mark.parametrize("N,total", [(1 << 18, 512), (1 << 17, 256), (1 << 18, 256), (1 << 18, 1024),
                                     (1 << 17, 1024)])
def test_spread_rows_cover_every_microbatch_and_its_tail(N, total):
    rows = fs.spread_rows(N, total)
    assert rows.size == total and np.all(np.diff(rows) > 0) and rows[0] >= 0 and rows[-1] < N
    nb = (N + fs.MICRO - 1) // fs.MICRO
    counts = np.bincount(rows // fs.MICRO, minlength=nb)
    assert np.all(counts == total // nb)
    for j in range(nb):
        hi = min(N, (j + 1) * fs.MICRO)
        assert np.isin(np.arange(hi - 32, hi), rows).all()


def _spread_rows_1024(N, tail=32):
    """The 1024-row selection as first written: per micro-batch, 1024 / nb rows evenly spread plus the tail."""
    out = []
    nb = (N + fs.MICRO - 1) // fs.MICRO
    per = 1024 // nb
    for j in range(nb):
        lo, hi = j * fs.MICRO, min(N, (j + 1) * fs.MICRO)
        spread = np.linspace(lo, hi - tail - 1, per - tail).round().astype(np.int64)
        out.append(np.unique(np.concatenate([spread, np.arange(hi - tail, hi)])))
    return np.unique(np.concatenate(out))


@pytest.mark.parametrize("N", [1 << 17, 1 << 18])
def test_smaller_replays_check_a_subset_of_the_1024_rows(N):
    full = fs.spread_rows(N, 1024)
    assert np.array_equal(full, _spread_rows_1024(N))
    for total in (256, 512):
        assert np.isin(fs.spread_rows(N, total), full).all(), total


def test_default_modes_fit_their_calls():
    for name, (prec, chunk, N, total, tol, orig_tol) in fs.MODES.items():
        assert fs.spread_rows(N, total).size == total, name


@pytest.mark.parametrize("planes", [1, 2])
def test_fast_fp16_store_equals_the_oracle_restatement(planes):
    b, ts, _ = gen.mps_tensors(6, 4, 256, base_seed=99, skew=1.5, dtype=np.complex64)
    for A in ts:
        assert np.array_equal(fs.store_f16(A, planes), quant.dequant_fp16(A, planes))
    # entries spread over the binary16 subnormal range after scaling, and signed zeros
    A = ts[3].copy()
    A.flat[:6] = [1e-9 + 2e-9j, -3e-8, 2.5e-6j, 0.0, -0.0 - 0.0j, 7e-7 - 1e-12j]
    assert np.array_equal(fs.store_f16(A, planes), quant.dequant_fp16(A, planes))


def test_replay_through_prefetch_equals_the_chain_itself():
    """The full-size test hands the oracle a prefetching callable over the dequantised sites; replaying
    through it (sites asked for chunk by chunk, computed ahead in worker threads) gives the oracle's own
    conditionals exactly, and every site is computed once."""
    import oracle
    import parity

    b, ts, _ = gen.mps_tensors(40, 4, 64, base_seed=5, skew=1.5, dtype=np.complex64)
    stores = [fs.store_f16(A, 1) for A in ts]
    smp, lp, pr = oracle.sample(b, stores, 42, 24, want_probs=True)
    rows = np.arange(24)
    calls = []

    def f(k):
        calls.append(k)
        return fs.store_f16(ts[k], 1)

    fetch = parity.Prefetch(f, len(ts), ahead=8, workers=3)
    try:
        rep = parity.check(b, fetch, 42, rows, smp, lp, 1e-12, dev_trace=np.transpose(pr, (1, 0, 2)),
                           dev_trace_list=rows, site_chunk=5)
    finally:
        fetch.close()
    assert rep["prob_max_err"] == 0.0 and rep["mismatches"] == 0 and rep["prob_rows"] == 24
    assert sorted(calls) == list(range(len(ts)))
