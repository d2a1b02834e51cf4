"""FP16 operands and promoted accumulation against the FP64 oracle (needs a GB300).

FP16x2 keeps each left row as two binary16 residual planes at a per-row power-of-two scale (22
significant bits) and the site tensor in binary16 at a per-site power-of-two scale; FP16x3 keeps the
site tensor as two binary16 planes (hi + lo) at that scale.  The oracle runs on the tensors the store
represents (oracle.quant.dequant_fp16 with one or two planes).  Promoted accumulation (accum_chunk = c)
lets the tensor cores accumulate only c k-blocks at a time and adds the chunk sums in FP32 registers.
Every conditional of every row is compared at the low-precision tolerance; ragged rows, several
micro-batches and chunk counts that do not divide the contraction index are covered.
"""
import numpy as np
import pytest

import gen
import parity
from oracle import quant

pytestmark = pytest.mark.gpu


def _oracle_tensors(ts, precision):
    if precision in ("fp16x2", "fp16x3"):
        return [quant.dequant_fp16(A, 2 if precision == "fp16x3" else 1) for A in ts]
    return [quant.dequant_bf16(A, 2 if precision in ("bf16x3", "bf16x4") else 1) for A in ts]


@pytest.mark.parametrize("precision,accum_chunk", [("fp16x2", 0), ("fp16x2", 4), ("fp16x2", 3), ("bf16x2", 2),
                                                   ("bf16x3l", 4), ("fp16x3", 0), ("fp16x3", 4)])
def test_precision_modes_against_oracle(precision, accum_chunk):
    import paper_2512_20064_gb300 as F

    b, ts, _ = gen.mps_tensors(30, 4, 288, base_seed=21, skew=1.5, dtype=np.complex64)
    N = 5000
    with F.Sampler(precision=precision, accum_chunk=accum_chunk, max_microbatch=2048) as s:
        s.load_chain(ts)
        smp, lp, tr = s.sample(b, 4, N, 31, trace_rows=N)
    rep = parity.check(b, _oracle_tensors(ts, precision), 31, np.arange(N), smp, lp, 1e-4, dev_trace=tr,
                       trace_rows=N)
    print(precision, accum_chunk, rep["prob_max_err"], rep["mismatches"])
    assert rep["prob_rows"] == N


def test_fp16x2_tiny_chain_every_row(tiny_chain):
    import paper_2512_20064_gb300 as F

    b, ts = tiny_chain
    with F.Sampler(precision="fp16x2", accum_chunk=2) as s:
        s.load_chain(ts)
        smp, lp, tr = s.sample(b, 3, 10_000, 42, trace_rows=10_000)
    rep = parity.check(b, _oracle_tensors(ts, "fp16x2"), 42, np.arange(10_000), smp, lp, 1e-4, dev_trace=tr,
                       trace_rows=10_000)
    print(rep["prob_max_err"], rep["mismatches"])
    assert rep["prob_rows"] == 10_000


@pytest.mark.parametrize("precision", ["fp16x2", "fp16x3"])
def test_fp16_streamed_equals_resident(precision):
    """Host-streamed FP16 tensors (binary16 conversion of one or two planes on the host, expanded on the
    device at every site) give bitwise the results of tensors converted on the device."""
    import paper_2512_20064_gb300 as F

    b, ts, _ = gen.mps_tensors(20, 3, 200, base_seed=13, skew=1.5)
    out = {}
    for residency in ("hbm", "host_stream"):
        with F.Sampler(precision=precision, residency=residency, accum_chunk=4) as s:
            s.load_chain(ts)
            out[residency] = s.sample(b, 3, 3000, 5)
    assert np.array_equal(out["hbm"][0], out["host_stream"][0])
    assert np.array_equal(out["hbm"][1], out["host_stream"][1])


@pytest.mark.parametrize("precision", ["fp16x2", "fp16x3"])
def test_fp16_is_rejected_where_unsupported(precision):
    import paper_2512_20064_gb300 as F

    b, ts, _ = gen.mps_tensors(8, 2, 8, base_seed=1)
    with F.Sampler(precision=precision) as s:
        s.load_chain(ts)
        with pytest.raises(F.FastMPSError) as e:
            s.sample(b, 2, 10, 1, mu=np.zeros((8, 10), np.complex64))
        assert e.value.code == -7
