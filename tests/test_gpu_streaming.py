"""Host-streaming residency: BF16 site tensors stay in pinned host memory and are copied into two
device slots on a copy stream, overlapped with the previous site's compute (needs a GB300).

Small chains check the streamed path against the resident path bitwise (same arithmetic, different
residency) and against the oracle; a chain at the streaming workload's bond dimension chi = 10^4
(d = 3, a pool of isometries reused along the chain) checks sampled rows against the oracle.
"""
import numpy as np
import pytest

import gen
import parity
from oracle import quant

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["bf16x2", "bf16x3"])
def test_streamed_equals_resident_and_oracle(precision):
    import paper_2512_20064_gb300 as F

    b, ts, idx = gen.mps_tensors(48, 3, 64, base_seed=11, skew=1.5, pool=5)
    N = 3000
    with F.Sampler(precision=precision) as s:
        s.load_chain(ts, site_index=idx)
        ref_s, ref_l = s.sample(b, 3, N, 5)
    with F.Sampler(precision=precision, residency="host_stream") as s:
        s.load_chain(ts, site_index=idx)
        got_s, got_l, tr = s.sample(b, 3, N, 5, trace_rows=256)
        st = s.stats()
    assert np.array_equal(ref_s, got_s) and np.array_equal(ref_l, got_l)
    assert st["h2d_bytes"] > 0
    planes = 2 if precision == "bf16x3" else 1
    ots = [quant.dequant_bf16(A, planes) for A in ts]
    rep = parity.check(b, ots, 5, np.arange(256), got_s[:256], got_l[:256], 1e-4, dev_trace=tr, trace_rows=256,
                       site_index=idx)
    print(precision, rep)


def test_streaming_bond_dimension_1e4_sampled_rows():
    """chi = 10^4, d = 3, M = 24 (sites 9..14 at full bond dimension, pool of 4 reused), N = 512 rows;
    the oracle replays 6 traced rows."""
    import torch

    import paper_2512_20064_gb300 as F

    M, d, chi, N, R = 24, 3, 10_000, 512, 6
    b, ts, idx = gen.mps_tensors(M, d, chi, base_seed=1234, skew=1.5, pool=4, device="cuda")
    with F.Sampler(precision="bf16x2", residency="host_stream") as s:
        s.load_chain(ts, site_index=idx)
        smp, lp, tr = s.sample(b, d, N, 42, trace_rows=R)
        st = s.stats()
    print({k: st[k] for k in ("ms_total", "ms_contract", "ms_measure", "h2d_bytes", "launches")})
    host = {}

    def tensor(k):
        j = idx[k]
        if j not in host:
            host.clear()
            host[j] = quant.dequant_bf16(ts[j].cpu().numpy(), 1).astype(np.complex64)
        return host[j]

    rep = parity.check(b, tensor, 42, np.arange(R), smp[:R], lp[:R], 1e-4, dev_trace=tr, trace_rows=R,
                       site_chunk=1)
    print(rep)
    assert np.isfinite(lp).all() and smp.max() < d
    del torch
