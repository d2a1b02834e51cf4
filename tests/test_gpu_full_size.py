"""Full-size parity of the precision workload (M=1024, d=4, chi=1024) in the benchmark's launch
configuration: one macro-batch of 2^18 rows per call, site tensors generated on the device.

The oracle replays sampled rows (the first 48, traced at every site, and the last 16) along the
device's outcomes, 32 sites at a time, on the tensors the BF16 store represents.
"""
import numpy as np
import pytest

import gen
import parity
from oracle import quant

pytestmark = pytest.mark.gpu

ROWS_PER_CALL = 1 << 18
TRACE = 48


@pytest.fixture(scope="module")
def precision_chain():
    w = gen.WORKLOADS["precision"]
    b, ts, idx = gen.mps_tensors(w.M, w.d, w.chi, base_seed=w.base_seed, skew=w.skew, device="cuda")
    return w, b, ts


@pytest.mark.parametrize("precision,planes", [("bf16x2", 1)])
def test_precision_workload_sampled_rows(precision_chain, precision, planes):
    import torch

    import paper_2512_20064_gb300 as F

    w, b, ts = precision_chain
    N = ROWS_PER_CALL
    out_s = torch.empty((N, w.M), dtype=torch.uint8, device="cuda")
    out_l = torch.empty(N, dtype=torch.float64, device="cuda")
    with F.Sampler(precision=precision) as s:
        for k in range(w.M):
            s.load_site(k, ts[k])
        _, _, tr = s.sample(b, w.d, N, w.sampler_seed, out_samples=out_s, out_logprob=out_l, trace_rows=TRACE)
        st = s.stats()
    rows = np.concatenate([np.arange(TRACE), np.arange(N - 16, N)])
    smp = out_s[torch.as_tensor(rows, device="cuda")].cpu().numpy()
    lp = out_l[torch.as_tensor(rows, device="cuda")].cpu().numpy()

    def tensor(k):
        return quant.dequant_bf16(ts[k].cpu().numpy(), planes).astype(np.complex64)

    rep = parity.check(b, tensor, w.sampler_seed, rows, smp, lp, 1e-4, dev_trace=tr, trace_rows=TRACE,
                       site_chunk=32)
    print(precision, rep, {k: st[k] for k in ("ms_contract", "ms_measure", "launches")})
    assert np.isfinite(out_l.cpu().numpy()).all()
