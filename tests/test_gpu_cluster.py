"""Single-pass cluster measurement (contraction + Algorithm 2 in one kernel, no FP32 scratch) against
the two-pass path and the oracle, and the split-K cluster variant against the oracle (needs a GB300).

The cluster kernel sums the same per-tile FP32 squares in the same order and draws with the same
FP64 arithmetic as the two-pass path, so samples, log-probabilities and traced conditionals must
agree bit for bit.  The chains cover every cluster shape the engine uses: one tile per CTA (C = 4,
8, 9, 12 CTAs), two tiles per CTA (C = 16), a block padded beyond 2 chi_r (chi = 300), sites that
fall back to the two-pass kernel in the same call (small end bonds), ragged row counts, row offsets,
several micro-batches per site, and every BF16 plane count.
"""
import numpy as np
import pytest

import gen
import parity
from oracle import quant

pytestmark = pytest.mark.gpu


def _both(F, precision, b, ts, d, N, seed, n0=0, trace_rows=64, max_microbatch=0):
    out = {}
    for mode in ("separate", "cluster"):
        with F.Sampler(precision=precision, fused_measure=mode, max_microbatch=max_microbatch) as s:
            s.load_chain(ts)
            out[mode] = s.sample(b, d, N, seed, n0=n0, trace_rows=trace_rows)
            out[mode + "_stats"] = s.stats()
    return out


@pytest.mark.parametrize("case", [
    # (M, d, chi, N, precision, max_microbatch)
    (40, 4, 256, 20_000, "bf16x2", 0),       # interior C = 8 (T = 1), ends: C = 4 and the two-pass fallback
    (40, 4, 256, 20_000, "bf16x3l", 8192),   # three left planes, several micro-batches, ragged tail
    (24, 3, 300, 5_000, "bf16x3", 0),        # C = 9, block padded from 600 to 768 columns (zeros 600..639)
    (24, 3, 512, 6_000, "bf16x4", 0),        # C = 12
    (12, 4, 1024, 4_096, "bf16x2", 0),       # chi = 1024 sites: C = 16 CTAs of two tiles each
])
def test_cluster_equals_two_pass_bitwise(case):
    import paper_2512_20064_gb300 as F

    M, d, chi, N, precision, mb = case
    b, ts, _ = gen.mps_tensors(M, d, chi, base_seed=300 + chi, skew=1.5, dtype=np.complex64)
    out = _both(F, precision, b, ts, d, N, 99, n0=13, trace_rows=64, max_microbatch=mb)
    sep, clu = out["separate"], out["cluster"]
    assert np.array_equal(sep[0], clu[0]), "outcomes differ"
    assert np.array_equal(sep[1], clu[1]), "log-probabilities differ"
    assert np.array_equal(sep[2], clu[2]), "traced conditionals differ"
    # the cluster path launched one kernel per site and micro-batch and no measurement kernel
    st = out["cluster_stats"]
    assert st["ms_measure"] < out["separate_stats"]["ms_measure"]
    print(case, "launches", st["launches"], "vs", out["separate_stats"]["launches"])


def test_cluster_against_oracle_tiny_rows():
    """The cluster path against the FP64 oracle directly (tensors the BF16 store represents)."""
    import paper_2512_20064_gb300 as F

    b, ts, _ = gen.mps_tensors(30, 4, 256, base_seed=5, skew=1.5, dtype=np.complex64)
    with F.Sampler(precision="bf16x2", fused_measure="cluster") as s:
        s.load_chain(ts)
        smp, lp, tr = s.sample(b, 4, 3000, 42, trace_rows=3000)
    rep = parity.check(b, [quant.dequant_bf16(A, 1) for A in ts], 42, np.arange(3000), smp, lp, 1e-4, dev_trace=tr,
                       trace_rows=3000)
    print(rep["prob_max_err"], rep["mismatches"])
    assert rep["prob_rows"] == 3000


@pytest.mark.parametrize("ksplit", [2, 4])
def test_split_k_cluster_against_oracle(ksplit):
    """On-chip split-K (a cluster of 2 or 4 blocks per output tile, partial tiles added through
    distributed shared memory): the same draws as the oracle within the BF16 tolerance; rows of a
    ragged micro-batch and sites whose contraction index has an odd number of k-blocks."""
    import paper_2512_20064_gb300 as F

    b, ts, _ = gen.mps_tensors(30, 4, 288, base_seed=17, skew=1.5, dtype=np.complex64)
    with F.Sampler(precision="bf16x2", k_split=ksplit, max_microbatch=2048) as s:
        s.load_chain(ts)
        smp, lp, tr = s.sample(b, 4, 3000, 8, trace_rows=3000)
    rep = parity.check(b, [quant.dequant_bf16(A, 1) for A in ts], 8, np.arange(3000), smp, lp, 1e-4, dev_trace=tr,
                       trace_rows=3000)
    print(ksplit, rep["prob_max_err"], rep["mismatches"])
    assert rep["prob_rows"] == 3000
