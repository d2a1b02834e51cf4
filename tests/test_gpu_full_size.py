"""Full-size parity of the precision workload (M=1024, d=4, chi=1024) in the benchmark's launch
configuration: site tensors generated on the device, one call of 2^18 rows (tensor-core modes: four
micro-batches of 65536 rows) or 2^17 rows (FP32: two micro-batches).

Modes: FP16x2 operands with promoted accumulation (the benchmark's low-precision mode; gated at 1e-4),
the FP32 SIMT path (gated at 1e-5), and FP16x3 (the site tensor in two binary16 planes), gated at 1e-4
both against the tensors its store represents and, on the storage subset below, against the original
tensors.  (BF16x2 without promotion misses 1e-4 at this chain length -- 3.2e-4 on 1024 rows -- and
is not run by default.)  Further modes can be replayed and reported, ungated, by naming them in
FASTMPS_PARITY_MODES, e.g. "bf16x2:0,bf16x3l:4,fp16x2:8" (precision:accum_chunk).

Replayed rows, the same number in every micro-batch, spread over it and including its last 32 rows:
512 for FP16x2 (128 per micro-batch) and 256 for FP32 and FP16x3, so that the whole GPU suite stays
within a 20-minute run (one oracle replay of 1024 rows through this chain is ~3.5e13 flops).  They are
a subset of the 1024-row selection.
FASTMPS_PARITY_ROWS=1024 replays 1024 rows in every mode.  The device traces exactly the replayed
rows, so every conditional of every replayed row at every site is compared (low-precision modes on the
tensors their 16-bit store represents; FP32 on the complex64 tensors).  The printed report gives the
per-site error profile; for the 16-bit modes the oracle also replays 64 of the rows (128 with
FASTMPS_PARITY_ROWS=1024) on the original tensors, which gives the storage error (16-bit store vs original, oracle vs oracle) and the device's
total error against the original tensors (gated for FP16x3, reported for the others).

The binary16 stores are dequantised with torch's CPU float16 casts at the per-site power-of-two scale,
bitwise the oracle's restatement of the format (oracle.quant.dequant_fp16, pinned on the CPU against
the same casts); the test checks that equality again on three sites of the chain.
"""
import os

import numpy as np
import pytest

import gen
import oracle
import parity
from oracle import quant

pytestmark = pytest.mark.gpu

MICRO = 1 << 16
_ROWS = int(os.environ.get("FASTMPS_PARITY_ROWS", "0"))
# mode: (precision, accum_chunk, rows per call, replayed rows, tolerance gated or None,
#        tolerance against the original tensors gated or None)
MODES = {"fp16x2-promoted": ("fp16x2", 4, 1 << 18, _ROWS or 512, 1e-4, None),
         "fp32": ("fp32", 0, 1 << 17, _ROWS or 256, 1e-5, None),
         "fp16x3-promoted": ("fp16x3", 4, 1 << 18, _ROWS or 256, 1e-4, 1e-4)}
for _spec in filter(None, os.environ.get("FASTMPS_PARITY_MODES", "").split(",")):
    _prec, _chunk = _spec.split(":")
    MODES[_spec] = (_prec, int(_chunk), 1 << 18, _ROWS or 256, None, None)
STORAGE_ROWS = 128 if _ROWS >= 1024 else 64


def store_f16(A, planes):
    """The complex128 tensor an FP16 store of the complex64 array A (one or two binary16 planes at the
    per-site power-of-two scale) represents, with torch's CPU float16 casts (round to nearest, ties to
    even, subnormals kept): the same values as oracle.quant.dequant_fp16, faster."""
    import torch

    t = torch.from_numpy(np.ascontiguousarray(A))
    re, im = t.real.float(), t.imag.float()
    m = float(torch.maximum(re.abs().max(), im.abs().max()))
    s = 1.0 if m == 0.0 else float(2.0 ** np.floor(np.log2(quant.FP16_TOP / m)))
    parts = []
    for x in (re, im):
        xs = x * s                       # exact: a power-of-two scale
        v = xs.half().double()
        if planes == 2:
            v = v + (xs.double() - v).float().half().double()
        parts.append(v / s)
    return torch.complex(parts[0], parts[1]).numpy()


def spread_rows(N, total=1024, tail=32, full=1024):
    """total rows, the same number in every micro-batch, taken from the full-row selection: in every
    micro-batch, rows evenly spread over it plus its last `tail` rows.  Fewer rows than `full` keep
    the tail and an evenly strided subset of the spread rows, so a smaller replay checks a subset of
    the rows of the full one."""
    out = []
    nb = (N + MICRO - 1) // MICRO
    per_full = max(full, total) // nb
    per_batch = total // nb
    for j in range(nb):
        lo, hi = j * MICRO, min(N, (j + 1) * MICRO)
        spread = np.linspace(lo, hi - tail - 1, per_full - tail).round().astype(np.int64)
        if per_batch < per_full:
            spread = spread[np.linspace(0, spread.size - 1, per_batch - tail).round().astype(np.int64)]
        out.append(np.unique(np.concatenate([spread, np.arange(hi - tail, hi)])))
    rows = np.unique(np.concatenate(out))
    assert rows.size == per_batch * len(out)
    return rows


def profile(err_by_site):
    e = np.asarray(err_by_site)
    return {"first_64": float(e[:64].max()), "sites_64_to_M-64": float(e[64:-64].max()),
            "last_64": float(e[-64:].max()), "last_8": [float(f"{x:.2e}") for x in e[-8:]],
            "worst_site": int(e.argmax())}


@pytest.fixture(scope="module")
def precision_chain():
    w = gen.WORKLOADS["precision"]
    b, ts, idx = gen.mps_tensors(w.M, w.d, w.chi, base_seed=w.base_seed, skew=w.skew, device="cuda")
    return w, b, ts


@pytest.mark.parametrize("mode", list(MODES))
def test_precision_workload_replayed_rows(precision_chain, mode):
    import torch

    import paper_2512_20064_gb300 as F

    w, b, ts = precision_chain
    precision, accum_chunk, N, n_rows, tol, orig_tol = MODES[mode]
    rows = spread_rows(N, n_rows)
    assert rows.size == n_rows
    out_s = torch.empty((N, w.M), dtype=torch.uint8, device="cuda")
    out_l = torch.empty(N, dtype=torch.float64, device="cuda")
    with F.Sampler(precision=precision, accum_chunk=accum_chunk) as s:
        for k in range(w.M):
            s.load_site(k, ts[k])
        _, _, tr = s.sample(b, w.d, N, w.sampler_seed, out_samples=out_s, out_logprob=out_l, trace_list=rows)
        st = s.stats()
    idx = torch.as_tensor(rows, device="cuda")
    smp = out_s[idx].cpu().numpy()
    lp = out_l[idx].cpu().numpy()
    assert np.isfinite(out_l.cpu().numpy()).all()

    if precision == "fp32":
        def tensor(k):
            return ts[k].cpu().numpy()
    elif precision in ("fp16x2", "fp16x3"):
        planes = 2 if precision == "fp16x3" else 1
        for k in (0, w.M // 2, w.M - 1):
            A = ts[k].cpu().numpy()
            assert np.array_equal(store_f16(A, planes), quant.dequant_fp16(A, planes)), k

        def tensor(k):
            return store_f16(ts[k].cpu().numpy(), planes)
    else:
        def tensor(k):
            # what the BF16 store holds (hi + lo of a float32 fits a float32 again: complex64 is exact)
            planes = 2 if precision in ("bf16x3", "bf16x4") else 1
            return quant.dequant_bf16(ts[k].cpu().numpy(), planes).astype(np.complex64)

    fetch = parity.Prefetch(tensor, w.M)
    try:
        rep = parity.check(b, fetch, w.sampler_seed, rows, smp, lp, tol if tol else 1.0, dev_trace=tr,
                           dev_trace_list=rows, site_chunk=32)
    finally:
        fetch.close()
    assert rep["prob_rows"] == rows.size == n_rows
    summary = {k: v for k, v in rep.items() if not isinstance(v, np.ndarray)}
    summary["profile"] = profile(rep["prob_err_by_site"])
    summary["rows_per_microbatch"] = int(np.bincount(rows // MICRO).min())
    summary.update({k: st[k] for k in ("ms_contract", "ms_measure", "launches")})
    if tol is None:
        summary["ungated_max_error"] = summary.get("prob_max_err")
    if precision != "fp32":
        # storage error: the oracle on the original tensors along the same outcomes, for a row subset
        sub = np.linspace(0, rows.size - 1, STORAGE_ROWS).round().astype(np.int64)
        fetch = parity.Prefetch(lambda k: ts[k].cpu().numpy(), w.M)
        try:
            r0 = oracle.replay(b, fetch, w.sampler_seed, rows[sub], np.ascontiguousarray(smp[sub]), site_chunk=32)
        finally:
            fetch.close()
        storage = np.abs(r0["probs"] - rep["oracle_probs"][sub])
        dev = np.transpose(tr[:, sub, :], (1, 0, 2))
        total = np.abs(r0["probs"] - dev)
        summary["storage_error_max"] = float(storage.max())
        summary["storage_error_last_64"] = float(storage[:, -64:].max())
        summary["device_vs_original_max"] = float(total.max())
    print(f"\nPRECISION_PARITY {mode} N={N} rows={rows.size} {summary}", flush=True)
    if orig_tol is not None:
        assert summary["device_vs_original_max"] <= orig_tol
