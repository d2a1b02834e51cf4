"""Teacher-forced parity of a device run against the FP64 oracle.

Given the device's outcomes for a set of rows, the oracle replays those rows
along the device's outcome prefix and reports, at every (row, site), its own
conditionals, the outcome its own uniform picks and that uniform's distance
to the nearest interior CDF boundary.  The rules (identical uniforms on both
sides):

* conditionals: |p_dev(s) - p_orc(s)| <= tol for every traced (row, site, s);
* outcomes: identical, except where the oracle's uniform lies within tol of a
  CDF boundary (a "boundary draw"); mismatches must also be < 0.1 % of draws;
* log-probability: |logp_dev - logp_orc| <= sum_k tol / p_orc(s_k) (first
  order bound from the conditional tolerance), plus rounding slack.
"""
from __future__ import annotations

from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle


class Prefetch:
    """A ``tensors(k)`` callable for a replay that asks for sites in increasing order: it computes
    ``f(k)`` for the next ``ahead`` sites in ``workers`` threads while the oracle works on the current
    ones (the oracle's C loop and torch's copies and casts run without the interpreter lock)."""

    def __init__(self, f, M, ahead=64, workers=4):
        self.f, self.M, self.ahead = f, M, ahead
        self.pool = ThreadPoolExecutor(max_workers=workers)
        self.pending = {}

    def __call__(self, k):
        for j in range(k, min(self.M, k + self.ahead)):
            if j not in self.pending:
                self.pending[j] = self.pool.submit(self.f, j)
        return self.pending.pop(k).result()

    def close(self):
        for fut in self.pending.values():
            fut.cancel()
        self.pool.shutdown(wait=True)
        self.pending.clear()


def check(bonds, tensors, seed, rows, dev_samples, dev_logprob, tol, dev_trace=None, trace_rows=0,
          site_index=None, job=0, nthreads=0, site_chunk=None, lams=None, mu=None, dev_trace_list=None):
    """rows: sample indices checked; dev_samples[i], dev_logprob[i] belong to rows[i].

    dev_trace: [M, trace_rows, d] device conditionals of rows 0..trace_rows-1
    (rows[i] < trace_rows are compared), or, with dev_trace_list, of the rows
    dev_trace_list[j] (every checked row in that list is compared).  The report
    carries the per-site maximum conditional error ("prob_err_by_site") and the
    oracle's conditionals of the checked rows ("oracle_probs", [R, M, d]).
    lams: Vidal form (tensors are Gamma_k).
    mu: displacement amplitudes of the device call, shape (M, N) with column n
    for sample n (the call started at n0 = 0).  Returns a report dict; raises
    AssertionError when a rule is broken.
    """
    rows = np.asarray(rows, np.int64)
    forced = np.ascontiguousarray(dev_samples)
    r = oracle.replay(bonds, tensors, seed, rows, forced, job=job, site_index=site_index, nthreads=nthreads,
                      site_chunk=site_chunk, lams=lams, mu=None if mu is None else np.asarray(mu)[:, rows])
    M = forced.shape[1]
    mism = r["own"] != forced
    boundary = r["margin"] <= tol
    bad_mism = mism & ~boundary
    report = {
        "rows": int(rows.size),
        "draws": int(mism.size),
        "mismatches": int(mism.sum()),
        "mismatch_frac": float(mism.mean()),
        "boundary_draws": int(boundary.sum()),
        "mismatch_outside_band": int(bad_mism.sum()),
    }
    assert not bad_mism.any(), f"outcome mismatch outside the tolerance band: {report}"
    assert report["mismatch_frac"] < 1e-3, f"too many boundary mismatches: {report}"
    # log-probability bound
    p_sel = np.take_along_axis(r["probs"], forced[:, :, None].astype(np.int64), axis=2)[:, :, 0]
    bound = (tol / np.maximum(p_sel, 1e-300)).sum(axis=1) + 1e-9 * M
    lp_err = np.abs(dev_logprob - r["logprob"])
    report["logprob_max_err"] = float(lp_err.max())
    report["logprob_max_err_over_bound"] = float((lp_err / bound).max())
    assert (lp_err <= bound).all(), f"log-probability outside its bound: {report}"
    report["oracle_probs"] = r["probs"]
    sel = np.zeros(0, np.int64)
    if dev_trace is not None and dev_trace_list is not None:
        pos = {int(x): j for j, x in enumerate(np.asarray(dev_trace_list, np.int64))}
        sel = np.asarray([i for i, x in enumerate(rows) if int(x) in pos], np.int64)
        cols = np.asarray([pos[int(rows[i])] for i in sel], np.int64)
    elif dev_trace is not None and trace_rows > 0:
        sel = np.nonzero(rows < trace_rows)[0]
        cols = rows[sel]
    if sel.size:
        dev = np.transpose(dev_trace[:, cols, :], (1, 0, 2))  # [R, M, d]
        err = np.abs(dev - r["probs"][sel])
        report["prob_max_err"] = float(err.max())
        report["prob_rows"] = int(sel.size)
        report["prob_err_by_site"] = err.max(axis=(0, 2))
        assert err.max() <= tol, f"conditional probabilities differ by {err.max():.3e} > {tol}: {report}"
    return report
