"""Vidal-form input and GBS displacement on the device vs the FP64 oracle (needs a GB300).

* ``fastmps_displacement``: the batched Zassenhaus matrices (FP32) against the
  oracle's FP64 matrices, element by element.
* ``fastmps_load_site_vidal``: sampling a chain given as (Gamma, Lambda) against
  the oracle's Vidal-form sampling (FP32 path), and the BF16 path against the
  oracle on the tensors the BF16 store represents, bf16(Gamma * Lambda).
* ``fastmps_sample_displaced``: teacher-forced parity with per-sample
  amplitudes, for d in the three kernel variants (d <= 4, <= 8, <= 16), a
  ragged micro-batch tail and the plain workload size; 10^6-sample marginals.
"""
import math

import numpy as np
import pytest

import gen
import oracle
import parity
from oracle import quant

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "bf16x2": 1e-4, "bf16x3": 1e-4}


@pytest.fixture(scope="module")
def lib():
    import paper_2512_20064_gb300 as F

    F.load_library()
    return F


def _dq(tensors, precision):
    if precision == "bf16x2":
        return [quant.dequant_bf16(A, 1) for A in tensors]
    if precision == "bf16x3":
        return [quant.dequant_bf16(A, 2) for A in tensors]
    return tensors


# ---------------------------------------------------------------------------
# displacement matrices
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d", [2, 3, 4, 6, 10, 16])
def test_displacement_matrices(lib, d):
    N = 3000 + 17                                    # not a multiple of the block size
    mu = gen.gbs_amplitudes(1, N, sigma=0.6, seed=d)[0]
    with lib.Sampler() as s:
        D = s.displacement(mu, d)                    # [d, d, N], batch last
    assert D.shape == (d, d, N) and D.dtype == np.complex64
    worst = 0.0
    for n in range(0, N, 7):
        ref = oracle.displacement(complex(mu[n]), d)
        worst = max(worst, float(np.abs(D[:, :, n] - ref).max()))
    print("d", d, "max |D_gpu - D_oracle|", worst)
    assert worst < 1e-6


def test_displacement_device_arrays_and_empty(lib):
    import torch

    N, d = 4096, 4
    mu = torch.from_numpy(gen.gbs_amplitudes(1, N, seed=3)[0]).cuda()
    out = torch.empty((d, d, N), dtype=torch.complex64, device="cuda")
    with lib.Sampler() as s:
        lib.fastmps_displacement(s.h, mu, d, out=out)
        host = s.displacement(mu.cpu().numpy(), d)
        empty = s.displacement(np.zeros(0, np.complex64), d)
    assert np.array_equal(out.cpu().numpy(), host)
    assert empty.shape == (d, d, 0)


# ---------------------------------------------------------------------------
# Vidal form
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def vidal_chain():
    return gen.decaying_vidal_chain(40, 3, 24, decay=0.3, seed=12)


@pytest.mark.parametrize("precision", ["fp32", "bf16x2", "bf16x3"])
def test_vidal_parity(lib, vidal_chain, precision):
    b, G, L = vidal_chain
    N, seed = 3000, 99
    with lib.Sampler(precision=precision, max_microbatch=1024) as s:
        s.load_chain_vidal(G, L)
        smp, lp, tr = s.sample(b, 3, N, seed, trace_rows=N)
    if precision == "fp32":
        rep = parity.check(b, G, seed, np.arange(N), smp, lp, TOL[precision], dev_trace=tr, trace_rows=N, lams=L)
    else:
        stored = _dq([G[k] * L[k][None, None, :] for k in range(len(G))], precision)
        rep = parity.check(b, stored, seed, np.arange(N), smp, lp, TOL[precision], dev_trace=tr, trace_rows=N)
    print(precision, rep)
    assert rep["prob_rows"] == N


def test_vidal_equals_canonical_load(lib, vidal_chain):
    """Loading (Gamma, Lambda) gives the same samples as loading Gamma * Lambda (complex64 inputs,
    identical FP32 products on the device and on the host)."""
    b, G, L = vidal_chain
    G32 = [g.astype(np.complex64) for g in G]
    L32 = [l.astype(np.float32) for l in L]
    A32 = [(g * l[None, None, :]).astype(np.complex64) for g, l in zip(G32, L32)]
    with lib.Sampler(precision="bf16x2") as s:
        s.load_chain_vidal(G32, L32)
        s1, l1 = s.sample(b, 3, 2000, 5)
    with lib.Sampler(precision="bf16x2") as s:
        s.load_chain(A32)
        s2, l2 = s.sample(b, 3, 2000, 5)
    assert np.array_equal(s1, s2) and np.array_equal(l1, l2)


def test_vidal_host_stream(lib, vidal_chain):
    b, G, L = vidal_chain
    N, seed = 2000, 4
    with lib.Sampler(precision="bf16x2") as s:
        s.load_chain_vidal(G, L)
        s1, l1 = s.sample(b, 3, N, seed)
    with lib.Sampler(precision="bf16x2", residency="host_stream") as s:
        s.load_chain_vidal(G, L)
        s2, l2 = s.sample(b, 3, N, seed)
    assert np.array_equal(s1, s2) and np.array_equal(l1, l2)


# ---------------------------------------------------------------------------
# displaced sampling
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision,d,chi", [("fp32", 4, 32), ("bf16x2", 4, 32), ("fp32", 6, 24),
                                             ("bf16x2", 6, 24), ("fp32", 12, 12), ("bf16x2", 16, 16)])
def test_displaced_parity(lib, precision, d, chi):
    M, N, seed = 20, 2500, 31
    b, ts, _ = gen.mps_tensors(M, d, chi, base_seed=55 + d, skew=1.5)
    mu = gen.gbs_amplitudes(M, N, sigma=0.5, seed=d)
    with lib.Sampler(precision=precision, max_microbatch=1024) as s:   # ragged tail: 2500 = 2 x 1024 + 452
        s.load_chain(ts)
        smp, lp, tr = s.sample(b, d, N, seed, trace_rows=N, mu=mu)
    rep = parity.check(b, _dq(ts, precision), seed, np.arange(N), smp, lp, TOL[precision], dev_trace=tr,
                       trace_rows=N, mu=mu)
    print(precision, d, rep)
    assert rep["prob_rows"] == N


def test_displaced_large_rows_unstaged(lib):
    """d = 16 with a 2048-wide bond: the scratch rows of site 2 (16 x 4096 floats = 256 KB) exceed the
    shared-memory staging limit and take the unstaged kernel; the other sites are staged."""
    M, d, N, seed = 6, 16, 512, 12
    b, ts, _ = gen.mps_tensors(M, d, 2048, base_seed=70, skew=4.0)
    assert max(b) == 2048
    mu = gen.gbs_amplitudes(M, N, sigma=0.5, seed=3)
    with lib.Sampler(precision="fp32") as s:
        s.load_chain(ts)
        smp, lp, tr = s.sample(b, d, N, seed, trace_rows=64, mu=mu)
    rows = np.arange(0, N, 4)
    rep = parity.check(b, ts, seed, rows, smp[rows], lp[rows], TOL["fp32"], dev_trace=tr, trace_rows=64, mu=mu)
    print(rep)


def test_displaced_device_amplitudes_and_strided(lib):
    """Device-resident amplitudes, and host amplitudes with a leading dimension above N, give the
    same result as contiguous host amplitudes."""
    import torch

    M, d, N = 16, 4, 1000
    b, ts, _ = gen.mps_tensors(M, d, 16, base_seed=8, skew=1.5)
    mu = gen.gbs_amplitudes(M, N, seed=2)
    wide = np.zeros((M, N + 24), np.complex64)
    wide[:, :N] = mu
    with lib.Sampler(precision="bf16x2") as s:
        s.load_chain(ts)
        a_s, a_l = s.sample(b, d, N, 3, mu=mu)
        b_s, b_l = s.sample(b, d, N, 3, mu=torch.from_numpy(mu).cuda())
        out_s = np.empty((N, M), np.uint8)
        out_l = np.empty(N, np.float64)
        lib.fastmps_sample_displaced(s.h, M, d, b, 0, N, 3, 0, wide, out_s, out_l)
    assert np.array_equal(a_s, b_s) and np.array_equal(a_l, b_l)
    assert np.array_equal(a_s, out_s) and np.array_equal(a_l, out_l)


def test_displaced_zero_amplitude_is_plain_sampling(lib):
    """mu = 0 makes D the identity: the displaced path reproduces the plain path's outcomes (the
    log-probabilities agree to FP32 rounding of the two measurement kernels)."""
    M, d, N = 24, 4, 4000
    b, ts, _ = gen.mps_tensors(M, d, 32, base_seed=19, skew=1.5)
    with lib.Sampler(precision="fp32") as s:
        s.load_chain(ts)
        p_s, p_l = s.sample(b, d, N, 6)
        z_s, z_l = s.sample(b, d, N, 6, mu=np.zeros((M, N), np.complex64))
    assert (p_s != z_s).mean() < 1e-3
    same = (p_s == z_s).all(axis=1)
    assert np.abs(p_l[same] - z_l[same]).max() < 1e-4


def test_displaced_errors(lib):
    M, d, N = 4, 4, 8
    b, ts, _ = gen.mps_tensors(M, d, 4, base_seed=1)
    mu = np.zeros((M, N), np.complex64)
    with lib.Sampler(precision="bf16x2") as s:
        s.load_chain(ts)
        with pytest.raises(lib.FastMPSError) as e:
            lib.fastmps_sample_displaced(s.h, M, d, b, 0, N, 1, 0, mu[:, :4], np.empty((N, M), np.uint8),
                                         np.empty(N))
        assert e.value.code == -1                    # ld_mu < N
    b17, ts17, _ = gen.mps_tensors(3, 17, 4, base_seed=1)
    with lib.Sampler(precision="fp32") as s:
        s.load_chain(ts17)
        with pytest.raises(lib.FastMPSError) as e:
            s.sample(b17, 17, N, 1, mu=np.zeros((3, N), np.complex64))
        assert e.value.code == -2                    # d above 16
    with lib.Sampler(precision="fp8x1") as s:
        s.load_chain(ts)
        with pytest.raises(lib.FastMPSError) as e:
            s.sample(b, d, N, 1, mu=mu)
        assert e.value.code == -7


def test_displaced_marginals_1e6(lib):
    """10^6 displaced samples (one fixed amplitude per site for every sample) against the exact law of
    the sequential sampler, computed by the oracle for all 3^7 configurations."""
    import itertools

    M, d, N = 7, 3, 1_000_000
    b, ts, _ = gen.mps_tensors(M, d, 9, base_seed=4, skew=1.5)
    site_mu = gen.gbs_amplitudes(M, 1, sigma=0.6, seed=9)[:, 0]
    configs = np.array(list(itertools.product(range(d), repeat=M)), np.uint8)
    mu_cfg = np.repeat(site_mu[:, None], len(configs), axis=1)
    r = oracle.replay(b, ts, 0, np.arange(len(configs)), configs, mu=mu_cfg)
    law = np.exp(r["logprob"]).reshape((d,) * M)
    assert abs(law.sum() - 1.0) < 1e-12
    mu = np.repeat(site_mu[:, None], N, axis=1).astype(np.complex64)
    with lib.Sampler(precision="fp32") as s:
        s.load_chain(ts)
        smp, _ = s.sample(b, d, N, 2024, mu=mu)
    import oracle_pins as P

    worst, where = P.marginals_5sigma(smp, law)
    print("worst z", worst, where)
    assert worst < 5.0


def test_displaced_plain_size(lib):
    """Plain workload shape (M = 256, d = 4, chi = 256, N = 2^17) with displacement, BF16x2: 256 sampled
    rows replayed by the oracle, plus the traced first rows."""
    w = gen.WORKLOADS["plain"]
    b, ts, idx = gen.mps_tensors(w.M, w.d, w.chi, base_seed=w.base_seed, skew=w.skew, pool=w.pool)
    mu = gen.gbs_amplitudes(w.M, w.N, sigma=0.3, seed=11)
    with lib.Sampler(precision="bf16x2") as s:
        s.load_chain(ts, site_index=idx)
        smp, lp, tr = s.sample(b, w.d, w.N, w.sampler_seed, trace_rows=32, mu=mu)
        st = s.stats()
    rng = np.random.Generator(np.random.PCG64(5))
    rows = np.sort(np.concatenate([np.arange(32), rng.choice(np.arange(32, w.N), 224, replace=False),
                                   [w.N - 1]]))
    rows = np.unique(rows)
    rep = parity.check(b, _dq(ts, "bf16x2"), w.sampler_seed, rows, smp[rows], lp[rows], TOL["bf16x2"],
                       dev_trace=tr, trace_rows=32, site_index=idx, mu=mu)
    print(rep, "ms_measure", st["ms_measure"], "ms_contract", st["ms_contract"])


# ---------------------------------------------------------------------------
# dynamic bond dimensions: truncated Vidal chains
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def area_law():
    return gen.area_law_vidal_chain(60, 3, 64, seed=21)


@pytest.mark.parametrize("precision", ["fp32", "bf16x2"])
def test_truncated_vidal_parity(lib, area_law, precision):
    from oracle import bond_filter as BF

    b, G, L = area_law
    bonds, disc = lib.fastmps_bond_filter(b, L, 3, 24)
    assert sum(bonds) < sum(min(x, 24) for x in b)
    Gt, Lt = BF.truncate_vidal(G, L, bonds)
    N, seed = 3000, 17
    with lib.Sampler(precision=precision, max_microbatch=1024) as s:
        s.load_chain_vidal_truncated(G, L, bonds)
        smp, lp, tr = s.sample(bonds, 3, N, seed, trace_rows=N)
    if precision == "fp32":
        rep = parity.check(bonds, Gt, seed, np.arange(N), smp, lp, TOL[precision], dev_trace=tr, trace_rows=N,
                           lams=Lt)
    else:
        stored = _dq([Gt[k] * Lt[k][None, None, :] for k in range(len(Gt))], precision)
        rep = parity.check(bonds, stored, seed, np.arange(N), smp, lp, TOL[precision], dev_trace=tr, trace_rows=N)
    print(precision, bonds[:10], rep)


def test_truncated_load_from_device_arrays(lib, area_law):
    """The leading-block gather from device memory (2D copy) equals the host gather."""
    import torch

    b, G, L = area_law
    bonds, _ = lib.fastmps_bond_filter(b, L, 3, 16)
    with lib.Sampler(precision="bf16x2") as s:
        s.load_chain_vidal_truncated(G, L, bonds)
        h_s, h_l = s.sample(bonds, 3, 1500, 8)
    with lib.Sampler(precision="bf16x2") as s:
        s.load_chain_vidal_truncated([torch.from_numpy(g).cuda() for g in G],
                                     [torch.from_numpy(l).cuda() for l in L], bonds)
        d_s, d_l = s.sample(bonds, 3, 1500, 8)
    assert np.array_equal(h_s, d_s) and np.array_equal(h_l, d_l)


@pytest.mark.parametrize("precision", ["fp32", "bf16x2"])
def test_displaced_microbatch_and_offsets_are_exact(lib, precision):
    """Displaced results depend only on (seed, n, mu[:, n]): micro-batch splits, ragged tails and n0
    offsets reproduce them bitwise (every row's reduction order is fixed by chi_r alone)."""
    M, d, N = 18, 4, 1000
    b, ts, _ = gen.mps_tensors(M, d, 64, base_seed=41, skew=1.5)
    mu = gen.gbs_amplitudes(M, N, sigma=0.5, seed=6)
    with lib.Sampler(precision=precision) as s:
        s.load_chain(ts)
        a_s, a_l = s.sample(b, d, N, 9, mu=mu)
    with lib.Sampler(precision=precision, max_microbatch=256) as s:
        s.load_chain(ts)
        b_s, b_l = s.sample(b, d, N, 9, mu=mu)
        c_s, c_l = s.sample(b, d, 100, 9, n0=333, mu=np.ascontiguousarray(mu[:, 333:433]))
        one_s, one_l = s.sample(b, d, 1, 9, n0=999, mu=np.ascontiguousarray(mu[:, 999:]))
    assert np.array_equal(a_s, b_s) and np.array_equal(a_l, b_l)
    assert np.array_equal(a_s[333:433], c_s) and np.array_equal(a_l[333:433], c_l)
    assert np.array_equal(a_s[999:], one_s) and np.array_equal(a_l[999:], one_l)


def test_displaced_host_stream_equals_resident(lib):
    """Host-streamed BF16 site tensors give the same displaced samples as resident ones."""
    M, d, N = 16, 4, 1500
    b, ts, _ = gen.mps_tensors(M, d, 32, base_seed=77, skew=1.5)
    mu = gen.gbs_amplitudes(M, N, sigma=0.4, seed=8)
    with lib.Sampler(precision="bf16x2") as s:
        s.load_chain(ts)
        r_s, r_l = s.sample(b, d, N, 5, mu=mu)
    with lib.Sampler(precision="bf16x2", residency="host_stream") as s:
        s.load_chain(ts)
        h_s, h_l = s.sample(b, d, N, 5, mu=mu)
    assert np.array_equal(r_s, h_s) and np.array_equal(r_l, h_l)


def test_vidal_pool_equals_sites(lib, vidal_chain):
    """Vidal-form pool entries mapped to sites sample exactly like the same tensors loaded per site."""
    b, G, L = vidal_chain
    M = len(G)
    with lib.Sampler(precision="bf16x2") as s:
        s.load_chain_vidal(G, L)
        a_s, a_l = s.sample(b, 3, 1000, 2)
    with lib.Sampler(precision="bf16x2") as s:
        for k in range(M):
            lib.fastmps_load_pool_vidal(s.h, k, G[k], L[k])
            lib.fastmps_map_site(s.h, k, k)
        p_s, p_l = s.sample(b, 3, 1000, 2)
    assert np.array_equal(a_s, p_s) and np.array_equal(a_l, p_l)
