"""The oracle pinned to facts other than itself (CPU only)."""
import math

import numpy as np
import pytest

import gen
import oracle
import oracle_pins as P


@pytest.mark.parametrize("pin", P.FAST_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    ok, detail = pin()
    assert ok, detail


@pytest.mark.parametrize("pin", P.QUANT_PINS, ids=lambda f: f.__name__)
def test_quant_pin(pin):
    from oracle import quant

    ok, detail = pin(quant)
    assert ok, detail


@pytest.mark.parametrize("pin", P.BOND_FILTER_PINS, ids=lambda f: f.__name__)
def test_bond_filter_pin(pin):
    from oracle import bond_filter as BF

    ok, detail = pin(BF)
    assert ok, detail


def test_uniform_range_and_uniformity():
    n = 200_000
    u = np.array([oracle.uniform(42, i, 7) for i in range(0, n)])
    assert (u > 0).all() and (u < 1).all()
    # 53-bit grid: u * 2^53 - 1/2 is an integer
    g = u * float(1 << 53) - 0.5
    assert np.all(g == np.floor(g))
    # chi-square on 100 equiprobable bins (p-value > 1e-6 at 99 dof: stat < 190)
    h = np.bincount(np.minimum((u * 100).astype(int), 99), minlength=100)
    stat = ((h - n / 100) ** 2 / (n / 100)).sum()
    assert stat < 190, stat
    # the low bits carry entropy too (from the second output word)
    low = (g.astype(np.uint64) & np.uint64(0xFF)).astype(int)
    assert len(np.unique(low)) == 256


def test_generator_right_canonical():
    for (M, d, chi, skew) in ((12, 3, 16, None), (9, 4, 32, 1.5), (6, 6, 20, 1.5)):
        b, ts, _ = gen.mps_tensors(M, d, chi, base_seed=21, skew=skew)
        assert b[0] == 1 and b[-1] == 1
        for k, A in enumerate(ts):
            cl, dd, cr = A.shape
            assert (cl, dd, cr) == (b[k], d, b[k + 1])
            G = np.einsum("asb,csb->ac", A, A.conj())
            assert np.abs(G - np.eye(cl)).max() < 1e-12


def test_bond_profile():
    assert gen.bond_dims(12, 3, 16) == [1, 3, 9, 16, 16, 16, 16, 16, 16, 16, 9, 3, 1]
    b = gen.bond_dims(256, 4, 256)
    assert b[:6] == [1, 4, 16, 64, 256, 256] and b[-5:] == [256, 64, 16, 4, 1]


def test_skew_tilts_outcomes():
    """The exp(-s/1.5) skew makes low outcomes dominate (GBS-like photon statistics)."""
    b, ts, _ = gen.mps_tensors(40, 4, 16, base_seed=8, skew=1.5)
    smp, _ = oracle.sample(b, ts, 1, 2000)
    f = np.bincount(smp.reshape(-1), minlength=4) / smp.size
    assert f[0] > f[1] > f[2] > f[3]


def test_replay_follows_own_path():
    b, ts = P._tiny()
    smp, lp, pr = oracle.sample(b, ts, 42, 64, want_probs=True)
    rows = np.arange(64)
    r = oracle.replay(b, ts, 42, rows, smp)
    assert (r["own"] == smp).all()
    assert np.array_equal(r["probs"], pr)
    assert np.array_equal(r["logprob"], lp)
    assert (r["margin"] >= 0).all() and (r["margin"] <= 1).all()


def test_replay_noncontiguous_rows_and_offset():
    b, ts = P._tiny()
    smp, lp = oracle.sample(b, ts, 42, 50, n0=1000)
    rows = np.array([1003, 1004, 1020, 1049])
    r = oracle.replay(b, ts, 42, rows, smp[rows - 1000])
    assert (r["own"] == smp[rows - 1000]).all()
    assert np.allclose(r["logprob"], lp[rows - 1000], rtol=0, atol=0)


def test_replay_other_path_changes_own_draws():
    """Forcing a different prefix changes the later conditionals (the chain has memory)."""
    b, ts = P._tiny()
    smp, _ = oracle.sample(b, ts, 42, 1)
    forced = smp.copy()
    forced[0, 2] = (forced[0, 2] + 1) % 3
    r0 = oracle.replay(b, ts, 42, [0], smp)
    r1 = oracle.replay(b, ts, 42, [0], forced)
    assert np.abs(r0["probs"][0, 3] - r1["probs"][0, 3]).max() > 1e-6


@pytest.mark.slow
def test_marginals_within_5_sigma(tiny_chain, tiny_brute):
    b, ts = tiny_chain
    smp, _ = oracle.sample(b, ts, 2024, 100_000)
    worst, where = P.marginals_5sigma(smp, tiny_brute)
    assert worst < 5.0, (worst, where)


def test_offset_rows_match():
    """Row n's result depends only on (seed, n): sampling a sub-range reproduces it."""
    b, ts = P._tiny()
    s_all, l_all = oracle.sample(b, ts, 42, 300)
    s_sub, l_sub = oracle.sample(b, ts, 42, 100, n0=150)
    assert np.array_equal(s_all[150:250], s_sub)
    assert np.array_equal(l_all[150:250], l_sub)


def test_thread_count_independent():
    b, ts = P._tiny()
    s1, l1 = oracle.sample(b, ts, 42, 500, nthreads=1)
    s2, l2 = oracle.sample(b, ts, 42, 500, nthreads=4)
    assert np.array_equal(s1, s2) and np.array_equal(l1, l2)


def test_thread_count_of_one_call_does_not_stick():
    """A call with an explicit thread count (the one-core CPU baseline) leaves the process's default
    thread count, which later calls and the baseline's reported core count use, unchanged."""
    b, ts = P._tiny()
    before = oracle.num_threads()
    oracle.sample(b, ts, 42, 40, nthreads=1)
    assert oracle.num_threads() == before


def test_row_batching_changes_no_result():
    """Rows are contracted in batches of up to 8 per thread, fewer when the rows would not keep every
    thread busy; a row's sums do not depend on its batch, so 24 rows with 1, 6 and 24 threads (batches of
    8, 4 and 1 rows) give bitwise the same outcomes, log-probabilities, conditionals and replays."""
    b, ts = P._tiny()
    runs = [oracle.sample(b, ts, 42, 24, want_probs=True, nthreads=t) for t in (1, 6, 24)]
    for smp, lp, pr in runs[1:]:
        assert np.array_equal(smp, runs[0][0]) and np.array_equal(lp, runs[0][1]) and np.array_equal(pr, runs[0][2])
    rows = np.arange(3, 24, 2)
    reps = [oracle.replay(b, ts, 42, rows, runs[0][0][rows], nthreads=t) for t in (1, 5, 16)]
    for r in reps[1:]:
        for key in ("probs", "own", "margin", "logprob"):
            assert np.array_equal(r[key], reps[0][key]), key


def test_pool_site_index():
    b, ts, idx = gen.mps_tensors(40, 3, 9, base_seed=4, pool=4)
    assert len(ts) < 40
    full = [ts[j] for j in idx]
    s1, l1 = oracle.sample(b, ts, 1, 50, site_index=idx)
    s2, l2 = oracle.sample(b, full, 1, 50)
    assert np.array_equal(s1, s2) and np.array_equal(l1, l2)
    assert all(math.isfinite(x) for x in l1)


def test_segmented_replay_equals_whole_chain():
    """Replaying 5 sites at a time with carried left vectors gives the whole-chain result bitwise."""
    b, ts = P._tiny()
    smp, lp, pr = oracle.sample(b, ts, 42, 40, want_probs=True)
    r1 = oracle.replay(b, ts, 42, np.arange(40), smp)
    r2 = oracle.replay(b, lambda k: ts[k], 42, np.arange(40), smp, site_chunk=5)
    for key in ("probs", "own", "margin"):
        assert np.array_equal(r1[key], r2[key]), key
    assert np.allclose(r1["logprob"], r2["logprob"], rtol=0, atol=1e-13)
    assert np.array_equal(r1["probs"], pr)


def test_prefix_sampling_and_complex64_inputs():
    b, ts = P._tiny()
    smp, lp = oracle.sample(b, ts, 42, 30)
    s5, _ = oracle.sample_prefix(b, ts[:5], 42, 30, 5)
    assert np.array_equal(s5, smp[:, :5])
    t64 = [t.astype(np.complex64) for t in ts]
    widened = [t.astype(np.complex128) for t in t64]
    a, la = oracle.sample(b, t64, 42, 30)
    c, lc = oracle.sample(b, widened, 42, 30)
    assert np.array_equal(a, c) and np.array_equal(la, lc)


def test_vidal_form_generator():
    """Gamma_k Lambda_k is right-canonical and Lambda_k is a normalised descending spectrum."""
    b, ts, _ = gen.mps_tensors(10, 3, 9, base_seed=3, skew=1.5)
    G, L = gen.vidal_form(b, ts)
    for k in range(10):
        B = G[k] * L[k][None, None, :]
        E = np.einsum("asb,csb->ac", B, B.conj())
        assert np.abs(E - np.eye(B.shape[0])).max() < 1e-10
        assert abs(np.sum(L[k] ** 2) - 1.0) < 1e-12 and np.all(np.diff(L[k]) <= 1e-15)
    b2, G2, L2 = gen.decaying_vidal_chain(6, 4, 16)
    for k in range(6):
        B = G2[k] * L2[k][None, None, :]
        assert np.abs(np.einsum("asb,csb->ac", B, B.conj()) - np.eye(B.shape[0])).max() < 1e-10


@pytest.mark.parametrize("n", [4, 6, 10])
def test_zassenhaus_vs_truncated_expm(n):
    """Against a dense FP64 expm of the generator truncated at the same n levels, the Zassenhaus
    matrix differs by < 0.2 % (relative, per element) on the elements of photon numbers at least
    two below the cutoff (i, j <= n-3) that are not negligible (>= 1e-3 of the largest), for
    |mu| <= 0.3.  Near the cutoff the same-size expm is itself the inexact one: it drops the
    coupling to level n, which the Zassenhaus product (equal to the closed form, pinned above)
    keeps."""
    import scipy.linalg

    a = np.diag(np.sqrt(np.arange(1, n)), 1)
    rng = np.random.Generator(np.random.PCG64(n))
    worst = 0.0
    for _ in range(300):
        mu = 0.3 * math.sqrt(rng.random()) * np.exp(2j * math.pi * rng.random())
        E = scipy.linalg.expm(mu * a.T - np.conj(mu) * a)
        Z = oracle.displacement(mu, n)
        sel = np.zeros((n, n), bool)
        sel[: n - 2, : n - 2] = True
        sel &= np.abs(E) >= 1e-3 * np.abs(E).max()
        rel = np.abs(Z - E)[sel] / np.abs(E)[sel]
        worst = max(worst, float(rel.max()))
    assert worst < 2e-3, worst


# ---------------------------------------------------------------------------
# dynamic bond-dimension filter (Sec. 3.4.2)
# ---------------------------------------------------------------------------

def test_bond_filter_geometric_spectrum_closed_form():
    """Lambda_j^2 = q^j (n values): eps(c) = (q^c - q^n) / (1 - q^n); the least c with eps(c) <= e is
    ceil(log(e (1 - q^n) + q^n) / log q)."""
    from oracle import bond_filter as BF

    for q, n, e in ((0.5, 40, 1e-6), (0.9, 200, 1e-3), (0.99, 500, 0.05), (0.7, 10, 1e-2)):
        lam = [math.sqrt(q ** j) for j in range(n)]
        want = math.ceil(math.log(e * (1 - q ** n) + q ** n) / math.log(q) - 1e-9)
        bonds, disc, es = BF.filter_bonds([lam, [1.0]], d=n, chi=n, eps=e)
        assert bonds[1] == max(1, want), (q, n, e, bonds[1], want)
        assert disc[1] <= e and abs(disc[1] - (q ** bonds[1] - q ** n) / (1 - q ** n)) < 1e-12


def test_bond_filter_invariants():
    """Budget = the fixed-chi filter's largest error; every bond within it, minimal, <= chi; the maximum
    error over bonds equals the fixed-chi one; edges keep fewer than the centre; isometry shapes hold."""
    from oracle import bond_filter as BF

    M, d, chi = 40, 3, 24
    b, G, L = gen.area_law_vidal_chain(M, d, 64)                  # spectra of up to 64 values, cap 24
    bonds, disc, es = BF.filter_bonds(L, d, chi)
    fixed = [BF.discarded_weight(L[k], min(chi, len(L[k]))) for k in range(M - 1)]
    assert es == max(fixed) > 0
    assert max(disc) == es or max(disc) <= es
    for k in range(M - 1):
        c = bonds[k + 1]
        assert 1 <= c <= min(chi, len(L[k]))
        assert disc[k + 1] <= es
        assert bonds[k] <= d * c
    assert bonds[2] < bonds[M // 2] and bonds[M - 2] < bonds[M // 2]
    assert sum(bonds) < sum(min(x, chi) for x in b)
    # minimality where the isometry rule did not raise the count
    for k in range(M - 1):
        c = bonds[k + 1]
        if c > 1 and c > -(-bonds[k] // d):
            assert BF.discarded_weight(L[k], c - 1) > es


def test_bond_filter_alignment():
    """Aligned counts: multiples of the alignment except where capped or raised for the isometry shape;
    never below the unaligned counts; discarded weights within the budget."""
    from oracle import bond_filter as BF

    M, d, chi = 40, 3, 48
    b, G, L = gen.area_law_vidal_chain(M, d, 64)
    plain, _, es = BF.filter_bonds(L, d, chi)
    al, disc, es2 = BF.filter_bonds(L, d, chi, align=16)
    assert es == es2
    for k in range(1, M):
        cap = min(chi, len(L[k - 1]))
        assert al[k] >= plain[k] and disc[k] <= es
        assert al[k] % 16 == 0 or al[k] == cap or al[k] == -(-al[k - 1] // d)


def test_truncated_vidal_sampling_error_bounded():
    """The Born law of the truncated chain stays within total-variation distance 2 sqrt(sum of discarded
    weights) of the full chain's (norm bound of Schmidt truncation; tiny chain, exact laws by brute
    force on both chains)."""
    from oracle import bond_filter as BF

    M, d, chi = 9, 3, 27
    b, G, L = gen.area_law_vidal_chain(M, d, chi, xi_max=3.0, seed=5)
    bonds, disc, es = BF.filter_bonds(L, d, chi, eps=1e-3)
    Gt, Lt = BF.truncate_vidal(G, L, bonds)
    full = oracle.brute_force(b, [G[k] * L[k][None, None, :] for k in range(M)])
    trunc = oracle.brute_force(bonds, [Gt[k] * Lt[k][None, None, :] for k in range(M)])
    trunc /= trunc.sum()
    assert sum(bonds) < sum(b)
    tv = 0.5 * np.abs(full - trunc).sum()
    assert tv < 2 * math.sqrt(sum(disc)), (tv, sum(disc))


def test_displacement_special_cases():
    """mu = 0: D is the identity and displaced sampling is plain sampling (bitwise); for a large
    truncation the leading block of D^dagger D is the identity (unitarity of the untruncated operator)."""
    for n in (2, 5, 9):
        assert np.array_equal(oracle.displacement(0.0, n), np.eye(n))
    b, ts, _ = gen.mps_tensors(10, 3, 9, base_seed=2, skew=1.5)
    s0, l0, p0 = oracle.sample(b, ts, 4, 200, want_probs=True)
    s1, l1, p1 = oracle.sample(b, ts, 4, 200, want_probs=True, mu=np.zeros((10, 200), np.complex128))
    assert np.array_equal(s0, s1) and np.array_equal(l0, l1) and np.array_equal(p0, p1)
    for mu in (0.3 + 0.1j, -0.5j, 0.8):
        D = oracle.displacement(mu, 60)
        G = (D.conj().T @ D)[:10, :10]
        assert np.abs(G - np.eye(10)).max() < 1e-12


def test_area_law_chain_torch_route_is_a_vidal_form():
    """The device route of the area-law generator (run here with torch on the CPU) yields a valid Vidal
    form: Gamma_k Lambda_k right-canonical (complex64 rounding) and Lambda_k the chain's Schmidt
    coefficients (an independent SVD sweep of Gamma Lambda reproduces them)."""
    b, G, L = gen.area_law_vidal_chain(10, 3, 27, xi_max=3.0, seed=5, device="cpu")
    Gs = [g.numpy().astype(np.complex128) for g in G]
    Ls = [l.numpy() for l in L]
    A = [Gs[k] * Ls[k][None, None, :] for k in range(10)]
    for B in A:
        E = np.einsum("asb,csb->ac", B, B.conj())
        assert np.abs(E - np.eye(B.shape[0])).max() < 1e-6
    _, L2 = gen.vidal_form(b, A)
    assert max(float(np.abs(L2[k] - Ls[k]).max()) for k in range(10)) < 1e-6
