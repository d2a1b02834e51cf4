"""Pins for the FP64 oracle: checks against facts fixed by the paper and the mathematics.

Each ``pin_*`` function runs one check against an oracle library (the built
one by default, or a mutated copy) and returns ``(ok, detail)``.  The tests in
``test_oracle_pins.py`` require every pin to pass on the real oracle, and
``test_oracle_mutants.py`` plants mistakes in copies of the oracle and requires
that some pin fails for each.

What pins what
--------------
* ``pin_philox_kat``      -- Philox4x32-10 known-answer vectors (golden file).
* ``pin_uniform_packing`` -- key/counter packing and the 53-bit mapping, from the
  same vectors, computed here from the golden numbers (not from the oracle).
* ``pin_brute_force_normalised`` -- sum of |psi(s)|^2 over all d^M is 1 for a
  right-canonical MPS (norm of a normalised state).
* ``pin_conditionals_vs_brute`` -- each conditional p(s | prefix) the sampler
  reports equals P(prefix, s) / P(prefix) from brute-force summation.
* ``pin_logprob_vs_brute`` -- exp(sum of log conditionals) equals the brute-force
  Born probability of the sampled configuration.
* ``pin_product_state``   -- chi = 1: the conditionals are the given per-site laws
  and each outcome is the inverse-CDF draw of that law at the sample's uniform.
* ``pin_ghz``             -- GHZ chain: perfectly correlated outcomes, log p = -log d.
* ``pin_scale_invariance`` -- multiplying every site tensor by a constant changes
  neither the outcomes nor the log-probabilities (the normalisation by Z).
* ``pin_long_chain``      -- 3000 sites: log-probabilities stay finite and equal the
  closed-form log |A_0[s_0] ... A_{M-1}[s_{M-1}]|^2 (per-sample rescaling).
* ``pin_marginals``       -- single-site and nearest-pair marginals of 10^5 samples
  within 5 sigma of brute force (in test_oracle_pins only; slow for mutants).
* ``pin_displacement_closed_form`` -- the Zassenhaus matrix of Sec. 3.4.1 equals the
  matrix elements of the displacement operator, <m|D(mu)|n> = sqrt(n!/m!) mu^(m-n)
  exp(-|mu|^2/2) L_n^(m-n)(|mu|^2) (generalised Laguerre polynomial, scipy), and the
  top-left block of a dense FP64 expm (scipy) of the generator in a 60-level space.
* ``pin_displaced_conditionals_vs_brute`` -- with per-sample displacements, each
  conditional equals the marginal of the full state vector displaced (closed-form
  matrices, numpy) on sites 0..k, right of k summed out.
* ``pin_vidal_conditionals_vs_brute`` / ``pin_vidal_logprob`` -- Vidal-form sampling
  (Gamma, Lambda) reproduces the brute-force Born law of the state
  Gamma_0 Lambda_0 Gamma_1 Lambda_1 ... for a converted chain and for a chain with
  decaying Schmidt spectra.
* ``QUANT_PINS`` (oracle/quant.py) -- bfloat16 and E4M3 rounding on hand-derived cases
  (ties to even of both parities, carries into the exponent, subnormal grids, the E4M3
  2^-6 boundary and saturation at 448, signed zero), cross-checked against torch's
  bfloat16 / float8_e4m3fn casts called as a library; the hi/lo split holds 16
  significant bits (binary16: 22); the FP8 site scale is the power of two that puts
  max|Re, Im| in [224, 448].
"""
from __future__ import annotations

import math
import os

import numpy as np

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def _tiny():
    w = gen.WORKLOADS["tiny"]
    b, ts, _ = gen.mps_tensors(w.M, w.d, w.chi, base_seed=w.base_seed, skew=w.skew)
    return b, ts


def pin_philox_kat(lib=None):
    for ctr, key, want in read_kat():
        got = [int(x) for x in oracle.philox(ctr, key, lib=lib)]
        if got != want:
            return False, f"philox({ctr},{key}) = {got} != {want}"
    return True, ""


def pin_uniform_packing(lib=None):
    """seed = key1:key0, n = ctr1:ctr0, k = ctr2, job = ctr3; u = (x0<<21 | x1>>11) + 1/2 over 2^53."""
    for ctr, key, want in read_kat():
        seed = (key[1] << 32) | key[0]
        n = (ctr[1] << 32) | ctr[0]
        bits = (want[0] << 21) | (want[1] >> 11)
        u_want = (bits + 0.5) / float(1 << 53)
        u = oracle.uniform(seed, n, ctr[2], ctr[3], lib=lib)
        if u != u_want:
            return False, f"uniform({seed:#x},{n:#x},{ctr[2]:#x},{ctr[3]:#x}) = {u!r} != {u_want!r}"
    return True, ""


def pin_brute_force_normalised(lib=None):
    cases = [(_tiny()), gen.mps_tensors(10, 2, 8, base_seed=77)[:2], gen.mps_tensors(7, 4, 12, base_seed=5,
                                                                                        skew=1.5)[:2]]
    for b, ts in cases:
        p = oracle.brute_force(b, ts, lib=lib)
        if not abs(p.sum() - 1.0) < 1e-12 or p.min() < 0:
            return False, f"sum |psi|^2 = {p.sum()!r}"
    return True, ""


def _prefix_marg(bf, prefix):
    return bf[tuple(prefix)].sum()


def pin_conditionals_vs_brute(lib=None, rows=40, seed=42):
    b, ts = _tiny()
    bf = oracle.brute_force(b, ts)  # the real brute force: this pin checks the sampler
    smp, lp, pr = oracle.sample(b, ts, seed, rows, want_probs=True, lib=lib)
    M = len(b) - 1
    worst = 0.0
    for i in range(rows):
        for k in range(M):
            pre = list(smp[i, :k])
            den = _prefix_marg(bf, pre)
            for s in range(bf.shape[0]):
                num = _prefix_marg(bf, pre + [s])
                worst = max(worst, abs(pr[i, k, s] - num / den))
    if not worst < 1e-12:
        return False, f"max |p_oracle - p_brute| = {worst:.3e}"
    return True, ""


def pin_logprob_vs_brute(lib=None, rows=200, seed=42):
    b, ts = _tiny()
    bf = oracle.brute_force(b, ts)
    smp, lp = oracle.sample(b, ts, seed, rows, lib=lib)
    for i in range(rows):
        p = bf[tuple(smp[i])]
        if not (p > 0 and abs(lp[i] - math.log(p)) < 1e-11):
            return False, f"row {i}: logp = {lp[i]!r}, log |psi|^2 = {math.log(p) if p > 0 else p!r}"
        born = oracle.born_logprob(b, ts, smp[i], lib=lib)  # closed form
        if not abs(born - math.log(p)) < 1e-11:
            return False, f"row {i}: born_logprob {born!r} vs log brute {math.log(p)!r}"
    return True, ""


def pin_product_state(lib=None, seed=9, N=400):
    rng = np.random.Generator(np.random.PCG64(3))
    M, d = 20, 4
    laws = rng.random((M, d)) ** 2
    laws[3] = [0.0, 1.0, 0.0, 0.0]          # a certain outcome
    laws[4] = [0.5, 0.0, 0.0, 0.5]          # zero-probability middle outcomes
    laws /= laws.sum(axis=1, keepdims=True)
    b, ts = gen.product_state(M, laws)
    smp, lp, pr = oracle.sample(b, ts, seed, N, want_probs=True, lib=lib)
    if not np.abs(pr - laws[None]).max() < 1e-14:
        return False, f"conditionals differ from the per-site laws by {np.abs(pr - laws[None]).max():.3e}"
    cdf = np.cumsum(laws, axis=1)
    for i in range(N):
        want_lp = 0.0
        for k in range(M):
            u = oracle.uniform(seed, i, k)    # the generator is pinned on its own above
            s = int(np.sum(cdf[k, :d - 1] < u * cdf[k, -1]))
            if smp[i, k] != s:
                return False, f"row {i} site {k}: outcome {smp[i, k]} != inverse-CDF draw {s}"
            want_lp += math.log(laws[k, s])
        if not abs(lp[i] - want_lp) < 1e-12:
            return False, f"row {i}: logp {lp[i]!r} != {want_lp!r}"
    return True, ""


def pin_ghz(lib=None, N=3000, seed=5):
    for M, d in ((8, 3), (16, 2), (5, 4)):
        b, ts = gen.ghz_chain(M, d)
        smp, lp = oracle.sample(b, ts, seed, N, lib=lib)
        if not (smp == smp[:, :1]).all():
            return False, f"GHZ(M={M},d={d}): outcomes not perfectly correlated"
        if not np.abs(lp + math.log(d)).max() < 1e-12:
            return False, f"GHZ(M={M},d={d}): logp != -log d"
        f = np.bincount(smp[:, 0], minlength=d) / N
        sig = math.sqrt((1 / d) * (1 - 1 / d) / N)
        if not np.abs(f - 1 / d).max() < 5 * sig:
            return False, f"GHZ first-site frequencies {f}"
    return True, ""


def pin_scale_invariance(lib=None, N=200, seed=11):
    b, ts = _tiny()
    scaled = [t * (1.7 if k % 2 else 0.6) for k, t in enumerate(ts)]
    s0, l0, p0 = oracle.sample(b, ts, seed, N, want_probs=True, lib=lib)
    s1, l1, p1 = oracle.sample(b, scaled, seed, N, want_probs=True, lib=lib)
    if not (s0 == s1).all():
        return False, "outcomes change when site tensors are scaled"
    if not np.abs(l0 - l1).max() < 1e-11:
        return False, f"logp changes by {np.abs(l0 - l1).max():.3e} when site tensors are scaled"
    if not np.abs(p0 - p1).max() < 1e-12:
        return False, "conditionals change when site tensors are scaled"
    return True, ""


def pin_long_chain(lib=None, N=8, seed=3):
    b, ts, _ = gen.mps_tensors(3000, 4, 4, base_seed=100, skew=1.5)
    smp, lp = oracle.sample(b, ts, seed, N, lib=lib)
    for i in range(N):
        if not math.isfinite(lp[i]):
            return False, f"row {i}: logp {lp[i]!r} is not finite"
        born = oracle.born_logprob(b, ts, smp[i], lib=lib)
        if not abs(lp[i] - born) < 1e-8 * max(1.0, abs(born)):
            return False, f"row {i}: logp {lp[i]!r} vs closed form {born!r}"
    return True, ""


def displacement_closed_form(mu: complex, n: int) -> np.ndarray:
    """<m|D(mu)|j> for m, j < n from the Laguerre closed form (Cahill-Glauber)."""
    from scipy.special import eval_genlaguerre

    x = abs(mu) ** 2
    g = math.exp(-x / 2)
    D = np.zeros((n, n), np.complex128)
    for m in range(n):
        for j in range(n):
            if m >= j:
                D[m, j] = math.sqrt(math.factorial(j) / math.factorial(m)) * mu ** (m - j) * g * \
                    eval_genlaguerre(j, m - j, x)
            else:
                D[m, j] = math.sqrt(math.factorial(m) / math.factorial(j)) * (-np.conj(mu)) ** (j - m) * g * \
                    eval_genlaguerre(m, j - m, x)
    return D


def pin_displacement_closed_form(lib=None):
    import scipy.linalg

    big = 60
    a = np.diag(np.sqrt(np.arange(1, big)), 1)
    rng = np.random.Generator(np.random.PCG64(17))
    for n in (2, 3, 4, 6, 10):
        for _ in range(6):
            mu = complex(*(rng.standard_normal(2) * 0.6))
            got = oracle.displacement(mu, n, lib=lib)
            want = displacement_closed_form(mu, n)
            err = np.abs(got - want).max()
            if not err < 1e-12:
                return False, f"n={n} mu={mu:.3f}: |D - closed form| = {err:.3e}"
            E = scipy.linalg.expm(mu * a.T - np.conj(mu) * a)[:n, :n]
            err = np.abs(got - E).max()
            if not err < 1e-10:
                return False, f"n={n} mu={mu:.3f}: |D - expm block| = {err:.3e}"
    return True, ""


def _state_vector(bonds, tensors):
    """psi[s_0, ..., s_{M-1}] by plain tensor contraction (numpy)."""
    psi = np.ones((1, 1), np.complex128)          # [configs so far, bond]
    for A in tensors:
        cl, d, cr = A.shape
        psi = np.einsum("xa,asb->xsb", psi, A).reshape(-1, cr)
    return psi.reshape(-1)


def pin_displaced_conditionals_vs_brute(lib=None, rows=12, seed=77):
    M, d, chi = 7, 3, 9
    b, ts, _ = gen.mps_tensors(M, d, chi, base_seed=31, skew=1.5)
    psi = _state_vector(b, ts).reshape((d,) * M)
    mu = gen.gbs_amplitudes(M, rows, sigma=0.5, seed=5).astype(np.complex128)
    smp, lp, pr = oracle.sample(b, ts, seed, rows, want_probs=True, lib=lib, mu=mu)
    worst = 0.0
    for i in range(rows):
        Ds = [displacement_closed_form(complex(mu[k, i]), d) for k in range(M)]
        phi = psi
        for k in range(M):
            phi = np.moveaxis(np.tensordot(Ds[k], phi, axes=([1], [k])), 0, k)   # displace site k
            pre = tuple(int(x) for x in smp[i, :k])
            block = np.abs(phi[pre]) ** 2                                       # axes: s_k, s_{k+1}, ...
            marg = block.reshape(d, -1).sum(axis=1)
            worst = max(worst, float(np.abs(pr[i, k] - marg / marg.sum()).max()))
    if not worst < 1e-12:
        return False, f"max |p_oracle - p_brute| = {worst:.3e}"
    return True, ""


def _vidal_cases():
    b, ts = _tiny()
    g1, l1 = gen.vidal_form(b, ts)
    b2, g2, l2 = gen.decaying_vidal_chain(8, 3, 12, decay=0.4, seed=3)
    return [(b, ts, g1, l1), (b2, [g2[k] * l2[k][None, None, :] for k in range(8)], g2, l2)]


def pin_vidal_conditionals_vs_brute(lib=None, rows=25, seed=8):
    worst = 0.0
    for b, state, G, L in _vidal_cases():
        bf = oracle.brute_force(b, state)           # Born law of Gamma_0 Lambda_0 Gamma_1 Lambda_1 ...
        smp, lp, pr = oracle.sample(b, G, seed, rows, want_probs=True, lib=lib, lams=L)
        M = len(b) - 1
        for i in range(rows):
            for k in range(M):
                pre = list(smp[i, :k])
                den = _prefix_marg(bf, pre)
                for s in range(bf.shape[0]):
                    worst = max(worst, abs(pr[i, k, s] - _prefix_marg(bf, pre + [s]) / den))
    if not worst < 1e-11:
        return False, f"max |p_vidal - p_brute| = {worst:.3e}"
    return True, ""


def pin_vidal_logprob(lib=None, rows=100, seed=21):
    for b, state, G, L in _vidal_cases():
        bf = oracle.brute_force(b, state)
        smp, lp = oracle.sample(b, G, seed, rows, lib=lib, lams=L)
        for i in range(rows):
            p = bf[tuple(smp[i])]
            if not (p > 0 and abs(lp[i] - math.log(p)) < 1e-10):
                return False, f"row {i}: logp {lp[i]!r} vs log |psi|^2 {math.log(p) if p > 0 else p!r}"
    return True, ""


FAST_PINS = [pin_philox_kat, pin_uniform_packing, pin_brute_force_normalised, pin_conditionals_vs_brute,
             pin_logprob_vs_brute, pin_product_state, pin_ghz, pin_scale_invariance, pin_long_chain,
             pin_displacement_closed_form, pin_displaced_conditionals_vs_brute, pin_vidal_conditionals_vs_brute,
             pin_vidal_logprob]


def marginals_5sigma(samples: np.ndarray, bf: np.ndarray):
    """Return the worst |f - p| / sigma over single-site and nearest-pair marginals."""
    N, M = samples.shape
    d = bf.shape[0]
    worst = 0.0
    where = ""
    for k in range(M):
        axes = tuple(a for a in range(M) if a != k)
        p = bf.sum(axis=axes)
        f = np.bincount(samples[:, k], minlength=d) / N
        sig = np.sqrt(np.maximum(p * (1 - p), 1e-300) / N)
        z = np.abs(f - p) / sig
        z[(p == 0) & (f == 0)] = 0
        if z.max() > worst:
            worst, where = float(z.max()), f"site {k}"
    for k in range(M - 1):
        axes = tuple(a for a in range(M) if a not in (k, k + 1))
        p = bf.sum(axis=axes).reshape(-1)
        f = np.bincount(samples[:, k].astype(np.int64) * d + samples[:, k + 1], minlength=d * d) / N
        sig = np.sqrt(np.maximum(p * (1 - p), 1e-300) / N)
        z = np.abs(f - p) / sig
        z[(p == 0) & (f == 0)] = 0
        if z.max() > worst:
            worst, where = float(z.max()), f"pair ({k},{k+1})"
    return worst, where


# ---------------------------------------------------------------------------
# Dynamic bond-dimension filter (Sec. 3.4.2): pins taking the filter module as an argument, so that
# mutated copies can be checked too
# ---------------------------------------------------------------------------

def pin_bf_geometric(BF):
    """Lambda_j^2 = q^j: eps(c) = (q^c - q^n) / (1 - q^n), least c with eps(c) <= e is
    ceil(log(e (1 - q^n) + q^n) / log q); the discarded weight reported is that closed form."""
    for q, n, e in ((0.5, 40, 1e-6), (0.9, 200, 1e-3), (0.99, 500, 0.05), (0.7, 10, 1e-2)):
        lam = [math.sqrt(q ** j) for j in range(n)]
        want = max(1, math.ceil(math.log(e * (1 - q ** n) + q ** n) / math.log(q) - 1e-9))
        bonds, disc, _ = BF.filter_bonds([lam, [1.0]], d=n, chi=n, eps=e)
        if bonds[1] != want:
            return False, f"q={q} n={n} e={e}: kept {bonds[1]} != {want}"
        if not abs(disc[1] - (q ** bonds[1] - q ** n) / (1 - q ** n)) < 1e-12:
            return False, f"discarded weight {disc[1]!r} is not the closed form"
    return True, ""


def pin_bf_budget_and_minimality(BF):
    """Default budget = the largest discarded weight of keeping min(chi, n) at any bond; every bond within
    it and minimal (where the isometry rule did not raise it); isometry shapes hold."""
    M, d, chi = 40, 3, 24
    b, G, L = gen.area_law_vidal_chain(M, d, 64)
    bonds, disc, es = BF.filter_bonds(L, d, chi)
    fixed = []
    for k in range(M - 1):
        lam2 = np.asarray(L[k], np.float64) ** 2
        c = min(chi, len(L[k]))
        fixed.append(float(lam2[c:].sum() / lam2.sum()))
    if not abs(es - max(fixed)) <= 1e-12 * max(fixed):
        return False, f"budget {es!r} != largest fixed-chi discarded weight {max(fixed)!r}"
    for k in range(M - 1):
        c = bonds[k + 1]
        lam2 = np.asarray(L[k], np.float64) ** 2
        if not 1 <= c <= min(chi, len(L[k])):
            return False, f"bond {k + 1}: {c} outside [1, cap]"
        if not lam2[c:].sum() / lam2.sum() <= es * (1 + 1e-12):
            return False, f"bond {k + 1}: discarded weight above the budget"
        if bonds[k] > d * c:
            return False, f"site {k}: d * chi_r < chi_l"
        if c > 1 and c > -(-bonds[k] // d) and lam2[c - 1:].sum() / lam2.sum() <= es * (1 - 1e-12):
            return False, f"bond {k + 1}: {c} is not the least count within the budget"
    if not (bonds[2] < bonds[M // 2] and bonds[M - 2] < bonds[M // 2]):
        return False, "edges do not keep fewer coefficients than the centre"
    return True, ""


def pin_bf_alignment(BF):
    """Aligned counts are multiples of the alignment unless capped or raised for an isometry shape, and
    never below the unaligned counts."""
    M, d, chi = 40, 3, 48
    b, G, L = gen.area_law_vidal_chain(M, d, 64)
    plain, _, _ = BF.filter_bonds(L, d, chi)
    al, _, _ = BF.filter_bonds(L, d, chi, align=16)
    for k in range(1, M):
        cap = min(chi, len(L[k - 1]))
        if al[k] < plain[k]:
            return False, f"bond {k}: aligned {al[k]} below unaligned {plain[k]}"
        if not (al[k] % 16 == 0 or al[k] == cap or al[k] == -(-al[k - 1] // d)):
            return False, f"bond {k}: {al[k]} is not aligned"
    return True, ""


def pin_bf_isometry_raise(BF):
    """A flat spectrum followed by a peaked one: the threshold keeps 4 then 1, and the isometry rule must
    raise the second count to ceil(4 / d) = 2 (d = 2), since a site needs d * chi_r >= chi_l."""
    flat = [0.5] * 4
    peaked = [1.0] + [1e-9] * 7
    bonds, disc, _ = BF.filter_bonds([flat, peaked, [1.0]], d=2, chi=8, eps=1e-12)
    if bonds != [1, 4, 2, 1]:
        return False, f"bonds {bonds} != [1, 4, 2, 1]"
    return True, ""


BOND_FILTER_PINS = [pin_bf_geometric, pin_bf_budget_and_minimality, pin_bf_alignment, pin_bf_isometry_raise]


# ---------------------------------------------------------------------------
# Low-precision storage formats (oracle/quant.py; Sec. 3.3.2 16-bit storage, the FP8 experiment):
# pins taking the module as an argument, so that mutated copies can be checked too.  The expected
# values are derived by hand from the format definitions (bfloat16: 8 significant bits, 8 exponent
# bits, round to nearest, ties to even; E4M3FN: 4 significant bits, bias 7, subnormal spacing 2^-9,
# largest finite 448, saturating stores) and, separately, from torch's casts called as a library.
# ---------------------------------------------------------------------------

def _f32(values):
    return np.asarray(values, dtype=np.float32)


def _same_bits(a, b):
    a = np.ascontiguousarray(np.asarray(a, np.float32))
    b = np.ascontiguousarray(np.asarray(b, np.float32))
    return np.array_equal(a.view(np.uint32), b.view(np.uint32))


def pin_bf16_hand_cases(Q):
    """Ties to even (both parities), just above a tie, carry into the exponent, subnormals, signed zero."""
    u = 2.0 ** -8  # half an ulp of bfloat16 at 1.0 (spacing 2^-7 in [1, 2))
    cases = [
        (1.0, 1.0),
        (1.0 + u, 1.0),                          # tie, lower neighbour 1.0 has an even last bit
        (1.0 + 3 * u, 1.0 + 4 * u),              # tie between 1+2^-7 (odd) and 1+2^-6 (even): up
        (1.0 + u + 2.0 ** -20, 1.0 + 2 * u),     # just above the tie: up
        (1.0 + u - 2.0 ** -20, 1.0),             # just below the tie: down
        (2.0 - u, 2.0),                          # tie between 2-2^-7 (all ones, odd) and 2: carry
        (2.0 - 2 * u, 2.0 - 2 * u),              # representable: unchanged
        (-(1.0 + u), -1.0),                      # symmetric in the sign
        (-(1.0 + 3 * u), -(1.0 + 4 * u)),
        (3 * 2.0 ** -134, 2.0 ** -132),          # subnormal tie (spacing 2^-133): to the even neighbour
        (2.0 ** -134, 0.0),                      # subnormal tie between 0 and 2^-133: to zero
        (5 * 2.0 ** -135, 2.0 ** -133),          # below the tie 1.25 * 2^-133: down
        (1.5 * 2.0 ** 100, 1.5 * 2.0 ** 100),
    ]
    x = _f32([c[0] for c in cases])
    want = _f32([c[1] for c in cases])
    got = Q.bf16_round(x)
    if not _same_bits(got, want):
        bad = [(float(a), float(g), float(w)) for a, g, w in zip(x, got, want) if float(g) != float(w)]
        return False, f"bf16_round hand cases differ: {bad[:4]}"
    z = Q.bf16_round(_f32([-0.0, 0.0]))
    if not (np.signbit(z[0]) and not np.signbit(z[1])):
        return False, "bf16_round loses the sign of zero"
    return True, ""


def pin_bf16_vs_torch(Q, n=200000, seed=1):
    """bf16_round equals torch's float32 -> bfloat16 cast (round to nearest even) on random bit patterns
    over the finite range and on values with 9 to 17 significant bits (dense in ties)."""
    import torch

    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    exp = (bits >> 23) & 0xFF
    x = bits[exp != 0xFF].view(np.float32)
    ties = (rng.integers(1 << 8, 1 << 17, size=n) * 2.0 ** rng.integers(-140, 100, size=n)).astype(np.float32)
    for arr in (x, ties, -ties):
        want = torch.from_numpy(arr.copy()).to(torch.bfloat16).float().numpy()
        if not _same_bits(Q.bf16_round(arr), want):
            return False, "bf16_round differs from torch's bfloat16 cast"
    return True, ""


def pin_bf16_split(Q, n=50000, seed=2):
    """hi = bf16(x), lo = bf16(x - hi) (difference in float32): checked against torch's casts, and
    |x - hi - lo| <= 2^-16 |x| (two 8-bit planes hold 16 significant bits) for normal x."""
    import torch

    rng = np.random.default_rng(seed)
    x = (rng.standard_normal(n) * 2.0 ** rng.integers(-30, 30, size=n)).astype(np.float32)
    hi, lo = Q.bf16_split(x)
    th = torch.from_numpy(x.copy()).to(torch.bfloat16)
    tl = (torch.from_numpy(x.copy()) - th.float()).to(torch.bfloat16)
    if not (_same_bits(hi, th.float().numpy()) and _same_bits(lo, tl.float().numpy())):
        return False, "bf16_split planes differ from torch's casts"
    err = np.abs(x.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64))
    if not (err <= 2.0 ** -16 * np.abs(x.astype(np.float64))).all():
        return False, f"hi + lo misses x by {float((err / np.abs(x)).max()):.3e} relative"
    # a value with exactly 16 significant bits is held exactly by the two planes
    y = _f32([1.0 + 2.0 ** -15, -(3.0 + 2.0 ** -14)])
    h, l = Q.bf16_split(y)
    if not np.array_equal(h.astype(np.float64) + l.astype(np.float64), y.astype(np.float64)):
        return False, "a 16-bit value is not held exactly by hi + lo"
    return True, ""


def pin_dequant_bf16(Q, seed=3):
    """dequant_bf16: real and imaginary parts through float32 then the planes, for 1 and 2 planes."""
    import torch

    rng = np.random.default_rng(seed)
    A = rng.standard_normal((5, 3, 7)) + 1j * rng.standard_normal((5, 3, 7))
    re = torch.from_numpy(A.real.astype(np.float32))
    im = torch.from_numpy(A.imag.astype(np.float32))
    one = re.to(torch.bfloat16).double().numpy() + 1j * im.to(torch.bfloat16).double().numpy()
    if not np.array_equal(Q.dequant_bf16(A, 1), one):
        return False, "dequant_bf16(planes=1) is not the bfloat16 cast of each part"
    rl = (re - re.to(torch.bfloat16).float()).to(torch.bfloat16).double()
    il = (im - im.to(torch.bfloat16).float()).to(torch.bfloat16).double()
    two = (re.to(torch.bfloat16).double() + rl).numpy() + 1j * (im.to(torch.bfloat16).double() + il).numpy()
    if not np.array_equal(Q.dequant_bf16(A, 2), two):
        return False, "dequant_bf16(planes=2) is not hi + lo of each part"
    return True, ""


def pin_e4m3_hand_cases(Q):
    """Subnormal grid 2^-9, ties to even on it and among normals, the 2^-6 boundary, saturation at 448."""
    s = 2.0 ** -9
    cases = [
        (0.0, 0.0),
        (s, s), (7 * s, 7 * s),                  # subnormals are exact multiples of 2^-9
        (0.5 * s, 0.0),                          # tie between 0 and 2^-9: to zero (even)
        (1.5 * s, 2 * s),                        # tie between 2^-9 (odd) and 2^-8 (even): up
        (2.5 * s, 2 * s),                        # tie between 2^-8 (even) and 3 * 2^-9: down
        (7.5 * s, 2.0 ** -6),                    # largest subnormal tie rounds into the normals
        (2.0 ** -6, 2.0 ** -6),                  # least normal
        (2.0 ** -6 + 0.5 * s, 2.0 ** -6),        # spacing stays 2^-9 in [2^-6, 2^-5): tie to even
        (2.0 ** -6 + 1.5 * s, 2.0 ** -6 + 2 * s),
        (1.0 + 2.0 ** -4, 1.0),                  # spacing 2^-3 in [1, 2): tie, down to the even 1.0
        (1.0 + 3 * 2.0 ** -4, 1.25),             # tie, up to the even 1.25
        (1.0 + 2.0 ** -4 + 2.0 ** -10, 1.125),   # above the tie
        (240.0, 240.0), (256.0, 256.0), (416.0, 416.0), (448.0, 448.0),
        (432.0, 448.0),                          # tie between 416 (odd last bit) and 448 (even): up
        (400.0, 384.0), (420.0, 416.0),          # spacing 32 in [256, 512): 400 is a tie to even 384
        (460.0, 448.0), (500.0, 448.0), (1e6, 448.0),  # saturating store
        (-1.5 * s, -2 * s), (-1e6, -448.0),
    ]
    x = np.asarray([c[0] for c in cases], np.float64)
    want = np.asarray([c[1] for c in cases], np.float64)
    got = Q.e4m3_round(x)
    if not np.array_equal(got, want):
        bad = [(a, g, w) for a, g, w in zip(x, got, want) if g != w]
        return False, f"e4m3_round hand cases differ: {bad[:4]}"
    return True, ""


def pin_e4m3_vs_torch(Q, n=200000, seed=4):
    """e4m3_round equals torch's float32 -> float8_e4m3fn cast below the saturation region
    (|x| < 464, where torch rounds to 448 too; above it torch gives NaN and the store saturates)."""
    import torch

    rng = np.random.default_rng(seed)
    x = (rng.uniform(-1, 1, size=n) * 2.0 ** rng.integers(-14, 9, size=n)).astype(np.float32)
    x = x[np.abs(x) < 464.0]
    grid = (np.arange(-3712, 3713) * 2.0 ** -13).astype(np.float32)  # every half-spacing tie up to 0.45
    for arr in (x, grid):
        want = torch.from_numpy(arr.copy()).to(torch.float8_e4m3fn).double().numpy()
        if not np.array_equal(Q.e4m3_round(arr.astype(np.float64)), want):
            return False, "e4m3_round differs from torch's float8_e4m3fn cast"
    return True, ""


def pin_e4m3_site_scale(Q, seed=5):
    """The site scale is a power of two 2^j with max|Re, Im| * 2^j in [224, 448] (the largest such j)."""
    rng = np.random.default_rng(seed)
    for m in (448.0, 1.0, 1.75, 0.3, 3e-5, 1000.0, 224.0, 223.9):
        A = rng.standard_normal((4, 2, 4)) + 1j * rng.standard_normal((4, 2, 4))
        A *= m / max(np.abs(A.real).max(), np.abs(A.imag).max())
        sc = Q.e4m3_site_scale(A)
        mx = float(max(np.abs(A.real.astype(np.float32)).max(), np.abs(A.imag.astype(np.float32)).max()))
        j = math.log2(sc)
        if j != round(j):
            return False, f"scale {sc} is not a power of two"
        if not 224.0 <= mx * sc <= 448.0:
            return False, f"max {mx} * scale {sc} = {mx * sc} outside [224, 448]"
    if Q.e4m3_site_scale(np.zeros((2, 2, 2), complex)) != 1.0:
        return False, "all-zero tensor must get scale 1"
    return True, ""


def pin_dequant_e4m3(Q, seed=6):
    """dequant_e4m3 = e4m3(x * scale) / scale per part; values already on the scaled grid survive exactly."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((6, 2, 5)) + 1j * rng.standard_normal((6, 2, 5))
    sc = Q.e4m3_site_scale(A)
    D = Q.dequant_e4m3(A)
    re = A.real.astype(np.float32).astype(np.float64)
    im = A.imag.astype(np.float32).astype(np.float64)
    if not np.array_equal(D, (Q.e4m3_round(re * sc) + 1j * Q.e4m3_round(im * sc)) / sc):
        return False, "dequant_e4m3 is not the scaled rounding"
    if not np.array_equal(Q.dequant_e4m3(D), D):
        return False, "dequant_e4m3 is not idempotent"
    rel = np.abs(D.real - re) / np.maximum(np.abs(re), 2.0 ** -6 / sc)
    if rel.max() > 2.0 ** -4 * (1 + 1e-12):
        return False, f"relative error {rel.max():.3e} above half a 3-bit ulp"
    return True, ""


def pin_fp16_hand_cases(Q):
    """binary16: spacing 2^-10 in [1, 2), ties to even of both parities, the subnormal grid 2^-24, the
    2^-14 boundary, the largest finite value."""
    cases = [
        (1.0, 1.0), (1.0 + 2.0 ** -11, 1.0), (1.0 + 3 * 2.0 ** -11, 1.0 + 2.0 ** -9),
        (1.0 + 2.0 ** -11 + 2.0 ** -20, 1.0 + 2.0 ** -10), (2.0 - 2.0 ** -11, 2.0),
        (2.0 ** -25, 0.0), (3 * 2.0 ** -25, 2.0 ** -23), (5 * 2.0 ** -26, 2.0 ** -24),
        (2.0 ** -14 + 2.0 ** -25, 2.0 ** -14), (2.0 ** -14 + 3 * 2.0 ** -25, 2.0 ** -14 + 2.0 ** -23),
        (65504.0, 65504.0), (65504.0 + 15.0, 65504.0), (-(1.0 + 3 * 2.0 ** -11), -(1.0 + 2.0 ** -9)),
        (32768.0 + 16.0, 32768.0), (32768.0 + 48.0, 32768.0 + 64.0),
    ]
    x = np.asarray([c[0] for c in cases], np.float32)
    want = np.asarray([c[1] for c in cases], np.float64)
    got = Q.fp16_round(x)
    if not np.array_equal(got, want):
        bad = [(float(a), g, w) for a, g, w in zip(x, got, want) if g != w]
        return False, f"fp16_round hand cases differ: {bad[:4]}"
    return True, ""


def pin_fp16_vs_torch(Q, n=200000, seed=7):
    """fp16_round equals torch's float32 -> float16 cast on random magnitudes over the whole finite range,
    subnormals included, and on every half-spacing tie of a dense grid."""
    import torch

    rng = np.random.default_rng(seed)
    x = (rng.standard_normal(n) * 2.0 ** rng.integers(-30, 16, size=n)).astype(np.float32)
    x = x[np.abs(x) < 65504.0]
    grid = (np.arange(-40000, 40001) * 2.0 ** -14).astype(np.float32)
    for arr in (x, grid):
        want = torch.from_numpy(arr.copy()).to(torch.float16).double().numpy()
        if not np.array_equal(Q.fp16_round(arr), want):
            return False, "fp16_round differs from torch's float16 cast"
    return True, ""


def pin_fp16_site_scale_and_dequant(Q, seed=8):
    """The FP16 site scale is the power of two putting max|Re, Im| in [16384, 32768]; dequant_fp16 is
    fp16(x * scale) / scale per part and is idempotent."""
    rng = np.random.default_rng(seed)
    for m in (1.0, 0.7, 3e-3, 32768.0, 16384.0, 20000.0):
        A = rng.standard_normal((4, 2, 4)) + 1j * rng.standard_normal((4, 2, 4))
        A *= m / max(np.abs(A.real).max(), np.abs(A.imag).max())
        sc = Q.fp16_site_scale(A)
        mx = float(max(np.abs(A.real.astype(np.float32)).max(), np.abs(A.imag.astype(np.float32)).max()))
        if math.log2(sc) != round(math.log2(sc)) or not 16384.0 <= mx * sc <= 32768.0:
            return False, f"scale {sc} for max {mx}"
        D = Q.dequant_fp16(A)
        re = A.real.astype(np.float32).astype(np.float64)
        if not np.array_equal(D.real, Q.fp16_round((re * sc).astype(np.float32)) / sc):
            return False, "dequant_fp16 is not the scaled rounding"
        if not np.array_equal(Q.dequant_fp16(D), D):
            return False, "dequant_fp16 is not idempotent"
        rel = np.abs(D.real - re) / np.abs(re)
        if rel[np.abs(re) * sc >= 2.0 ** -14].max() > 2.0 ** -11 * (1 + 1e-12):
            return False, "relative error above half an 11-bit ulp among normals"
    return True, ""


def pin_fp16_split(Q, n=100000, seed=9):
    """hi = fp16(x), lo = fp16(x - hi): checked against torch's casts; two 11-bit planes hold 22
    significant bits, |x - hi - lo| <= 2^-22 |x| wherever |x| >= 2^-3 (below, lo is subnormal and the
    error is at most 2^-25); values with 22 significant bits are held exactly."""
    import torch

    rng = np.random.default_rng(seed)
    x = (rng.standard_normal(n) * 2.0 ** rng.integers(-20, 15, size=n)).astype(np.float32)
    x = x[np.abs(x) <= 32768.0]
    hi, lo = Q.fp16_split(x)
    th = torch.from_numpy(x.copy()).to(torch.float16)
    tl = (torch.from_numpy(x.copy()) - th.float()).to(torch.float16)
    if not (np.array_equal(hi, th.double().numpy()) and np.array_equal(lo, tl.double().numpy())):
        return False, "fp16_split planes differ from torch's casts"
    a = np.abs(x.astype(np.float64))
    err = np.abs(x.astype(np.float64) - hi - lo)
    if not (err <= np.maximum(2.0 ** -22 * a, 2.0 ** -25)).all():
        return False, f"hi + lo misses x by {float(err.max()):.3e}"
    if not (err[a >= 0.125] <= 2.0 ** -22 * a[a >= 0.125]).all():
        return False, "relative error above 2^-22 among |x| >= 2^-3"
    y = _f32([1000.0 + 2.0 ** -12, -(3.0 + 2.0 ** -18), 1.0 + 2.0 ** -21, 20000.0 + 2.0 ** -6])
    h, l = Q.fp16_split(y)
    if not np.array_equal(h + l, y.astype(np.float64)):
        return False, "a 22-bit value is not held exactly by hi + lo"
    if not np.array_equal(h, _f32([1000.0, -3.0, 1.0, 20000.0]).astype(np.float64)):
        return False, "hi is not the nearest binary16 value"
    return True, ""


def pin_dequant_fp16_two_planes(Q, seed=10):
    """dequant_fp16(A, 2) is (hi + lo) / scale of each scaled part at the one-plane scale, within
    2^-22 relative of the float32 parts (entries not tiny against the scale), and is idempotent."""
    rng = np.random.default_rng(seed)
    for m in (1.0, 0.37, 5e-4):
        A = rng.standard_normal((6, 3, 5)) + 1j * rng.standard_normal((6, 3, 5))
        A *= m / max(np.abs(A.real).max(), np.abs(A.imag).max())
        sc = Q.fp16_site_scale(A)
        D = Q.dequant_fp16(A, 2)
        for part, dpart in ((A.real, D.real), (A.imag, D.imag)):
            xs = (part.astype(np.float32) * np.float32(sc)).astype(np.float32)
            hi = Q.fp16_round(xs)
            lo = Q.fp16_round((xs.astype(np.float64) - hi).astype(np.float32))
            if not np.array_equal(dpart, (hi + lo) / sc):
                return False, "dequant_fp16(A, 2) is not the two-plane value"
            ref = part.astype(np.float32).astype(np.float64)
            big = np.abs(ref) * sc >= 0.125
            if (np.abs(dpart - ref)[big] > 2.0 ** -22 * np.abs(ref)[big]).any():
                return False, "two planes do not hold 22 bits"
        if not np.array_equal(Q.dequant_fp16(D, 2), D):
            return False, "dequant_fp16(., 2) is not idempotent"
        if np.array_equal(Q.dequant_fp16(A, 1), D):
            return False, "the second plane adds nothing"
    return True, ""


QUANT_PINS = [pin_bf16_hand_cases, pin_bf16_vs_torch, pin_bf16_split, pin_dequant_bf16, pin_e4m3_hand_cases,
              pin_e4m3_vs_torch, pin_e4m3_site_scale, pin_dequant_e4m3, pin_fp16_hand_cases, pin_fp16_vs_torch,
              pin_fp16_site_scale_and_dequant, pin_fp16_split, pin_dequant_fp16_two_planes]
