"""Plant plausible mistakes in copies of the oracle (on the CPU) and require that a pin catches each.

This guards the pins themselves: an oracle with a dropped term, a wrong sign,
a transposed index, a missing normalisation or a mis-keyed uniform must fail
at least one of them.
"""
import os

import pytest

import oracle
import oracle_pins as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "drop_imag_cross_term": ("yr[c] += vr * ar[c] - vi * ai[c];", "yr[c] += vr * ar[c];"),
    "imag_sign_flip": ("yi[c] += vr * ai[c] + vi * ar[c];", "yi[c] += vr * ai[c] - vi * ar[c];"),
    "transposed_site_index": ("const size_t row = (size_t)2 * ((size_t)a * cols + c0);",
                              "const size_t row = (size_t)2 * ((size_t)a * (cols == chi_l ? cols : chi_r) + c0);"),
    "no_cumulative_sum": ("        acc += w[s];\n        C[s] = acc;", "        acc += w[s];\n        C[s] = w[s];"),
    "threshold_not_scaled_by_Z": ("const double t = u * Z;", "const double t = u;"),
    "logprob_without_Z": ("lps[j] += log(w[s]) - log(Z);", "lps[j] += log(w[s]);"),
    "no_renormalisation": ("const double inv = 1.0 / sqrt(w[s]);", "const double inv = 1.0;"),
    "uniform_wrong_site_key": ("orc_uniform(seed, n, (uint32_t)k, job)", "orc_uniform(seed, n, (uint32_t)(k + 1), job)"),
    "philox_wrong_multiplier": ("#define ORC_PHILOX_M1 0xCD9E8D57u", "#define ORC_PHILOX_M1 0xCD9E8D59u"),
    "uniform_drops_second_word": ("| (uint64_t)(x[1] >> 11);", "| 0u;"),
    "select_previous_block": ("v[2 * b] = y[2 * (s * cr + b)] * inv;",
                              "v[2 * b] = y[2 * (((s + 1) % d) * cr + b)] * inv;"),
    "vidal_lambda_not_squared": ("acc += (re * re + im * im) * lam[b] * lam[b];",
                                 "acc += (re * re + im * im) * lam[b];"),
    "vidal_carry_without_lambda": ("v[2 * b] *= lam[k][b];\n                            v[2 * b + 1] *= lam[k][b];",
                                   "v[2 * b] *= 1.0;\n                            v[2 * b + 1] *= 1.0;"),
    "displacement_transposed": ("const double dr = D[2 * (s * d + t)], di = D[2 * (s * d + t) + 1];",
                                "const double dr = D[2 * (t * d + s)], di = D[2 * (t * d + s) + 1];"),
    "zassenhaus_lowering_sign": ("Y[(j - 1) * n + j] = -conj(mu) * r;", "Y[(j - 1) * n + j] = conj(mu) * r;"),
    "zassenhaus_missing_conjugate": ("Y[(j - 1) * n + j] = -conj(mu) * r;", "Y[(j - 1) * n + j] = -mu * r;"),
    "zassenhaus_factor_order": ("orc_cmatmul(n, EX, EY, P);", "orc_cmatmul(n, EY, EX, P);"),
    "zassenhaus_no_gaussian_factor": ("const double g = exp(-0.5 * (mu_re * mu_re + mu_im * mu_im));",
                                      "const double g = 1.0;"),
    "displacement_on_wrong_site": ("const double *m = mu + 2 * ((size_t)k * ldmu + (size_t)i);",
                                   "const double *m = mu + 2 * ((size_t)((k + 1) % M) * ldmu + (size_t)i);"),
    "born_conjugates_one_factor": ("im += r[2 * a] * e[1] + r[2 * a + 1] * e[0];\n            }\n            t[2 * b] = re;",
                                   "im += -r[2 * a] * e[1] + r[2 * a + 1] * e[0];\n            }\n            t[2 * b] = re;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    find, repl = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(find) == 1, f"mutation site for {name} not unique/absent"
    lib = oracle.load_variant(oracle.build_variant(src.replace(find, repl), str(tmp_path / f"{name}.so")))
    failures = []
    for pin in P.FAST_PINS:
        try:
            ok, detail = pin(lib=lib)
        except Exception as e:  # a crash or a raised error also counts as caught
            ok, detail = False, repr(e)
        if not ok:
            failures.append(pin.__name__)
    assert failures, f"mutant {name} passed every pin"


# ---------------------------------------------------------------------------
# the bond-dimension filter's restatement (oracle/bond_filter.py)
# ---------------------------------------------------------------------------
BF_SRC = os.path.join(os.path.dirname(oracle.__file__), "bond_filter.py")

BF_MUTANTS = {
    "tail_sum_from_the_front": ("    for j in range(n - 1, -1, -1):", "    for j in range(0, n):"),
    "kept_count_off_by_one": ("                keep = c\n", "                keep = c - 1 if c > 1 else c\n"),
    "strict_budget_comparison": ("            if T[c] / T[0] <= eps_star:", "            if T[c] / T[0] < eps_star * 0.5:"),
    "budget_from_first_bond_only": ("            if e > eps_star:\n                eps_star = e", "            if k == 0:\n                eps_star = e"),
    "alignment_rounds_down": ("            keep = min(-(-keep // align) * align, caps[k])",
                              "            keep = max(1, min(keep // align * align, caps[k]))"),
    "no_isometry_sweep": ("        bonds[k + 1] = min(max(bonds[k + 1], need), caps[k])", "        pass"),
    "discarded_not_normalised": ("        disc[k + 1] = tails[k][bonds[k + 1]] / tails[k][0]",
                                 "        disc[k + 1] = tails[k][bonds[k + 1]]"),
}


@pytest.mark.parametrize("name", sorted(BF_MUTANTS))
def test_bond_filter_mutant_is_caught(name):
    import types

    find, repl = BF_MUTANTS[name]
    src = open(BF_SRC).read()
    assert src.count(find) == 1, f"mutation site for {name} not unique/absent"
    mod = types.ModuleType(f"bf_mutant_{name}")
    exec(compile(src.replace(find, repl), f"<mutant {name}>", "exec"), mod.__dict__)
    failures = []
    for pin in P.BOND_FILTER_PINS:
        try:
            ok, detail = pin(mod)
        except Exception as e:  # a crash also counts as caught
            ok, detail = False, repr(e)
        if not ok:
            failures.append(pin.__name__)
    assert failures, f"mutant {name} passed every pin"


# ---------------------------------------------------------------------------
# the low-precision storage formats (oracle/quant.py)
# ---------------------------------------------------------------------------
Q_SRC = os.path.join(os.path.dirname(oracle.__file__), "quant.py")

QUANT_MUTANTS = {
    "bf16_truncates": ("    u = (u + 0x7FFF + lsb) & 0xFFFF0000", "    u = u & 0xFFFF0000"),
    "bf16_ties_away_from_zero": ("    u = (u + 0x7FFF + lsb) & 0xFFFF0000", "    u = (u + 0x8000) & 0xFFFF0000"),
    "bf16_ties_to_odd": ("    u = (u + 0x7FFF + lsb) & 0xFFFF0000", "    u = (u + 0x8000 - lsb) & 0xFFFF0000"),
    "bf16_lo_plane_unrounded": ("    lo = bf16_round((x - hi).astype(np.float32))", "    lo = (x - hi).astype(np.float32)"),
    "bf16_lo_from_x": ("    lo = bf16_round((x - hi).astype(np.float32))", "    lo = bf16_round(x) * 0"),
    "dequant_drops_lo_plane": ("    return (rh.astype(np.float64) + rl.astype(np.float64)) + 1j",
                               "    return (rh.astype(np.float64) + 0.0 * rl.astype(np.float64)) + 1j"),
    "dequant_imag_from_real": ("    return bf16_round(re).astype(np.float64) + 1j * bf16_round(im).astype(np.float64)",
                               "    return bf16_round(re).astype(np.float64) + 1j * bf16_round(re).astype(np.float64)"),
    "e4m3_no_saturation": ("    r = np.minimum(r, E4M3_MAX)", "    r = r"),
    "e4m3_subnormal_floor_off_by_one": ("    e = np.maximum(ex - 1, -6)", "    e = np.maximum(ex - 1, -7)"),
    "e4m3_four_mantissa_bits": ("    q = np.ldexp(1.0, (e - 3).astype(np.int64))", "    q = np.ldexp(1.0, (e - 4).astype(np.int64))"),
    "e4m3_ties_away_from_zero": ("    r = np.round(a / q) * q                  # numpy rounds halves to even",
                                 "    r = np.floor(a / q + 0.5) * q"),
    "e4m3_truncates": ("    r = np.round(a / q) * q                  # numpy rounds halves to even",
                       "    r = np.floor(a / q) * q"),
    "e4m3_scale_ceil": ("    return float(2.0 ** np.floor(np.log2(E4M3_MAX / m)))",
                        "    return float(2.0 ** np.ceil(np.log2(E4M3_MAX / m)))"),
    "e4m3_scale_one_too_small": ("    return float(2.0 ** np.floor(np.log2(E4M3_MAX / m)))",
                                 "    return float(2.0 ** (np.floor(np.log2(E4M3_MAX / m)) - 1))"),
    "dequant_e4m3_not_unscaled": ("    return (e4m3_round(re * s) + 1j * e4m3_round(im * s)) / s",
                                  "    return (e4m3_round(re * s) + 1j * e4m3_round(im * s))"),
    "fp16_ten_mantissa_bits": ("    q = np.ldexp(1.0, (e - 10).astype(np.int64))", "    q = np.ldexp(1.0, (e - 9).astype(np.int64))"),
    "fp16_subnormal_floor": ("    e = np.maximum(ex - 1, -14)", "    e = np.maximum(ex - 1, -15)"),
    "fp16_ties_away": ("    r = np.round(a / q) * q                  # a / q is exact",
                       "    r = np.floor(a / q + 0.5) * q            # a / q is exact"),
    "fp16_scale_too_large": ("    return float(2.0 ** np.floor(np.log2(FP16_TOP / m)))",
                             "    return float(2.0 ** np.ceil(np.log2(FP16_TOP / m)))"),
    "dequant_fp16_imag_unscaled": ("    im = np.asarray(A.imag, dtype=np.float32) * np.float32(s)",
                                   "    im = np.asarray(A.imag, dtype=np.float32)"),
    "fp16_lo_plane_unrounded": ("    lo = fp16_round((x.astype(np.float64) - hi).astype(np.float32))",
                                "    lo = (x.astype(np.float64) - hi).astype(np.float32).astype(np.float64)"),
    "fp16_lo_plane_dropped": ("    lo = fp16_round((x.astype(np.float64) - hi).astype(np.float32))",
                              "    lo = hi * 0"),
    "fp16_lo_as_bf16": ("    lo = fp16_round((x.astype(np.float64) - hi).astype(np.float32))",
                        "    lo = bf16_round((x.astype(np.float64) - hi).astype(np.float32)).astype(np.float64)"),
    "dequant_fp16_two_planes_lo_sign": ("    return ((rh + rl) + 1j * (ih + il)) / s",
                                        "    return ((rh + rl) + 1j * (ih - il)) / s"),
}


@pytest.mark.parametrize("name", sorted(QUANT_MUTANTS))
def test_quant_mutant_is_caught(name):
    import types

    find, repl = QUANT_MUTANTS[name]
    src = open(Q_SRC).read()
    assert src.count(find) == 1, f"mutation site for {name} not unique/absent"
    mod = types.ModuleType(f"quant_mutant_{name}")
    exec(compile(src.replace(find, repl), f"<mutant {name}>", "exec"), mod.__dict__)
    failures = []
    for pin in P.QUANT_PINS:
        try:
            ok, detail = pin(mod)
        except Exception as e:  # a crash also counts as caught
            ok, detail = False, repr(e)
        if not ok:
            failures.append(pin.__name__)
    assert failures, f"mutant {name} passed every pin"
