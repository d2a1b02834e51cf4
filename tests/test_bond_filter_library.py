"""The library's dynamic bond-dimension filter (host code, no GPU) against the oracle's restatement.

Integer results (the kept counts) must be identical, and the discarded weights
bitwise equal: both sides take every decision in FP64 with the same summation
order.
"""
import numpy as np
import pytest

import gen
from oracle import bond_filter as BF


@pytest.fixture(scope="module")
def F():
    import paper_2512_20064_gb300 as F

    F.load_library()
    return F


@pytest.mark.parametrize("M,d,chi_gen,chi,eps,align", [(40, 3, 64, 24, 0.0, 1), (40, 3, 64, 64, 1e-4, 1),
                                                        (30, 4, 48, 8, 0.0, 1), (25, 2, 32, 32, 0.0, 1),
                                                        (60, 3, 27, 20, 1e-6, 1), (3, 5, 5, 2, 0.0, 1),
                                                        (40, 3, 64, 48, 0.0, 16), (30, 4, 48, 40, 1e-5, 8)])
def test_filter_matches_oracle(F, M, d, chi_gen, chi, eps, align):
    b, G, L = gen.area_law_vidal_chain(M, d, chi_gen, seed=M + d)
    got, disc = F.fastmps_bond_filter(b, L, d, chi, eps, align)
    want, wdisc, es = BF.filter_bonds(L, d, chi, eps, align)
    assert got == want
    assert np.array_equal(disc, np.asarray(wdisc))
    for k in range(M):
        assert got[k] <= d * got[k + 1]


def test_filter_random_spectra(F):
    """Unsorted and degenerate spectra, a single site, and a budget no bond can meet."""
    rng = np.random.Generator(np.random.PCG64(8))
    for trial in range(40):
        M = int(rng.integers(1, 12))
        d = int(rng.integers(2, 5))
        b = [1] + [int(rng.integers(1, 30)) for _ in range(M - 1)] + [1]
        L = [rng.random(b[k + 1]) ** 3 for k in range(M - 1)] + [np.ones(1)]
        if trial % 5 == 0 and M > 1:
            L[0] = np.ones(b[1])                        # flat spectrum
        chi = int(rng.integers(1, 35))
        eps = [0.0, 1e-9, 1e-3, 0.3][trial % 4]
        align = [1, 4, 7, 32][(trial // 4) % 4]
        got, disc = F.fastmps_bond_filter(b, L, d, chi, eps, align)
        want, wdisc, _ = BF.filter_bonds(L, d, chi, eps, align)
        assert got == want, (trial, got, want)
        assert np.array_equal(disc, np.asarray(wdisc))


def test_filter_rejects_bad_input(F):
    with pytest.raises(F.FastMPSError) as e:
        F.fastmps_bond_filter([2, 3, 1], [np.ones(3), np.ones(1)], 3, 4)
    assert e.value.code == -2
    with pytest.raises(F.FastMPSError) as e:
        F.fastmps_bond_filter([1, 3, 1], [np.zeros(3), np.ones(1)], 3, 4)
    assert e.value.code == -1


def test_filter_isometry_raise(F):
    """The library raises a count for the isometry shape exactly as the oracle does."""
    b = [1, 4, 8, 1]
    L = [np.full(4, 0.5), np.array([1.0] + [1e-9] * 7), np.ones(1)]
    got, _ = F.fastmps_bond_filter(b, L, 2, 8, 1e-12)
    want, _, _ = BF.filter_bonds(L, 2, 8, 1e-12)
    assert got == want == [1, 4, 2, 1]
