"""Dynamic bond dimensions (Sec. 3.4.2) -- TEST INFRASTRUCTURE.

Plain restatement of the bond-dimension filter, used to check the library's
``fastmps_bond_filter`` (integer results, compared exactly) and to truncate
chains for the parity tests.  It shares no code with the library.

Reading of the paper.  A fixed-chi filter keeps the chi largest Schmidt
coefficients at every bond; its truncation error comes almost entirely from
the central bonds, where the spectra decay slowest (area law).  The modified
filter keeps, at every bond, only as many coefficients as needed to stay
within the largest error the fixed-chi filter already makes anywhere on the
chain -- fewer at the edges, the same at the centre -- so the maximum
truncation error over all bonds is unchanged.

Definitions (both sides take the integer decisions in FP64 with the same
summation order):

* discarded weight of keeping c of the n coefficients of a bond:
  eps(c) = T_c / T_0 with T_c = sum_{j=c}^{n-1} Lambda_j^2, summed from j = n-1
  down to j = c;
* budget eps* = max over bonds of eps(min(chi, n)), or a given eps > 0;
* kept count chi_b = the least c in [1, min(chi, n)] with eps(c) <= eps*
  (min(chi, n) if there is none);
* alignment (optional, align > 1): chi_b is rounded up to a multiple of align,
  capped at min(chi, n) -- keeping more coefficients only lowers the discarded
  weight, and tile-aligned bonds waste no tensor-core work on padding;
* isometry shapes: a left-to-right sweep raises chi_b to ceil(chi_{b-1} / d)
  (chi_0 = 1) so that d * chi_r >= chi_l holds at every site.
"""
from __future__ import annotations

import math


def tail_weights(lam):
    """[T_0, T_1, ..., T_n] with T_c = sum_{j >= c} lam_j^2, accumulated from the last index."""
    n = len(lam)
    T = [0.0] * (n + 1)
    acc = 0.0
    for j in range(n - 1, -1, -1):
        acc += float(lam[j]) * float(lam[j])
        T[j] = acc
    return T


def discarded_weight(lam, c: int) -> float:
    T = tail_weights(lam)
    return T[c] / T[0]


def filter_bonds(lams, d: int, chi: int, eps: float | None = None, align: int = 1):
    """lams[k]: Schmidt coefficients right of site k (k = 0..M-1; the last is ignored).

    Returns (bonds[M+1], discarded[M+1], eps_star)."""
    M = len(lams)
    tails = [tail_weights(lams[k]) for k in range(M - 1)]
    caps = [min(chi, len(lams[k])) for k in range(M - 1)]
    if eps is None or eps <= 0:
        eps_star = 0.0
        for k in range(M - 1):
            e = tails[k][caps[k]] / tails[k][0]
            if e > eps_star:
                eps_star = e
    else:
        eps_star = float(eps)
    bonds = [1] * (M + 1)
    for k in range(M - 1):
        T = tails[k]
        keep = caps[k]
        for c in range(1, caps[k] + 1):
            if T[c] / T[0] <= eps_star:
                keep = c
                break
        if align > 1:
            keep = min(-(-keep // align) * align, caps[k])
        bonds[k + 1] = keep
    for k in range(M - 1):
        need = -(-bonds[k] // d)          # ceil(bonds[k] / d)
        bonds[k + 1] = min(max(bonds[k + 1], need), caps[k])
    disc = [0.0] * (M + 1)
    for k in range(M - 1):
        disc[k + 1] = tails[k][bonds[k + 1]] / tails[k][0]
    return bonds, disc, eps_star


def truncate_vidal(gammas, lams, bonds):
    """Leading blocks Gamma_k[:b_k, :, :b_{k+1}] and Lambda_k[:b_{k+1}] of a Vidal chain."""
    G = [g[: bonds[k], :, : bonds[k + 1]].copy() for k, g in enumerate(gammas)]
    L = [l[: bonds[k + 1]].copy() for k, l in enumerate(lams)]
    return G, L
