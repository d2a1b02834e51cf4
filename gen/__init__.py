"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no sampling arithmetic.  It only makes the inputs the
sampler consumes: bond-dimension profiles and right-canonical complex site
tensors (Haar-random isometries), plus the workload recipes that stand in for
the paper's Gaussian-boson-sampling MPS data, which is not available here.

Conventions
-----------
* Site ``k`` holds ``A_k[chi_l, d, chi_r]`` with ``chi_l = b_k`` and
  ``chi_r = b_{k+1}``; ``b_0 = b_M = 1``.
* Right-canonical: ``sum_s A_k[:, s, :] A_k[:, s, :]^dagger = I_{chi_l}``.
  The tensor is the reshaped ``Q`` factor of a QR decomposition of a seeded
  complex Gaussian ``(d*chi_r) x chi_l`` matrix,
  ``A[a, s, b] = Q[s*chi_r + b, a]``, with the phases of ``diag(R)`` moved
  into ``Q`` so that ``diag(R) > 0`` (the Haar-measure convention).
* Skew: before the QR, the Gaussian rows of physical index ``s`` are scaled
  by ``exp(-s / skew)``, so low outcomes dominate, as photon-number
  distributions do in Gaussian boson sampling (Sec. 2.1, Sec. 4.2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "bond_dims",
    "isometry",
    "mps_tensors",
    "product_state",
    "ghz_chain",
    "Workload",
    "WORKLOADS",
    "batch_jobs",
    "vidal_form",
    "gbs_amplitudes",
    "decaying_vidal_chain",
    "area_law_vidal_chain",
]


def bond_dims(M: int, d: int, chi: int) -> list[int]:
    """Bond profile ``b_k = min(d^k, d^(M-k), chi)`` for ``k = 0..M``.

    The cap at the chain ends is the exact bond dimension an open chain of
    ``M`` sites can carry (Sec. 2.2: the bond dimension bounded by the
    Hilbert-space size of either side).
    """
    if M < 1 or d < 2 or chi < 1:
        raise ValueError("need M >= 1, d >= 2, chi >= 1")
    out = []
    for k in range(M + 1):
        left = 1
        for _ in range(k):
            left = min(left * d, chi)
        right = 1
        for _ in range(M - k):
            right = min(right * d, chi)
        out.append(min(left, right, chi))
    return out


def _gaussian(seed: int, rows: int, cols: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    g = rng.standard_normal((rows, cols, 2))
    return (g[..., 0] + 1j * g[..., 1]) / math.sqrt(2.0)


def _haar_from_gaussian(g, chi_l: int, d: int, chi_r: int, skew: float | None):
    """QR of the (optionally skewed) Gaussian, reshaped to ``A[chi_l, d, chi_r]``.

    Works for numpy arrays and torch tensors (CPU or CUDA) alike.
    """
    is_np = isinstance(g, np.ndarray)
    if skew:
        w = np.exp(-np.arange(d) / float(skew)).repeat(chi_r)
        if is_np:
            g = g * w[:, None]
        else:
            import torch

            g = g * torch.as_tensor(w, dtype=g.real.dtype, device=g.device)[:, None]
    if is_np:
        q, r = np.linalg.qr(g, mode="reduced")
        dg = np.diagonal(r)
        ph = dg / np.abs(dg)
        q = q * ph[None, :]
        # A[a, s, b] = Q[s*chi_r + b, a]
        return np.ascontiguousarray(q.T.reshape(chi_l, d, chi_r))
    import torch

    q, r = torch.linalg.qr(g, mode="reduced")
    dg = torch.diagonal(r)
    ph = dg / dg.abs()
    q = q * ph[None, :]
    return q.transpose(0, 1).reshape(chi_l, d, chi_r).contiguous()


def isometry(seed: int, chi_l: int, d: int, chi_r: int, skew: float | None = None,
             dtype=np.complex128, device: str | None = None):
    """One right-canonical site tensor ``A[chi_l, d, chi_r]`` (complex).

    ``device=None`` returns a numpy array (complex128 arithmetic, then cast to
    ``dtype``).  ``device='cuda'`` (or any torch device string) draws the
    Gaussian with a seeded torch generator on that device and returns a torch
    complex64 tensor there; that route exists for the large workloads whose
    QR would take minutes on the host.
    """
    if d * chi_r < chi_l:
        raise ValueError("an isometry needs d*chi_r >= chi_l")
    if device is None:
        g = _gaussian(seed, d * chi_r, chi_l)
        return _haar_from_gaussian(g, chi_l, d, chi_r, skew).astype(dtype, copy=False)
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    re = torch.randn((d * chi_r, chi_l), generator=gen, device=device, dtype=torch.float32)
    im = torch.randn((d * chi_r, chi_l), generator=gen, device=device, dtype=torch.float32)
    g = torch.complex(re, im) * (1.0 / math.sqrt(2.0))
    return _haar_from_gaussian(g, chi_l, d, chi_r, skew)


def mps_tensors(M: int, d: int, chi: int, base_seed: int = 1234, skew: float | None = None,
                pool: int | None = None, dtype=np.complex128, device: str | None = None,
                bonds: list[int] | None = None):
    """Site tensors of a random right-canonical MPS.

    Site ``k`` is drawn from seed ``base_seed + k``.  With ``pool=P``, every
    interior site (``b_k = b_{k+1} = chi``) reuses ``pool[k mod P]`` whose
    seed is ``base_seed + 1_000_000 + (k mod P)``; end sites keep their own
    seed.  Returns ``(bond_dims, tensors, site_to_tensor)``, where
    ``site_to_tensor[k]`` indexes ``tensors`` (identity without a pool).
    """
    b = list(bonds) if bonds is not None else bond_dims(M, d, chi)
    tensors = []
    index = []
    pool_slot: dict[int, int] = {}
    for k in range(M):
        cl, cr = b[k], b[k + 1]
        if pool and cl == chi and cr == chi:
            j = k % pool
            if j not in pool_slot:
                pool_slot[j] = len(tensors)
                tensors.append(isometry(base_seed + 1_000_000 + j, cl, d, cr, skew, dtype, device))
            index.append(pool_slot[j])
        else:
            index.append(len(tensors))
            tensors.append(isometry(base_seed + k, cl, d, cr, skew, dtype, device))
    return b, tensors, index


def product_state(M: int, probs: np.ndarray, phases_seed: int = 7) -> tuple[list[int], list[np.ndarray]]:
    """A bond-dimension-1 MPS whose site ``k`` has outcome law ``probs[k]``.

    ``A_k[0, s, 0] = sqrt(probs[k, s]) * exp(i phi)``: right-canonical because
    ``sum_s |A_k[0, s, 0]|^2 = 1``.  Its outcomes are independent categorical
    draws, the textbook special case of MPS sampling.
    """
    probs = np.asarray(probs, dtype=np.float64)
    M2, d = probs.shape
    assert M2 == M
    rng = np.random.Generator(np.random.PCG64(phases_seed))
    out = []
    for k in range(M):
        ph = np.exp(2j * np.pi * rng.random(d))
        out.append((np.sqrt(probs[k]) * ph).reshape(1, d, 1).astype(np.complex128))
    return [1] * (M + 1), out


def ghz_chain(M: int, d: int) -> tuple[list[int], list[np.ndarray]]:
    """The GHZ state ``(|00..0> + |11..1> + ... + |d-1..d-1>)/sqrt(d)`` as an MPS.

    Right-canonical form with bonds ``1, d, d, ..., d, 1``:
    ``A_0[0, s, s] = 1/sqrt(d)``, ``A_k[s, s, s] = 1`` for interior ``k`` and
    ``A_{M-1}[s, s, 0] = 1``.  Every sample has all outcomes equal and
    ``P(s, s, ..., s) = 1/d``.
    """
    assert M >= 2
    b = [1] + [d] * (M - 1) + [1]
    ts = []
    a0 = np.zeros((1, d, d), np.complex128)
    for s in range(d):
        a0[0, s, s] = 1.0 / math.sqrt(d)
    ts.append(a0)
    for _ in range(1, M - 1):
        a = np.zeros((d, d, d), np.complex128)
        for s in range(d):
            a[s, s, s] = 1.0
        ts.append(a)
    al = np.zeros((d, d, 1), np.complex128)
    for s in range(d):
        al[s, s, 0] = 1.0
    ts.append(al)
    return b, ts


# ---------------------------------------------------------------------------
# Workload recipes: synthetic stand-ins for the paper's GBS MPS data
# (Sec. 4.2, Tables 1-3: d = 3..4, chi up to 10^4, M up to 8176).
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class Workload:
    name: str
    M: int
    d: int
    chi: int
    N: int
    skew: float | None
    pool: int | None = None
    base_seed: int = 1234
    sampler_seed: int = 42
    note: str = ""
    extra: dict = field(default_factory=dict)

    def bonds(self) -> list[int]:
        return bond_dims(self.M, self.d, self.chi)

    def flops_per_sample(self) -> float:
        """Algorithmic real flops of the complex contraction per sample (all sites)."""
        b = self.bonds()
        return float(sum(8 * b[k] * self.d * b[k + 1] for k in range(self.M)))


WORKLOADS = {
    "tiny": Workload("tiny", M=12, d=3, chi=16, N=10_000, skew=None,
                     note="M=12 d=3 chi<=16 unskewed Haar, N=1e4; brute force over 3^12"),
    "plain": Workload("plain", M=256, d=4, chi=256, N=1 << 17, skew=1.5,
                      note="M=256 d=4 chi=256 skew exp(-s/1.5), N=2^17, complex64 resident"),
    "precision": Workload("precision", M=1024, d=4, chi=1024, N=1 << 20, skew=1.5,
                          note="M=1024 d=4 chi=1024 skew exp(-s/1.5), N=2^20, 16-bit split operands"),
    "streaming": Workload("streaming", M=2048, d=3, chi=10_000, N=1 << 16, skew=1.5, pool=16,
                          note="M=2048 d=3 chi=1e4, pool of 16 interior isometries, host-streamed BF16, N=2^16"),
}


def batch_jobs(count: int = 64, seed: int = 2025, rows_cap: int | None = None):
    """Job parameters of the batching workload: ``count`` independent MPS with M ~ U[64, 2048],
    d in {2, 3, 4, 6}, chi log-uniform in [32, 2048] (bond profile capped at the chain ends as in
    ``bond_dims``), N log-uniform in [10^3, 10^6]; ``rows_cap`` bounds the rows drawn per job.
    Returns a list of dicts (M, d, chi, N, N_full, base_seed, sampler_seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    jobs = []
    for j in range(count):
        M = int(rng.integers(64, 2049))
        d = int(rng.choice([2, 3, 4, 6]))
        chi = int(round(math.exp(rng.uniform(math.log(32), math.log(2048)))))
        N = int(round(math.exp(rng.uniform(math.log(1e3), math.log(1e6)))))
        jobs.append({"M": M, "d": d, "chi": chi, "N_full": N, "N": min(N, rows_cap) if rows_cap else N,
                     "base_seed": 10_000 * (j + 1), "sampler_seed": 7 + j})
    return jobs


# ---------------------------------------------------------------------------
# Vidal form and GBS displacement amplitudes (inputs of the Vidal-form and
# displaced sampling entry points)
# ---------------------------------------------------------------------------

def vidal_form(bonds, tensors):
    """Vidal form ``(Gammas, Lambdas)`` of the state held by right-canonical ``tensors``.

    A left-to-right sweep of singular value decompositions (FP64): with
    ``R_0 = [[1]]``, the matrix ``(R_k A_k)`` reshaped to ``(chi_l d) x chi_r`` is
    ``U S V^dagger``; ``U`` is the left-canonical tensor ``L_k``, ``Lambda_k = S``
    (Schmidt coefficients of the cut right of site k, descending) and
    ``R_{k+1} = S V^dagger``.  Then ``Gamma_k = Lambda_{k-1}^{-1} L_k`` (``Lambda_{-1} = [1]``),
    so that ``Gamma_0 Lambda_0 Gamma_1 Lambda_1 ... Gamma_{M-1} Lambda_{M-1}`` is the
    same state and ``Gamma_k Lambda_k`` is right-canonical.  The bond dimensions
    are kept (the profile ``bond_dims`` never exceeds the rank of a cut).
    """
    M = len(bonds) - 1
    R = np.ones((1, 1), np.complex128)
    lam_prev = np.ones(1)
    gammas, lams = [], []
    for k in range(M):
        A = np.asarray(tensors[k], np.complex128)
        cl, d, cr = A.shape
        T = np.einsum("xa,asb->xsb", R, A).reshape(cl * d, cr)
        U, S, Vh = np.linalg.svd(T, full_matrices=False)
        if S.shape[0] != cr:
            raise ValueError(f"cut {k + 1} has rank {S.shape[0]} < bond {cr}")
        # fix the gauge of each singular pair: largest entry of V^dagger's row real positive
        j = np.argmax(np.abs(Vh), axis=1)
        ph = Vh[np.arange(cr), j] / np.abs(Vh[np.arange(cr), j])
        U = U * ph[None, :]
        Vh = Vh * ph.conj()[:, None]
        L = U.reshape(cl, d, cr)
        gammas.append(L / lam_prev[:, None, None])
        lams.append(S.copy())
        R = S[:, None] * Vh
        lam_prev = S
    return gammas, lams


def gbs_amplitudes(M: int, N: int, sigma: float = 0.3, seed: int = 4242, dtype=np.complex64) -> np.ndarray:
    """Random displacement amplitudes ``mu[k, n]`` for M sites and N samples.

    Stand-in for the classical noise of a lossy Gaussian boson sampler: the
    thermal part of the state is a random displacement with a complex Gaussian
    amplitude per mode and sample.  Here each amplitude is drawn i.i.d.,
    ``Re mu, Im mu ~ N(0, sigma^2 / 2)`` (so ``E|mu|^2 = sigma^2``).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    mu = (rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N))) * (sigma / math.sqrt(2.0))
    return mu.astype(dtype)


def decaying_vidal_chain(M: int, d: int, chi: int, decay: float = 0.35, seed: int = 99):
    """A Vidal-form chain whose Schmidt spectra decay like ``exp(-decay * j)``, bond by bond.

    Built from a right-canonical chain by re-weighting: ``Lambda_k`` is the
    normalised spectrum ``exp(-decay * j)`` (descending), and ``Gamma_k`` is chosen
    so that ``Gamma_k Lambda_k`` equals a Haar-random right-canonical tensor: the
    chain is then a valid MPS (``Gamma_k Lambda_k`` right-canonical), the Lambda
    weights of Algorithm 2 are non-trivial and truncation of the smallest
    values removes a controlled weight.  Returns ``(bonds, Gammas, Lambdas)``.
    """
    bonds, As, _ = mps_tensors(M, d, chi, base_seed=seed, skew=1.5)
    gammas, lams = [], []
    for k in range(M):
        cr = bonds[k + 1]
        lam = np.exp(-decay * np.arange(cr))
        lam /= np.linalg.norm(lam)
        gammas.append(As[k] / lam[None, None, :])
        lams.append(lam)
    return bonds, gammas, lams


def area_law_vidal_chain(M: int, d: int, chi: int, xi_max: float = 10.0, seed: int = 314,
                         device: str | None = None):
    """A chain in Vidal form whose Schmidt spectra decay fastest at the edges (Sec. 3.4.2: entanglement
    grows from the edges to the centre).

    Site k is a right-canonical isometry whose Gaussian is damped along the right bond index,
    ``exp(-b / xi_k)`` with ``xi_k = 1 + xi_max sin(pi (k+1) / M)``, before the QR; the Vidal form
    (true Schmidt coefficients, descending) then comes from the SVD sweep of ``vidal_form``.  Returns
    ``(bonds, Gammas, Lambdas)`` with ``bonds = bond_dims(M, d, chi)``.  ``device='cuda'`` draws the
    Gaussians with a seeded torch generator and runs the QR and SVD sweep there (complex64 torch
    tensors out) for chains whose host SVDs would take minutes.
    """
    bonds = bond_dims(M, d, chi)
    if device is not None:
        return bonds, *_area_law_vidal_torch(M, d, bonds, xi_max, seed, device)
    As = []
    for k in range(M):
        cl, cr = bonds[k], bonds[k + 1]
        g = _gaussian(seed + k, d * cr, cl)
        xi = 1.0 + xi_max * math.sin(math.pi * (k + 1) / M)
        g = g * np.tile(np.exp(-np.arange(cr) / xi), d)[:, None]
        q, r = np.linalg.qr(g, mode="reduced")
        dg = np.diagonal(r)
        q = q * (dg / np.abs(dg))[None, :]
        As.append(np.ascontiguousarray(q.T.reshape(cl, d, cr)))
    gammas, lams = vidal_form(bonds, As)
    return bonds, gammas, lams


def _area_law_vidal_torch(M, d, bonds, xi_max, seed, device):
    """The same construction with torch on ``device``: damped Gaussian, QR, then the left-to-right SVD
    sweep of ``vidal_form`` (complex64 Gammas, float64 Lambdas on the device)."""
    import torch

    R = torch.ones((1, 1), dtype=torch.complex128, device=device)
    lam_prev = torch.ones(1, dtype=torch.float64, device=device)
    gammas, lams = [], []
    for k in range(M):
        cl, cr = bonds[k], bonds[k + 1]
        gen_ = torch.Generator(device=device)
        gen_.manual_seed(int(seed + k))
        g = torch.complex(torch.randn((d * cr, cl), generator=gen_, device=device, dtype=torch.float64),
                          torch.randn((d * cr, cl), generator=gen_, device=device, dtype=torch.float64))
        xi = 1.0 + xi_max * math.sin(math.pi * (k + 1) / M)
        w = torch.exp(-torch.arange(cr, device=device, dtype=torch.float64) / xi).repeat(d)
        q, r = torch.linalg.qr(g * w[:, None], mode="reduced")
        dg = torch.diagonal(r)
        q = q * (dg / dg.abs())[None, :]
        A = q.transpose(0, 1).reshape(cl, d, cr)
        T = torch.einsum("xa,asb->xsb", R, A).reshape(cl * d, cr)
        U, S, Vh = torch.linalg.svd(T, full_matrices=False)
        j = torch.argmax(Vh.abs(), dim=1)
        ph = Vh[torch.arange(cr, device=device), j]
        ph = ph / ph.abs()
        U = U * ph[None, :]
        Vh = Vh * ph.conj()[:, None]
        gammas.append((U.reshape(cl, d, cr) / lam_prev[:, None, None]).to(torch.complex64).contiguous())
        lams.append(S.clone())
        R = S[:, None].to(torch.complex128) * Vh
        lam_prev = S
    return gammas, lams
