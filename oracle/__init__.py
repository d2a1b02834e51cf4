"""FP64 CPU oracle for perfect MPS sampling -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg use this package.  The product library (``paper_2512_20064_gb300``) never
imports it, and the two share no code: the C file ``oracle.c`` restates the
method (Sec. 2.2 sampling workflow, Algorithm 2, Sec. 3.3.1 per-sample
scaling) in complex double precision with plain loops, and implements its own
Philox4x32-10.

Functions
---------
``sample``        rows ``n0 .. n0+N-1``: outcomes, log-probabilities and
                  (optionally) every conditional distribution.
``replay``        teacher-forced replay: follow given outcomes and report the
                  oracle's conditionals, its own draw and the CDF margin.
``born_logprob``  ``log |A_0[s_0] ... A_{M-1}[s_{M-1}]|^2`` (plain definition).
``displacement``  the Zassenhaus displacement matrix of Sec. 3.4.1 (GBS).

``sample`` and ``replay`` also take ``lams`` (Vidal form: the tensors are
Gamma_k and ``lams[k]`` the Schmidt coefficients right of site k) and ``mu``
(GBS: one complex displacement amplitude per sample and site, ``mu[k, i]``
for row i of the call).
``brute_force``   ``|psi(s)|^2`` for all ``d^M`` configurations.
``philox``/``uniform``  the counter-based generator.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc (-O2, OpenMP).  Returns the .so path."""
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def build_variant(src_text: str, out_path: str) -> str:
    """Compile a given oracle source text to ``out_path`` (used by the
    mutation tests, which plant a mistake in a copy of the oracle)."""
    c = out_path[:-3] + ".c"
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", out_path, c, "-lm"],
                   check=True)
    return out_path


def _bind(lib):
    P = ctypes.POINTER
    lib.orc_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
    lib.orc_philox4x32_10.restype = None
    lib.orc_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
    lib.orc_uniform.restype = ctypes.c_double
    lib.orc_sample.argtypes = [
        ctypes.c_int, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_void_p), ctypes.c_uint64, ctypes.c_uint32,
        ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    lib.orc_sample.restype = ctypes.c_int
    lib.orc_sample_segment.argtypes = [
        ctypes.c_int, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_void_p), ctypes.c_int, ctypes.c_uint64,
        ctypes.c_uint32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
        ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    lib.orc_sample_segment.restype = ctypes.c_int
    lib.orc_displacement.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_void_p]
    lib.orc_displacement.restype = None
    lib.orc_born_logprob.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_void_p),
                                     ctypes.c_void_p]
    lib.orc_born_logprob.restype = ctypes.c_double
    lib.orc_brute_force.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_void_p),
                                    ctypes.c_void_p]
    lib.orc_brute_force.restype = ctypes.c_int
    lib.orc_num_threads.argtypes = []
    lib.orc_num_threads.restype = ctypes.c_int
    return lib


def load_variant(path: str):
    """Load an oracle shared object built by :func:`build_variant`."""
    return _bind(ctypes.CDLL(path))


def _load(lib=None):
    global _lib
    if lib is not None:
        return lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


class _Chain:
    """Keeps contiguous copies of the site tensors alive for one C call.

    Tensors are passed as complex128, or as complex64 when every tensor is
    complex64 (the oracle widens float entries to double exactly).
    """

    def __init__(self, bonds, tensors, site_index=None, sites=None):
        self.M = len(bonds) - 1
        self.bonds = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32))
        idx = list(range(self.M)) if site_index is None else list(site_index)
        if len(idx) != self.M:
            raise ValueError("site_index must have M entries")
        sites = range(self.M) if sites is None else sites
        used = sorted({idx[k] for k in sites})
        self.f32 = all(np.asarray(tensors[j]).dtype == np.complex64 for j in used)
        want = np.complex64 if self.f32 else np.complex128
        self.d = None
        conv = {}
        ptrs = [None] * self.M
        for k in sites:
            j = idx[k]
            if j not in conv:
                conv[j] = np.ascontiguousarray(np.asarray(tensors[j], dtype=want))
            A = conv[j]
            if A.ndim != 3 or A.shape[0] != bonds[k] or A.shape[2] != bonds[k + 1]:
                raise ValueError(f"site {k}: shape {A.shape} does not match bonds ({bonds[k]}, {bonds[k+1]})")
            if self.d is None:
                self.d = A.shape[1]
            elif A.shape[1] != self.d:
                raise ValueError("all sites must share d")
            ptrs[k] = A.ctypes.data
        self._keep = conv
        self.ptrs = (ctypes.c_void_p * self.M)(*ptrs)

    def bond_ptr(self):
        return self.bonds.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _vp(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


class _Extras:
    """Optional Vidal weights and GBS displacement amplitudes of one call."""

    def __init__(self, M, bonds, lams=None, mu=None, rows=None, N=None):
        self.lam_ptrs = None
        self._lams = None
        if lams is not None:
            if len(lams) != M:
                raise ValueError("lams must have M entries")
            self._lams = [np.ascontiguousarray(np.asarray(l, dtype=np.float64)) for l in lams]
            for k, l in enumerate(self._lams):
                if l.shape != (bonds[k + 1],):
                    raise ValueError(f"lams[{k}] must have bond[{k + 1}] = {bonds[k + 1]} entries")
            self.lam_ptrs = (ctypes.c_void_p * M)(*[l.ctypes.data for l in self._lams])
        self.mu = None
        if mu is not None:
            mu = np.asarray(mu)
            if mu.ndim != 2 or mu.shape[0] != M:
                raise ValueError("mu must have shape (M, N)")
            self.mu = np.ascontiguousarray(mu.astype(np.complex128))

    def mu_rows(self, i, j):
        """(pointer, ld) of the amplitudes of call rows i .. j-1."""
        if self.mu is None:
            return None, 0
        sub = np.ascontiguousarray(self.mu[:, i:j])
        self._keep = sub
        return ctypes.c_void_p(sub.ctypes.data), sub.shape[1]


def displacement(mu: complex, n: int, lib=None) -> np.ndarray:
    """``exp(-|mu|^2/2) exp(mu a^dag) exp(-mu^* a)`` in the n-level truncation (complex128, n x n)."""
    lib = _load(lib)
    out = np.zeros(2 * n * n, np.float64)
    lib.orc_displacement(float(np.real(mu)), float(np.imag(mu)), int(n), _vp(out))
    return (out[0::2] + 1j * out[1::2]).reshape(n, n)


def philox(ctr, key, lib=None) -> np.ndarray:
    lib = _load(lib)
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def uniform(seed: int, n: int, k: int, job: int = 0, lib=None) -> float:
    return float(_load(lib).orc_uniform(seed, n, k, job))


def num_threads(lib=None) -> int:
    return int(_load(lib).orc_num_threads())


def sample(bonds, tensors, seed: int, N: int, n0: int = 0, job: int = 0, site_index=None,
           want_probs: bool = False, nthreads: int = 0, lib=None, lams=None, mu=None):
    """Sample rows ``n0..n0+N-1``.  Returns ``(samples[N,M] u8, logprob[N] f64[, probs[N,M,d]])``.

    ``lams``: Vidal form (``tensors`` are Gamma_k).  ``mu``: GBS displacement
    amplitudes, shape (M, N), column i for row ``n0 + i``."""
    lib = _load(lib)
    ch = _Chain(bonds, tensors, site_index)
    M, d = ch.M, ch.d
    ex = _Extras(M, bonds, lams, mu)
    if ex.mu is not None and ex.mu.shape[1] != N:
        raise ValueError("mu must have N columns")
    mp, ld = ex.mu_rows(0, N)
    smp = np.zeros((N, M), np.uint8)
    lp = np.zeros(N, np.float64)
    pr = np.zeros((N, M, d), np.float64) if want_probs else None
    rc = lib.orc_sample_segment(M, d, ch.bond_ptr(), ch.ptrs, int(ch.f32), seed, job, n0, N, 0, M, None, 0,
                                _vp(smp), _vp(lp), _vp(pr), None, None, None, nthreads, ex.lam_ptrs, mp, ld, None)
    if rc != 0:
        raise RuntimeError(f"orc_sample_segment failed ({rc})")
    return (smp, lp, pr) if want_probs else (smp, lp)


def sample_prefix(bonds, tensors, seed: int, N: int, K: int, n0: int = 0, nthreads: int = 0, lib=None):
    """Sample rows ``n0..n0+N-1`` over the first ``K`` sites only (used to time a bounded sample)."""
    lib = _load(lib)
    M = len(bonds) - 1
    ch = _Chain(bonds, list(tensors) + [None] * (M - len(tensors)), sites=range(K))
    ldv = max(bonds)
    vstate = np.zeros((N, 2 * ldv), np.float64)
    vstate[:, 0] = 1.0
    smp = np.zeros((N, M), np.uint8)
    lp = np.zeros(N, np.float64)
    rc = lib.orc_sample_segment(M, ch.d, ch.bond_ptr(), ch.ptrs, int(ch.f32), seed, 0, n0, N, 0, K, _vp(vstate),
                                ldv, _vp(smp), _vp(lp), None, None, None, None, nthreads, None, None, 0, None)
    if rc != 0:
        raise RuntimeError(f"orc_sample_segment failed ({rc})")
    return smp[:, :K], lp


def replay(bonds, tensors, seed: int, rows, forced, job: int = 0, site_index=None, nthreads: int = 0, lib=None,
           site_chunk: int | None = None, lams=None, mu=None):
    """Teacher-forced replay of rows ``rows`` (sample indices) along ``forced[R, M]``.

    Returns a dict with ``probs[R,M,d]`` (the oracle's conditionals along the
    forced path), ``own[R,M]`` (the outcome the oracle's own uniform picks at
    each step), ``margin[R,M]`` (distance of that uniform to the nearest
    interior CDF boundary) and ``logprob[R]`` (sum of log conditionals of the
    forced outcomes).

    ``tensors`` may be a list, or a callable ``tensors(k) -> A_k``; with
    ``site_chunk`` the chain is replayed ``site_chunk`` sites at a time,
    carrying the left vectors between segments, so only one chunk of tensors
    needs to be in host memory.  ``lams`` / ``mu`` as in :func:`sample`; for
    ``mu`` column r belongs to replayed row ``rows[r]`` (shape (M, R)).
    """
    lib = _load(lib)
    M = len(bonds) - 1
    ex = _Extras(M, bonds, lams, mu)
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    forced = np.ascontiguousarray(np.asarray(forced, dtype=np.uint8))
    R = rows.shape[0]
    assert forced.shape == (R, M)
    get = tensors if callable(tensors) else None
    chunk = site_chunk or M
    ldv = max(bonds)
    vstate = np.zeros((R, 2 * ldv), np.float64)
    vstate[:, 0] = 1.0
    probs = None
    own = np.zeros((R, M), np.uint8)
    margin = np.zeros((R, M), np.float64)
    lp = np.zeros(R, np.float64)
    for k0 in range(0, M, chunk):
        k1 = min(M, k0 + chunk)
        if get is not None:
            seg = [None] * M
            for k in range(k0, k1):
                seg[k] = get(k)
            ch = _Chain(bonds, seg, sites=range(k0, k1))
        else:
            ch = _Chain(bonds, tensors, site_index, sites=range(k0, k1))
        if probs is None:
            probs = np.zeros((R, M, ch.d), np.float64)
        # rows are arbitrary sample indices: one call over all of them, each row keyed by its own index
        mp, ld = ex.mu_rows(0, R)
        rc = lib.orc_sample_segment(M, ch.d, ch.bond_ptr(), ch.ptrs, int(ch.f32), seed, job, 0, R,
                                    k0, k1, _vp(vstate), ldv, None, _vp(lp), _vp(probs),
                                    _vp(forced), _vp(own), _vp(margin), nthreads, ex.lam_ptrs,
                                    mp, ld, _vp(rows))
        if rc != 0:
            raise RuntimeError(f"orc_sample_segment (replay) failed ({rc})")
        del ch
    return {"probs": probs, "own": own, "margin": margin, "logprob": lp}


def born_logprob(bonds, tensors, config, site_index=None, lib=None) -> float:
    lib = _load(lib)
    ch = _Chain(bonds, tensors, site_index)
    cfg = np.ascontiguousarray(np.asarray(config, dtype=np.uint8))
    assert cfg.shape == (ch.M,)
    return float(lib.orc_born_logprob(ch.M, ch.d, ch.bond_ptr(), ch.ptrs, _vp(cfg)))


def brute_force(bonds, tensors, site_index=None, lib=None) -> np.ndarray:
    """``|psi(s)|^2`` for all configurations, shape ``(d,)*M`` (s_0 first axis)."""
    lib = _load(lib)
    ch = _Chain(bonds, tensors, site_index)
    M, d = ch.M, ch.d
    if d ** M > 1 << 26:
        raise ValueError("too many configurations for brute force")
    out = np.zeros(d ** M, np.float64)
    rc = lib.orc_brute_force(M, d, ch.bond_ptr(), ch.ptrs, _vp(out))
    if rc != 0:
        raise RuntimeError(f"orc_brute_force failed ({rc})")
    return out.reshape((d,) * M)
