"""Python binding of ``libfastmps.so``: GB300 (sm_103a) perfect sampling from a right-canonical MPS.

The binding only marshals arguments for the C ABI declared in
``include/fastmps.h``; every step of the sampling runs in the library's CUDA
kernels.  There is no CPU fallback: if the library is not built, or the
device is not an sm_103a GPU, the calls raise.

Low-level functions carry the C names (``fastmps_create``, ``fastmps_load_site``,
``fastmps_sample``, ``fastmps_sample_ex``, ``fastmps_destroy`` ...); the
:class:`Sampler` class wraps a handle for convenience.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from .native import LIB, build

__all__ = [
    "FastMPSError", "Sampler", "load_library", "build", "PRECISIONS", "RESIDENCIES",
    "fastmps_create", "fastmps_destroy", "fastmps_last_error", "fastmps_load_site", "fastmps_load_pool",
    "fastmps_map_site", "fastmps_sample", "fastmps_sample_ex", "fastmps_sample_traced", "fastmps_sample_noalloc", "fastmps_sample_batch",
    "fastmps_get_stats", "fastmps_load_site_vidal", "fastmps_load_pool_vidal", "fastmps_displacement",
    "fastmps_sample_displaced", "fastmps_bond_filter", "fastmps_load_site_vidal_truncated",
    "fastmps_version",
    "fastmps_default_options",
]

OK = 0
ERR_NAMES = {-1: "INVALID_ARG", -2: "SHAPE", -3: "NOT_LOADED", -4: "OOM", -5: "CUDA", -6: "TIMEOUT",
             -7: "UNSUPPORTED", -8: "NUMERIC"}
PRECISIONS = {"fp32": 0, "bf16x2": 1, "bf16x3": 2, "bf16x3l": 3, "bf16x4": 4, "fp8x1": 5, "fp8x2": 6, "fp16x2": 7,
              "fp16x3": 8}
RESIDENCIES = {"hbm": 0, "host_stream": 1}
MEASUREMENTS = {"separate": 0, "cta": 1, "cluster": 2}
C64, C128 = 0, 1


class fastmps_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("residency", ctypes.c_int), ("max_microbatch", ctypes.c_int64),
                ("autotune", ctypes.c_int), ("stream", ctypes.c_void_p), ("fused_measure", ctypes.c_int),
                ("k_split", ctypes.c_int), ("accum_chunk", ctypes.c_int)]


class fastmps_stats(ctypes.Structure):
    _fields_ = [("ms_total", ctypes.c_double), ("ms_contract", ctypes.c_double), ("ms_measure", ctypes.c_double),
                ("launches", ctypes.c_int64), ("contract_launches", ctypes.c_int64),
                ("flops_algorithmic", ctypes.c_double), ("flops_issued", ctypes.c_double),
                ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64), ("ms_h2d", ctypes.c_double)]


class fastmps_job(ctypes.Structure):
    _fields_ = [("chain", ctypes.c_void_p), ("M", ctypes.c_int), ("d", ctypes.c_int),
                ("bond_dims", ctypes.POINTER(ctypes.c_int)), ("n0", ctypes.c_int64), ("N", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("job", ctypes.c_uint32), ("out_samples", ctypes.c_void_p),
                ("out_logprob", ctypes.c_void_p)]


class FastMPSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fastmps error {code} ({ERR_NAMES.get(code, '?')}): {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()


def load_library(path: str | None = None, build_if_missing: bool = True) -> ctypes.CDLL:
    """Load the shared library (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB
        if path is None and build_if_missing:
            build()
        if not os.path.exists(p):
            raise ImportError(f"libfastmps.so not found at {p}; run paper_2512_20064_gb300.native.build()")
        lib = ctypes.CDLL(p)
        H = ctypes.c_void_p
        P = ctypes.POINTER
        lib.fastmps_default_options.argtypes = [P(fastmps_options)]
        lib.fastmps_default_options.restype = None
        lib.fastmps_create.argtypes = [P(H), ctypes.c_int, P(fastmps_options)]
        lib.fastmps_create.restype = ctypes.c_int
        lib.fastmps_destroy.argtypes = [H]
        lib.fastmps_destroy.restype = None
        lib.fastmps_last_error.argtypes = [H]
        lib.fastmps_last_error.restype = ctypes.c_char_p
        for name in ("fastmps_load_site", "fastmps_load_pool"):
            f = getattr(lib, name)
            f.argtypes = [H, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
            f.restype = ctypes.c_int
        for name in ("fastmps_load_site_vidal", "fastmps_load_pool_vidal"):
            f = getattr(lib, name)
            f.argtypes = [H, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                          ctypes.c_int]
            f.restype = ctypes.c_int
        lib.fastmps_load_site_vidal_truncated.argtypes = [H, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                                          ctypes.c_int, ctypes.c_int]
        lib.fastmps_load_site_vidal_truncated.restype = ctypes.c_int
        lib.fastmps_bond_filter.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_void_p),
                                            ctypes.c_int, ctypes.c_double, ctypes.c_int, P(ctypes.c_int),
                                            ctypes.c_void_p]
        lib.fastmps_bond_filter.restype = ctypes.c_int
        lib.fastmps_displacement.argtypes = [H, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        lib.fastmps_displacement.restype = ctypes.c_int
        lib.fastmps_sample_displaced.argtypes = [H, ctypes.c_int, ctypes.c_int, P(ctypes.c_int), ctypes.c_int64,
                                                 ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p,
                                                 ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                 ctypes.c_void_p]
        lib.fastmps_sample_displaced.restype = ctypes.c_int
        lib.fastmps_map_site.argtypes = [H, ctypes.c_int, ctypes.c_int]
        lib.fastmps_map_site.restype = ctypes.c_int
        lib.fastmps_sample.argtypes = [H, ctypes.c_int, ctypes.c_int, P(ctypes.c_int), ctypes.c_int64,
                                       ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
        lib.fastmps_sample.restype = ctypes.c_int
        lib.fastmps_sample_ex.argtypes = [H, ctypes.c_int, ctypes.c_int, P(ctypes.c_int), ctypes.c_int64,
                                          ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        lib.fastmps_sample_ex.restype = ctypes.c_int
        lib.fastmps_sample_traced.argtypes = [H, ctypes.c_int, ctypes.c_int, P(ctypes.c_int), ctypes.c_int64,
                                              ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        lib.fastmps_sample_traced.restype = ctypes.c_int
        lib.fastmps_sample_noalloc.argtypes = [H, ctypes.c_int, ctypes.c_int, P(ctypes.c_int), ctypes.c_int64,
                                               ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p,
                                               ctypes.c_void_p]
        lib.fastmps_sample_noalloc.restype = ctypes.c_int
        lib.fastmps_sample_batch.argtypes = [H, ctypes.c_int, P(fastmps_job)]
        lib.fastmps_sample_batch.restype = ctypes.c_int
        lib.fastmps_get_stats.argtypes = [H, P(fastmps_stats)]
        lib.fastmps_get_stats.restype = ctypes.c_int
        lib.fastmps_selftest_bounded_wait.argtypes = [ctypes.c_int, ctypes.c_double, P(ctypes.c_int),
                                                      P(ctypes.c_double)]
        lib.fastmps_selftest_bounded_wait.restype = ctypes.c_int
        lib.fastmps_version.argtypes = []
        lib.fastmps_version.restype = ctypes.c_char_p
        if path is None:
            _lib = lib
        return lib


# ---------------------------------------------------------------------------
# Low-level functions with the C names (argument marshalling only).
# ---------------------------------------------------------------------------

def _check(lib, h, rc):
    if rc != OK:
        msg = lib.fastmps_last_error(h)
        raise FastMPSError(rc, msg.decode() if msg else "")


def fastmps_selftest_bounded_wait(device: int = 0, limit_ms: float = 50.0):
    """Run the bounded-wait self-test; returns (status code, device milliseconds waited)."""
    lib = load_library()
    st = ctypes.c_int()
    ms = ctypes.c_double()
    rc = lib.fastmps_selftest_bounded_wait(device, limit_ms, ctypes.byref(st), ctypes.byref(ms))
    _check(lib, None, rc)
    return st.value, ms.value


def fastmps_version() -> str:
    return load_library().fastmps_version().decode()


def fastmps_default_options() -> fastmps_options:
    o = fastmps_options()
    load_library().fastmps_default_options(ctypes.byref(o))
    return o


def fastmps_create(device: int = 0, options: fastmps_options | None = None) -> ctypes.c_void_p:
    lib = load_library()
    h = ctypes.c_void_p()
    rc = lib.fastmps_create(ctypes.byref(h), device, ctypes.byref(options) if options is not None else None)
    _check(lib, None, rc)
    return h


def fastmps_destroy(h) -> None:
    load_library().fastmps_destroy(h)


def fastmps_last_error(h) -> str:
    m = load_library().fastmps_last_error(h)
    return m.decode() if m else ""


def _tensor_arg(A):
    """(pointer, keep-alive object, dtype code, shape) of a site tensor: a numpy array or a torch tensor
    (host or CUDA) of shape (chi_l, d, chi_r), complex64 or complex128."""
    if hasattr(A, "data_ptr") and hasattr(A, "is_cuda"):
        import torch

        if A.dim() != 3:
            raise ValueError("site tensor must have shape (chi_l, d, chi_r)")
        if A.dtype not in (torch.complex64, torch.complex128):
            A = A.to(torch.complex128)
        A = A.contiguous()
        return A.data_ptr(), A, (C64 if A.dtype == torch.complex64 else C128), tuple(A.shape)
    A = np.asarray(A)
    if A.ndim != 3:
        raise ValueError("site tensor must have shape (chi_l, d, chi_r)")
    if A.dtype not in (np.complex64, np.complex128):
        A = A.astype(np.complex128)
    A = np.ascontiguousarray(A)
    return A.ctypes.data, A, (C64 if A.dtype == np.complex64 else C128), A.shape


def fastmps_load_site(h, k: int, A) -> None:
    lib = load_library()
    ptr, keep, dt, (cl, d, cr) = _tensor_arg(A)
    _check(lib, h, lib.fastmps_load_site(h, k, cl, d, cr, ptr, dt))
    del keep


def fastmps_load_pool(h, j: int, A) -> None:
    lib = load_library()
    ptr, keep, dt, (cl, d, cr) = _tensor_arg(A)
    _check(lib, h, lib.fastmps_load_pool(h, j, cl, d, cr, ptr, dt))
    del keep


def _lambda_arg(Lam, dt):
    """(pointer, keep-alive) of Schmidt coefficients in the real type matching tensor dtype code dt."""
    if hasattr(Lam, "data_ptr") and hasattr(Lam, "is_cuda"):
        import torch

        Lam = Lam.to(torch.float64 if dt == C128 else torch.float32).contiguous()
        return Lam.data_ptr(), Lam
    Lam = np.ascontiguousarray(np.asarray(Lam, dtype=np.float64 if dt == C128 else np.float32))
    return Lam.ctypes.data, Lam


def fastmps_load_site_vidal(h, k: int, Gamma, Lam) -> None:
    """Load a Vidal-form site: Gamma (chi_l, d, chi_r) complex and Lambda (chi_r,) real."""
    lib = load_library()
    ptr, keep, dt, (cl, d, cr) = _tensor_arg(Gamma)
    lp, lkeep = _lambda_arg(Lam, dt)
    _check(lib, h, lib.fastmps_load_site_vidal(h, k, cl, d, cr, ptr, lp, dt))
    del keep, lkeep


def fastmps_load_pool_vidal(h, j: int, Gamma, Lam) -> None:
    lib = load_library()
    ptr, keep, dt, (cl, d, cr) = _tensor_arg(Gamma)
    lp, lkeep = _lambda_arg(Lam, dt)
    _check(lib, h, lib.fastmps_load_pool_vidal(h, j, cl, d, cr, ptr, lp, dt))
    del keep, lkeep


def fastmps_load_site_vidal_truncated(h, k: int, Gamma, Lam, keep_l: int, keep_r: int) -> None:
    """Load the leading block Gamma[:keep_l, :, :keep_r], Lambda[:keep_r] of a Vidal-form site."""
    lib = load_library()
    ptr, keep, dt, (cl, d, cr) = _tensor_arg(Gamma)
    lp, lkeep = _lambda_arg(Lam, dt)
    _check(lib, h, lib.fastmps_load_site_vidal_truncated(h, k, cl, d, cr, ptr, lp, dt, keep_l, keep_r))
    del keep, lkeep


def fastmps_bond_filter(bonds, lams, d: int, chi: int, eps: float = 0.0, align: int = 1):
    """Dynamic bond dimensions from the Schmidt spectra ``lams[k]`` (right of site k; host code, no GPU).

    Returns ``(bonds_out[M+1], discarded[M+1])``."""
    lib = load_library()
    M = len(bonds) - 1
    bi = (ctypes.c_int * (M + 1))(*[int(x) for x in bonds])
    keep = [np.ascontiguousarray(np.asarray(lams[k], dtype=np.float64)) for k in range(max(0, M - 1))]
    ptrs = (ctypes.c_void_p * max(1, M - 1))(*[a.ctypes.data for a in keep])
    bo = (ctypes.c_int * (M + 1))()
    disc = np.zeros(M + 1, np.float64)
    rc = lib.fastmps_bond_filter(M, d, bi, ptrs, int(chi), float(eps), int(align), bo, disc.ctypes.data)
    _check(lib, None, rc)
    return [int(x) for x in bo], disc


def _complex64_arg(x):
    """(pointer, keep-alive, shape) of a complex64 array: numpy (converted if needed) or torch (host or CUDA)."""
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        import torch

        x = x.to(torch.complex64).contiguous()
        return x.data_ptr(), x, tuple(x.shape)
    x = np.ascontiguousarray(np.asarray(x, dtype=np.complex64))
    return x.ctypes.data, x, x.shape


def fastmps_displacement(h, mu, d: int, out=None):
    """Zassenhaus displacement matrices of N amplitudes: returns D[s, t, n] (complex64, batch last)."""
    lib = load_library()
    mp, keep, shape = _complex64_arg(mu)
    N = int(np.prod(shape))
    if out is None:
        out = np.empty((d, d, N), np.complex64)
    _check(lib, h, lib.fastmps_displacement(h, N, d, mp, _ptr(out)))
    del keep
    return out


def fastmps_sample_displaced(h, M: int, d: int, bonds, n0: int, N: int, seed: int, job: int, mu, out_samples,
                             out_logprob, trace_rows: int = 0, trace_probs=None) -> None:
    """``mu``: complex64 amplitudes of shape (M, N) (numpy, or a torch tensor on the host or the device)."""
    lib = load_library()
    mp, keep, shape = _complex64_arg(mu)
    if len(shape) != 2 or shape[0] != M:
        raise ValueError("mu must have shape (M, ld) with ld >= N")
    b = (ctypes.c_int * (M + 1))(*[int(x) for x in bonds])
    _check(lib, h, lib.fastmps_sample_displaced(h, M, d, b, n0, N, seed, job, mp, shape[1], _ptr(out_samples),
                                                _ptr(out_logprob), trace_rows, _ptr(trace_probs)))
    del keep


def fastmps_map_site(h, k: int, j: int) -> None:
    lib = load_library()
    _check(lib, h, lib.fastmps_map_site(h, k, j))


def _ptr(x):
    """Raw address of a numpy array or a torch tensor (host or device); None stays NULL."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("output arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("output tensors must be contiguous")
        return x.data_ptr()
    raise TypeError("outputs must be numpy arrays or torch tensors")


def fastmps_sample_ex(h, M: int, d: int, bonds, n0: int, N: int, seed: int, job: int, out_samples, out_logprob,
                      trace_rows: int = 0, trace_probs=None) -> None:
    lib = load_library()
    b = (ctypes.c_int * (M + 1))(*[int(x) for x in bonds])
    _check(lib, h, lib.fastmps_sample_ex(h, M, d, b, n0, N, seed, job, _ptr(out_samples), _ptr(out_logprob),
                                         trace_rows, _ptr(trace_probs)))


def fastmps_sample_traced(h, M: int, d: int, bonds, n0: int, N: int, seed: int, job: int, out_samples,
                          out_logprob, trace_list, trace_probs) -> None:
    """As ``fastmps_sample_ex``, tracing the conditionals of the listed call rows (any rows of the call)."""
    lib = load_library()
    b = (ctypes.c_int * (M + 1))(*[int(x) for x in bonds])
    rows = np.ascontiguousarray(np.asarray(trace_list, dtype=np.int64))
    _check(lib, h, lib.fastmps_sample_traced(h, M, d, b, n0, N, seed, job, _ptr(out_samples), _ptr(out_logprob),
                                             rows.ctypes.data if rows.size else None, rows.size, _ptr(trace_probs)))


def fastmps_sample_noalloc(h, M: int, d: int, bonds, n0: int, N: int, seed: int, job: int, out_samples,
                           out_logprob) -> None:
    """Sampling that allocates nothing (static 64 MiB device scratch); outputs must be device memory.

    For callers that cannot allocate device memory while they sample (memory owned by their own
    caching allocator, a fixed budget, a service that allocates only at start-up).  The first call on
    a device looks up the scratch address and should come before any stream capture; calls that
    overlap on the GPU share the scratch and must be serialised."""
    lib = load_library()
    b = (ctypes.c_int * (M + 1))(*[int(x) for x in bonds])
    _check(lib, h, lib.fastmps_sample_noalloc(h, M, d, b, n0, N, seed, job, _ptr(out_samples), _ptr(out_logprob)))


def fastmps_sample(h, M: int, d: int, bonds, N: int, seed: int, out_samples, out_logprob) -> None:
    lib = load_library()
    b = (ctypes.c_int * (M + 1))(*[int(x) for x in bonds])
    _check(lib, h, lib.fastmps_sample(h, M, d, b, N, seed, _ptr(out_samples), _ptr(out_logprob)))


def fastmps_sample_batch(runner, jobs) -> None:
    """Sample many independent MPS together.  ``jobs``: list of dicts with keys chain (a handle),
    bonds, d, N, seed and optionally n0, job, out_samples, out_logprob (numpy arrays or torch tensors)."""
    lib = load_library()
    arr = (fastmps_job * max(1, len(jobs)))()
    keep = []
    for i, j in enumerate(jobs):
        bonds = (ctypes.c_int * len(j["bonds"]))(*[int(x) for x in j["bonds"]])
        keep.append(bonds)
        arr[i].chain = j["chain"].value if isinstance(j["chain"], ctypes.c_void_p) else j["chain"]
        arr[i].M = len(j["bonds"]) - 1
        arr[i].d = int(j["d"])
        arr[i].bond_dims = bonds
        arr[i].n0 = int(j.get("n0", 0))
        arr[i].N = int(j["N"])
        arr[i].seed = int(j["seed"])
        arr[i].job = int(j.get("job", 0))
        arr[i].out_samples = _ptr(j.get("out_samples"))
        arr[i].out_logprob = _ptr(j.get("out_logprob"))
    _check(lib, runner, lib.fastmps_sample_batch(runner, len(jobs), arr))


def fastmps_get_stats(h) -> dict:
    lib = load_library()
    s = fastmps_stats()
    _check(lib, h, lib.fastmps_get_stats(h, ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in fastmps_stats._fields_}


class Sampler:
    """A handle of the library: load site tensors once, then sample many times."""

    def __init__(self, device: int = 0, precision: str = "fp32", residency: str = "hbm", max_microbatch: int = 0,
                 stream=None, fused_measure=False, autotune: bool = False, k_split: int = 0,
                 accum_chunk: int = 0):
        """``fused_measure``: False / "separate" (measurement kernel after each contraction), True / "cta"
        (measurement warps inside the contraction kernel), "cluster" (single-pass cluster kernel, no
        scratch, where a site's row fits one cluster)."""
        o = fastmps_default_options()
        o.fused_measure = MEASUREMENTS[fused_measure] if isinstance(fused_measure, str) else int(bool(fused_measure))
        o.autotune = int(bool(autotune))
        o.k_split = int(k_split)
        o.accum_chunk = int(accum_chunk)
        o.precision = PRECISIONS[precision]
        o.residency = RESIDENCIES[residency]
        o.max_microbatch = int(max_microbatch)
        if stream is not None:
            o.stream = int(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)
        self.precision = precision
        self.residency = residency
        self.h = fastmps_create(device, o)

    def close(self):
        if getattr(self, "h", None) is not None:
            fastmps_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def load_site(self, k: int, A):
        fastmps_load_site(self.h, k, A)

    def load_chain(self, tensors, site_index=None):
        """Load every site; with ``site_index`` the tensors form a pool and site k maps to ``site_index[k]``."""
        if site_index is None:
            for k, A in enumerate(tensors):
                fastmps_load_site(self.h, k, A)
        else:
            for j, A in enumerate(tensors):
                fastmps_load_pool(self.h, j, A)
            for k, j in enumerate(site_index):
                fastmps_map_site(self.h, k, j)

    def load_site_vidal(self, k: int, Gamma, Lam):
        fastmps_load_site_vidal(self.h, k, Gamma, Lam)

    def load_chain_vidal(self, gammas, lams):
        """Load a whole chain given in Vidal form (Gamma_k, Lambda_k)."""
        for k, (G, L) in enumerate(zip(gammas, lams)):
            fastmps_load_site_vidal(self.h, k, G, L)

    def load_chain_vidal_truncated(self, gammas, lams, bonds):
        """Load the leading blocks ``Gamma_k[:bonds[k], :, :bonds[k+1]]`` (e.g. from ``fastmps_bond_filter``)."""
        for k, (G, L) in enumerate(zip(gammas, lams)):
            fastmps_load_site_vidal_truncated(self.h, k, G, L, int(bonds[k]), int(bonds[k + 1]))

    def displacement(self, mu, d: int):
        """Batched Zassenhaus displacement matrices, D[s, t, n]."""
        return fastmps_displacement(self.h, mu, d)

    def sample(self, bonds, d: int, N: int, seed: int, n0: int = 0, job: int = 0, out_samples=None,
               out_logprob=None, trace_rows: int = 0, mu=None, trace_list=None):
        """Draw rows ``n0 .. n0+N-1``.  Returns ``(samples[N, M] uint8, logprob[N] float64[, trace[M, R, d]])``.

        Outputs are numpy arrays unless ``out_samples`` / ``out_logprob`` are given
        (numpy arrays or torch tensors, host or CUDA).  ``mu`` (shape (M, N), complex):
        per-sample GBS displacement amplitudes (Sec. 3.4.1).  The trace holds the conditionals
        of call rows ``0 .. trace_rows-1``, or of the call rows in ``trace_list``.
        """
        M = len(bonds) - 1
        if out_samples is None:
            out_samples = np.empty((N, M), np.uint8)
        if out_logprob is None:
            out_logprob = np.empty(N, np.float64)
        if trace_list is not None:
            trace = np.empty((M, len(trace_list), d), np.float64)
            fastmps_sample_traced(self.h, M, d, bonds, n0, N, seed, job, out_samples, out_logprob, trace_list, trace)
            return out_samples, out_logprob, trace
        trace = np.empty((M, trace_rows, d), np.float64) if trace_rows > 0 else None
        if mu is not None:
            fastmps_sample_displaced(self.h, M, d, bonds, n0, N, seed, job, mu, out_samples, out_logprob,
                                     trace_rows, trace)
        else:
            fastmps_sample_ex(self.h, M, d, bonds, n0, N, seed, job, out_samples, out_logprob, trace_rows, trace)
        if trace is not None:
            return out_samples, out_logprob, trace
        return out_samples, out_logprob

    def stats(self) -> dict:
        return fastmps_get_stats(self.h)
