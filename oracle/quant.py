"""What a low-precision store of a site tensor represents -- TEST INFRASTRUCTURE.

The low-precision device paths keep site tensors in bfloat16 (Sec. 3.3.2:
tensors kept in a 16-bit format for storage and transfer).  To measure their
arithmetic error rather than their storage error, the oracle is also run on
the tensors those stores represent.  This module restates the storage format
from its definition (IEEE-754 binary32 -> bfloat16, round to nearest, ties to
even) with integer operations on the float32 bit patterns; it shares nothing
with the CUDA path.

Pinned in ``tests/oracle_pins.py`` (``QUANT_PINS``): hand-derived rounding cases of
every format, the hi/lo splits of both 16-bit formats, and an independent cross-check against
torch's casts; planted
mistakes (truncation, ties away from zero, no saturation, a wrong subnormal
floor, a ceiling scale, ...) are each caught (``tests/test_oracle_mutants.py``).
"""
from __future__ import annotations

import numpy as np


def bf16_round(x) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float32.

    NaN inputs are not expected (site tensors are finite).
    """
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(x.shape)


def bf16_split(x):
    """``hi = bf16(x)``, ``lo = bf16(x - hi)``, the difference taken in float32."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    hi = bf16_round(x)
    lo = bf16_round((x - hi).astype(np.float32))
    return hi, lo


def dequant_bf16(A, planes: int = 1) -> np.ndarray:
    """The complex128 tensor that a BF16 store of ``A`` represents.

    ``planes=1``: real and imaginary parts each cast to float32, then rounded to
    bfloat16.  ``planes=2``: each stored as a ``hi + lo`` bfloat16 pair.
    """
    A = np.asarray(A)
    re = np.asarray(A.real, dtype=np.float32)
    im = np.asarray(A.imag, dtype=np.float32)
    if planes == 1:
        return bf16_round(re).astype(np.float64) + 1j * bf16_round(im).astype(np.float64)
    rh, rl = bf16_split(re)
    ih, il = bf16_split(im)
    return (rh.astype(np.float64) + rl.astype(np.float64)) + 1j * (ih.astype(np.float64) + il.astype(np.float64))


def complex64_of(A) -> np.ndarray:
    """The complex128 tensor that a complex64 store of ``A`` represents."""
    return np.asarray(A).astype(np.complex64).astype(np.complex128)


# ---------------------------------------------------------------------------
# FP8 E4M3 (the OCP "E4M3FN" format: 1 sign bit, 4 exponent bits with bias 7,
# 3 mantissa bits, largest finite value 448, subnormals down to 2^-9, no
# infinities), round to nearest, ties to even, saturating to +-448.
# ---------------------------------------------------------------------------

E4M3_MAX = 448.0


def e4m3_round(x) -> np.ndarray:
    """Round to the nearest E4M3 value (ties to even), saturating at +-448; float64 result."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    _, ex = np.frexp(a)                      # a = m * 2^ex, m in [0.5, 1)
    e = np.maximum(ex - 1, -6)               # exponent of the leading bit; -6 for subnormals
    q = np.ldexp(1.0, (e - 3).astype(np.int64))  # spacing of representable values at that exponent
    r = np.round(a / q) * q                  # numpy rounds halves to even
    r = np.minimum(r, E4M3_MAX)
    r[a == 0] = 0.0
    return np.copysign(r, x)


def e4m3_site_scale(A) -> float:
    """Power-of-two scale of an FP8 site store: the largest 2^j with max|Re, Im| * 2^j <= 448."""
    A = np.asarray(A)
    m = float(max(np.abs(np.asarray(A.real, np.float32)).max(), np.abs(np.asarray(A.imag, np.float32)).max()))
    if m == 0.0:
        return 1.0
    return float(2.0 ** np.floor(np.log2(E4M3_MAX / m)))


def dequant_e4m3(A) -> np.ndarray:
    """The complex128 tensor an FP8 E4M3 store with a per-site power-of-two scale represents."""
    s = e4m3_site_scale(A)
    re = np.asarray(A.real, dtype=np.float32).astype(np.float64)
    im = np.asarray(A.imag, dtype=np.float32).astype(np.float64)
    return (e4m3_round(re * s) + 1j * e4m3_round(im * s)) / s


# ---------------------------------------------------------------------------
# FP16 (IEEE-754 binary16: 11 significant bits, 5 exponent bits with bias 15,
# largest finite 65504, subnormals down to 2^-24), round to nearest, ties to
# even; stored with a per-site power-of-two scale.
# ---------------------------------------------------------------------------

FP16_TOP = 32768.0


def fp16_round(x) -> np.ndarray:
    """Round float32 values to the nearest binary16 value (ties to even), returned as float64.

    Restated from the format with integer arithmetic on the float32 bit patterns (finite inputs
    whose magnitude stays below 65520, so that nothing rounds to infinity)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    a = np.abs(x).astype(np.float64)
    _, ex = np.frexp(a)                      # a = m * 2^ex, m in [0.5, 1)
    e = np.maximum(ex - 1, -14)              # exponent of the leading bit; -14 for subnormals
    q = np.ldexp(1.0, (e - 10).astype(np.int64))  # spacing of representable values at that exponent
    r = np.round(a / q) * q                  # a / q is exact in float64; numpy rounds halves to even
    r[a == 0] = 0.0
    return np.copysign(r, x.astype(np.float64))


def fp16_site_scale(A) -> float:
    """Power-of-two scale of an FP16 site store: the largest 2^j with max|Re, Im| * 2^j <= 32768."""
    A = np.asarray(A)
    m = float(max(np.abs(np.asarray(A.real, np.float32)).max(), np.abs(np.asarray(A.imag, np.float32)).max()))
    if m == 0.0:
        return 1.0
    return float(2.0 ** np.floor(np.log2(FP16_TOP / m)))


def fp16_split(x):
    """``hi = fp16(x)``, ``lo = fp16(x - hi)``: two binary16 planes of float32 values (the difference is
    exact in float32), returned as float64."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    hi = fp16_round(x)
    lo = fp16_round((x.astype(np.float64) - hi).astype(np.float32))
    return hi, lo


def dequant_fp16(A, planes: int = 1) -> np.ndarray:
    """The complex128 tensor an FP16 store with a per-site power-of-two scale represents.

    ``planes=1``: each scaled part rounded to binary16.  ``planes=2``: each scaled part held as a
    ``hi + lo`` binary16 pair at the same scale (Sec. 3.3.2's 16-bit format, two planes)."""
    s = fp16_site_scale(A)
    re = np.asarray(A.real, dtype=np.float32) * np.float32(s)
    im = np.asarray(A.imag, dtype=np.float32) * np.float32(s)
    if planes == 1:
        return (fp16_round(re) + 1j * fp16_round(im)) / s
    rh, rl = fp16_split(re)
    ih, il = fp16_split(im)
    return ((rh + rl) + 1j * (ih + il)) / s

