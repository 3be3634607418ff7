"""Storage formats of the oracle: binary16/binary32 rounding and the 10-bit colour codes.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this package.

All functions take and return float64 numpy arrays (or integer code arrays) and
implement each format from its definition:

* IEEE 754 binary16 / binary32: round-to-nearest-even to ``p`` significant
  bits with gradual underflow below the smallest normal, overflow to infinity.
* UF10, the 10-bit unsigned float of the paper's A2RGB10F irradiance texture
  (Section 3.3, "Encoding Irradiance": three 10-bit unsigned small floats per
  texel): 5 exponent bits (bias 15), 5 mantissa bits, no sign. Reading
  adopted where the paper is ambiguous: one round-to-nearest-even from the
  stored value, subnormals kept, negative and NaN -> 0, values beyond the
  largest finite code (0x3DF = 64512) clamp to it.
* UNORM10, the alternative reading of the same paragraph (normalised values
  quantised to integers 0..1023): round(clamp(x, 0, 1) * 1023), ties to even.
"""
from __future__ import annotations

import numpy as np

FP16_MAX = 65504.0
UF10_MAX_CODE = 0x3DF
UF10_MAX = 64512.0


def round_to_binary(x, p: int, emin: int) -> np.ndarray:
    """Round to ``p`` significant bits, ties to even, quantum fixed at 2^(emin-p+1) below 2^emin.

    No overflow handling: the caller applies its format's range rule.
    """
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    _, e = np.frexp(a)                      # a = m * 2^e with m in [0.5, 1)
    lead = np.maximum(e - 1, emin)          # exponent of the leading bit (clamped: subnormals)
    quantum = np.ldexp(1.0, lead - (p - 1))
    with np.errstate(invalid="ignore"):
        r = np.rint(a / quantum) * quantum  # division by a power of two is exact; rint = RNE
    return np.copysign(r, x)


def round_fp16(x) -> np.ndarray:
    """binary16 value nearest to x (RNE), with subnormals; overflow -> +-inf."""
    r = round_to_binary(x, 11, -14)
    return np.where(np.abs(r) > FP16_MAX, np.copysign(np.inf, r), r)


def round_fp32(x) -> np.ndarray:
    """binary32 value nearest to x (RNE), with subnormals; overflow -> +-inf."""
    r = round_to_binary(x, 24, -126)
    big = np.ldexp(2.0 - 2.0 ** -23, 127)
    return np.where(np.abs(r) > big, np.copysign(np.inf, r), r)


def round_state(x, fmt: str) -> np.ndarray:
    """Round blended texels to the state storage format ("f16", "f32" or "f64")."""
    if fmt == "f16":
        return round_fp16(x)
    if fmt == "f32":
        return round_fp32(x)
    if fmt == "f64":
        return np.asarray(x, dtype=np.float64)
    raise ValueError(fmt)


def fp16_bits(v) -> np.ndarray:
    """Bit pattern (uint16) of binary16 values ``v`` (v must already be representable)."""
    v = np.asarray(v, dtype=np.float64)
    sign = np.signbit(v).astype(np.uint32) << 15
    a = np.abs(v)
    out = np.zeros(a.shape, dtype=np.uint32)
    nan = np.isnan(a)
    inf = np.isinf(a)
    fin = ~(nan | inf)
    sub = fin & (a < 2.0 ** -14)
    nrm = fin & ~sub
    out[sub] = np.rint(a[sub] / 2.0 ** -24).astype(np.uint32)
    _, e = np.frexp(a[nrm])
    E = e - 1
    mant = np.rint((a[nrm] / np.ldexp(1.0, E) - 1.0) * 1024.0).astype(np.uint32)
    out[nrm] = ((E + 15).astype(np.uint32) << 10) | mant
    out[inf] = 0x7C00
    out[nan] = 0x7E00
    return (out | np.where(nan, 0, sign)).astype(np.uint16)


def fp16_value(bits) -> np.ndarray:
    """float64 value of binary16 bit patterns."""
    b = np.asarray(bits, dtype=np.uint32)
    s = np.where(b & 0x8000, -1.0, 1.0)
    E = ((b >> 10) & 0x1F).astype(np.int64)
    m = (b & 0x3FF).astype(np.float64)
    sub = s * m * 2.0 ** -24
    nrm = s * np.ldexp(1.0 + m / 1024.0, E - 15)
    special = np.where(m == 0, s * np.inf, np.nan)
    return np.where(E == 0, sub, np.where(E == 31, special, nrm))


def uf10_code(x) -> np.ndarray:
    """10-bit unsigned-float code (uint16) of x: one RNE rounding, clamp to 0x3DF, <=0/NaN -> 0."""
    x = np.asarray(x, dtype=np.float64)
    with np.errstate(invalid="ignore"):
        pos = np.where(np.isnan(x) | (x <= 0.0), 0.0, x)
    r = round_to_binary(pos, 6, -14)
    r = np.minimum(r, UF10_MAX)
    out = np.zeros(r.shape, dtype=np.uint32)
    sub = r < 2.0 ** -14
    nrm = ~sub
    out[sub] = np.rint(r[sub] / 2.0 ** -19).astype(np.uint32)
    _, e = np.frexp(r[nrm])
    E = e - 1
    mant = np.rint((r[nrm] / np.ldexp(1.0, E) - 1.0) * 32.0).astype(np.uint32)
    out[nrm] = ((E + 15).astype(np.uint32) << 5) | mant
    return out.astype(np.uint16)


def uf10_value(code) -> np.ndarray:
    """float64 value of 10-bit unsigned-float codes (finite codes only)."""
    c = np.asarray(code, dtype=np.uint32)
    E = ((c >> 5) & 0x1F).astype(np.int64)
    m = (c & 0x1F).astype(np.float64)
    return np.where(E == 0, m * 2.0 ** -19, np.ldexp(1.0 + m / 32.0, E - 15))


def unorm10_code(x) -> np.ndarray:
    """round(clamp(x, 0, 1) * 1023), ties to even; NaN -> 0."""
    x = np.asarray(x, dtype=np.float64)
    x = np.where(np.isnan(x), 0.0, x)
    return np.rint(np.clip(x, 0.0, 1.0) * 1023.0).astype(np.uint16)


def unorm10_value(code) -> np.ndarray:
    return np.asarray(code, dtype=np.float64) / 1023.0


def color_code(x, kind: str) -> np.ndarray:
    if kind == "uf10":
        return uf10_code(x)
    if kind == "unorm10":
        return unorm10_code(x)
    raise ValueError(kind)


def color_value(code, kind: str) -> np.ndarray:
    if kind == "uf10":
        return uf10_value(code)
    if kind == "unorm10":
        return unorm10_value(code)
    raise ValueError(kind)
