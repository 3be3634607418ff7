"""Pins of the oracle's storage formats against library casts and brute force."""
import numpy as np
import pytest

from oracle import numerics as nu


def _all_fp16_values():
    bits = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)
    vals = bits.view(np.float16).astype(np.float64)
    return bits, vals


def test_fp16_rounding_matches_numpy_cast_on_values_midpoints_and_random():
    _, vals = _all_fp16_values()
    fin = np.sort(np.unique(vals[np.isfinite(vals)]))
    mids = (fin[:-1] + fin[1:]) / 2.0          # exact ties: RNE decides
    rng = np.random.default_rng(1)
    rand = np.concatenate([
        rng.standard_normal(200000) * 10.0 ** rng.integers(-9, 6, 200000),
        np.array([65504.0, 65519.999, 65520.0, 70000.0, -65520.0, 2.0 ** -25, 2.0 ** -26,
                  3 * 2.0 ** -26, 0.0, -0.0]),
    ])
    for x in (fin, mids, rand):
        with np.errstate(over="ignore"):
            want = x.astype(np.float16).astype(np.float64)
        got = nu.round_fp16(x)
        np.testing.assert_array_equal(got, want)


def test_fp32_rounding_matches_numpy_cast():
    rng = np.random.default_rng(2)
    x = rng.standard_normal(300000) * 10.0 ** rng.integers(-45, 38, 300000)
    f = x.astype(np.float32)
    up = np.nextafter(f, np.float32(np.inf)).astype(np.float64)
    mids = (f.astype(np.float64) + up) / 2.0
    for v in (x, mids):
        np.testing.assert_array_equal(nu.round_fp32(v), v.astype(np.float32).astype(np.float64))


def test_fp16_bits_and_values_match_numpy_views():
    bits, vals = _all_fp16_values()
    fin = np.isfinite(vals)
    np.testing.assert_array_equal(nu.fp16_bits(vals[fin]), bits[fin])
    got = nu.fp16_value(bits)
    np.testing.assert_array_equal(got[fin], vals[fin])
    assert np.all(np.isnan(got[np.isnan(vals)]))
    assert np.all(got[np.isinf(vals)] == vals[np.isinf(vals)])


def _uf10_table():
    codes = np.arange(0x3E0, dtype=np.int64)            # every finite code 0..0x3DF
    vals = np.array([((2.0 ** -14) * (c & 31) / 32.0) if (c >> 5) == 0
                     else (2.0 ** ((c >> 5) - 15)) * (1.0 + (c & 31) / 32.0) for c in codes])
    return codes, vals


def _uf10_brute(x):
    """Nearest finite UF10 value, ties to the even code; <=0/NaN -> 0; clamp above the top."""
    codes, vals = _uf10_table()
    out = np.zeros(len(x), dtype=np.int64)
    for k, v in enumerate(x):
        if not np.isfinite(v):
            out[k] = 0 if np.isnan(v) or v < 0 else 0x3DF
            continue
        if v <= 0:
            continue
        d = np.abs(vals - v)
        best = np.nonzero(d == d.min())[0]
        c = codes[best]
        pick = c[c % 2 == 0] if len(c) > 1 else c
        out[k] = pick[0]
    return out


def test_uf10_exhaustive_over_fp16_inputs_against_nearest_code():
    bits, vals = _all_fp16_values()
    fin = np.isfinite(vals)
    want = _uf10_brute(vals)
    got = nu.uf10_code(vals).astype(np.int64)
    np.testing.assert_array_equal(got[fin], want[fin])
    # +inf clamps to the largest finite code, -inf and NaN give 0
    np.testing.assert_array_equal(nu.uf10_code(np.array([np.inf, -np.inf, np.nan])), [0x3DF, 0, 0])


def test_uf10_against_nearest_code_on_random_fp32_inputs():
    rng = np.random.default_rng(3)
    x = (rng.lognormal(-1.0, 3.0, 20000)).astype(np.float32).astype(np.float64)
    np.testing.assert_array_equal(nu.uf10_code(x).astype(np.int64), _uf10_brute(x))


def test_uf10_codes_round_trip_and_are_monotone():
    codes, vals = _uf10_table()
    np.testing.assert_array_equal(nu.uf10_value(codes), vals)
    np.testing.assert_array_equal(nu.uf10_code(vals), codes)
    assert np.all(np.diff(vals) > 0)
    x = np.sort(np.random.default_rng(4).lognormal(0.0, 4.0, 50000))
    assert np.all(np.diff(nu.uf10_code(x).astype(np.int64)) >= 0)
    assert nu.UF10_MAX == vals[-1] and nu.UF10_MAX_CODE == 0x3DF


def test_unorm10_against_exact_rational_rounding():
    """round(clamp(x,0,1)*1023) with exact rationals, ties to even, on float32 inputs."""
    from fractions import Fraction
    x = np.concatenate([np.linspace(-0.5, 1.5, 20001), (np.arange(1023) + 0.5) / 1023.0])
    x = x.astype(np.float32).astype(np.float64)
    want = []
    for v in x:
        q = Fraction(min(max(v, 0.0), 1.0)) * 1023
        fl = q.numerator // q.denominator
        frac = q - fl
        want.append(fl + (1 if frac > Fraction(1, 2) or (frac == Fraction(1, 2) and fl % 2 == 1) else 0))
    np.testing.assert_array_equal(nu.unorm10_code(x).astype(np.int64), np.array(want))


@pytest.mark.parametrize("fmt", ["f16", "f32", "f64"])
def test_round_state_is_idempotent(fmt):
    x = np.random.default_rng(5).lognormal(0, 2, 1000)
    r = nu.round_state(x, fmt)
    np.testing.assert_array_equal(nu.round_state(r, fmt), r)


def test_unorm10_binary32_values_are_single_rounded():
    """The GPU client stores UNORM10 values as the correctly rounded binary32 quotient
    code / 1023; the oracle's binary64 value rounded to binary32 must be that same number
    (no double-rounding case among the 1024 codes)."""
    from fractions import Fraction
    for code in range(1024):
        via64 = float(np.float32(code / 1023.0))
        exact = Fraction(code, 1023)
        f = np.float32(float(exact))
        lo, hi = np.nextafter(f, np.float32(-1)), np.nextafter(f, np.float32(2))
        best = min((lo, f, hi), key=lambda x: (abs(Fraction(float(x)) - exact), int(np.float32(x).view(np.uint32)) & 1))
        assert via64 == float(best), code
