"""The arithmetic of the emulated-FP64 products (HTS_GEMM_EMU_BF16), checked against exact
rational arithmetic on the CPU.

Model (what the GPU kernels compute, restated from the mathematics):
- a line window a (up to 32 FP64 values) is written as integers x_k = round(a_k 2^-ua) with
  ua = e + 2 - 64, where 2^e is the smallest power of two above max |a_k|, so |x_k| < 2^62;
- U (entries in [-1, 1]) as y = round(u 2^61);
- each integer is split into 8 balanced base-256 digits d_1..d_8 in [-128, 127] (the bytes of
  x + 0x8080808080808080 minus 128), x = sum d_i 256^(8-i);
- level L = i + t collects the digit products d_i(x) d_t(y) over the window; levels 2..9 are
  kept, each must stay below 2^22 in magnitude (exact in an FP32 accumulator);
- the result in units 2^(ua+3) is sum_{L<=8} C_L 2^(8(8-L)) + floor((C_9 + 128) / 256).

The tests pin:
- the digit decomposition is exact and bounded;
- the level sums stay below 2^22 in the worst case the digit bounds allow;
- the result is within 2^(e-55) of the exact product. The main contributions are U's rounding
  (at most 2^-62 times sum |a_k|) and the dropped levels, which is well below one FP64 rounding
  unit of the window's largest entry. This is checked for windows of mixed magnitudes times
  the columns of an orthogonal matrix.
"""
from fractions import Fraction

import numpy as np
import pytest

OFFSET = 0x8080808080808080
UNIT_U = -61


def balanced_digits(x):
    u = (x + OFFSET) & ((1 << 64) - 1)
    return [((u >> (8 * (8 - i))) & 0xFF) - 128 for i in range(1, 9)]


def to_fixed(v, unit):
    """round(v 2^-unit), ties away from zero as the kernel's add-half-then-shift does for the
    magnitude (the value is exact in Fraction)."""
    q = Fraction(v) / Fraction(2) ** unit
    s = -1 if q < 0 else 1
    return s * int(abs(q) + Fraction(1, 2))


def exponent_above(vals):
    m = max(abs(float(v)) for v in vals)
    if m == 0.0:
        return None
    return int(np.frexp(m)[1])          # m < 2^e, e = floor(log2 m) + 1


def emulated_dot_units(a, u):
    """Returns (result integer in units 2^(ua+3), ua, level sums C_2..C_9)."""
    e = exponent_above(a)
    ua = (0 if e is None else e + 2) - 64
    xa = [to_fixed(v, ua) for v in a]
    xu = [to_fixed(v, UNIT_U) for v in u]
    assert all(abs(x) < 2 ** 62 for x in xa)
    da = np.array([balanced_digits(x) for x in xa], dtype=np.int64)   # [k][i]
    du = np.array([balanced_digits(y) for y in xu], dtype=np.int64)
    C = {}
    for L in range(2, 10):
        s = 0
        for i in range(1, 9):
            t = L - i
            if 1 <= t <= 8:
                s += int(np.dot(da[:, i - 1], du[:, t - 1]))
        C[L] = s
    val = sum(C[L] << (8 * (8 - L)) for L in range(2, 9)) + ((C[9] + 128) >> 8)
    return val, ua, C


def test_balanced_digits_are_exact_and_bounded():
    rng = np.random.default_rng(1)
    samples = [0, 1, -1, 2 ** 62 - 1, -(2 ** 62 - 1), 0x7F7F7F7F7F7F7F, -0x7F7F7F7F7F7F7F]
    samples += [int(v) for v in rng.integers(-2 ** 62 + 1, 2 ** 62 - 1, size=2000, dtype=np.int64)]
    for x in samples:
        d = balanced_digits(x)
        assert all(-128 <= v <= 127 for v in d)
        assert sum(v * 256 ** (8 - i) for i, v in enumerate(d, start=1)) == x
        # |x| < 2^62 bounds the leading digit by 64 (and by 32 for |x| <= 2^61)
        assert abs(d[0]) <= 64
    assert abs(balanced_digits(2 ** 61)[0]) <= 32


def test_digits_are_exact_in_bf16():
    # every digit value is an integer with at most 8 significant bits: its FP32 encoding has
    # 16 trailing zero bits, so the BF16 truncation is exact
    for v in range(-128, 128):
        bits = np.array([v], dtype=np.float32).view(np.uint32)[0]
        assert bits & 0xFFFF == 0


def test_level_sums_stay_below_2_22_in_the_worst_case():
    # worst case the digit bounds allow: 32 window positions, leading digits 64 (data) and
    # 32 (U), all other digits of magnitude 128, every product of the same sign
    K = 32
    bound = {}
    for L in range(2, 10):
        s = 0
        for i in range(1, 9):
            t = L - i
            if 1 <= t <= 8:
                di = 64 if i == 1 else 128
                dt = 32 if t == 1 else 128
                s += K * di * dt
        bound[L] = s
    assert max(bound.values()) < 2 ** 22, bound


def _haar(n, rng):
    q, r = np.linalg.qr(rng.standard_normal((n, n)))
    return q * np.sign(np.diag(r))


@pytest.mark.parametrize("spread", [0, 20, 40])
def test_emulated_product_error_bound(spread):
    """Windows of 31 values over 2^+-spread times the columns of a 31 x 31 orthogonal matrix:
    |result - exact| <= 2^(e - 55), where 2^e bounds the window; the typical error is near
    2^(e - 58)."""
    rng = np.random.default_rng(7 + spread)
    U = _haar(31, rng)
    worst = 0.0
    for trial in range(40):
        a = rng.standard_normal(31) * 2.0 ** rng.uniform(-spread, spread, 31)
        e = exponent_above(a)
        for col in range(0, 31, 5):
            val, ua, C = emulated_dot_units(a, U[:, col])
            assert all(abs(c) < 2 ** 22 for c in C.values())
            got = Fraction(val) * Fraction(2) ** (ua + 3)
            exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, U[:, col]))
            err = abs(got - exact) / Fraction(2) ** e
            worst = max(worst, float(err))
            assert err <= Fraction(1, 2 ** 55), (trial, col, float(err))
    assert worst > 0.0


def test_all_zero_and_single_entry_windows():
    U = np.eye(31)
    val, ua, C = emulated_dot_units([0.0] * 31, U[:, 3])
    assert val == 0 and all(c == 0 for c in C.values())
    a = [0.0] * 31
    a[3] = -1.2345678901234567e-200
    val, ua, C = emulated_dot_units(a, U[:, 3])
    assert Fraction(val) * Fraction(2) ** (ua + 3) == Fraction(a[3])
