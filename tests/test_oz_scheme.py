"""CPU pins of the arithmetic of the FP64-accurate tensor-core pass
(csrc/tq_apply_oz.cu), emulated bit by bit in numpy: every FP64 operand cut
into eight 7-bit digits of a 56-bit fixed-point number aligned to the largest
exponent of its group (inputs) or row (superoperator), the digit products
summed exactly per order t = i + j (orders 0..7, each in its own FP32
accumulator), each accumulator turned into its integer by the
1.5 * 2^(23 - u) float addition (order 7 rounded to units of 2^-42), the
integers combined in wrapped 64-bit arithmetic and converted to FP64 with
integer operations only, the exponent placed directly. The exact reference is the dot product in rational arithmetic. These
pin the digit layout, the orders, the magic constants and the scaling; the GPU
tests hold the kernel itself to the oracle."""
from fractions import Fraction

import numpy as np

MASK64 = (1 << 64) - 1


def fields(v: float):
    b = int(np.array([v], dtype=np.float64).view(np.uint64)[0])
    return b >> 63, (b >> 52) & 0x7FF, b & ((1 << 52) - 1)


def digits8(v: float, E: int):
    """The kernel's digits: +-d_i 2^(-7 i) as float32, d_i = 7-bit digit i of
    F, the significand aligned to biased exponent E and rounded to nearest."""
    sgn, ev, frac = fields(v)
    sh = E - ev
    M3 = ((1 << 52) | frac) << 3
    if ev == 0 or sh > 56:
        F = 0
    elif sh == 0:
        F = M3
    else:
        F = ((M3 >> (sh - 1)) + 1) >> 1
    assert F < (1 << 56)
    out = []
    for i in range(8):
        d = (F >> (49 - 7 * i)) & 0x7F
        out.append(np.float32((-1.0 if sgn else 1.0) * d * 2.0 ** (-7 * i)))
    return out


def max_exp(vals):
    return max(fields(float(v))[1] for v in vals)


def magic_bits(u):
    return ((150 - u) << 23) | 0x400000


def magic_int(a, u):
    """The float32 bit pattern of a + 1.5 * 2^(23 - u) (one float32 addition)."""
    f = np.float32(np.float32(a) + np.array([magic_bits(u)], dtype=np.uint32).view(np.float32)[0])
    return int(np.array([f], dtype=np.float32).view(np.uint32)[0])


def int_to_f64_scaled(Z, scale):
    """The kernel's integer-only conversion of a two's-complement 64-bit Z to
    FP64 times 2^scale: normalise |Z|, round to 53 bits (ties away from
    zero), place the exponent 1086 - lz + scale; 0 for Z = 0 or below the
    normal range."""
    Zs = Z - (1 << 64) if Z >> 63 else Z
    if Zs == 0:
        return 0.0
    a = abs(Zs)
    lz = 64 - a.bit_length()
    a = (a << lz) & MASK64
    mant = (a >> 11) + ((a >> 10) & 1)
    eb = 1085 - lz + scale
    if eb < 0:
        return 0.0
    b = ((1 << 63) if Zs < 0 else 0) + (eb << 52) + mant
    return float(np.array([b], dtype=np.uint64).view(np.float64)[0])


def recombine(c, scale):
    """c: 8 float32 accumulator values, orders 0..7."""
    b = [magic_int(a, u) for a, u in zip(c[:7], (0, 7, 14, 21, 28, 35, 42))]
    b.append(magic_int(c[7], 42))                        # order 7 rounded to units of 2^-42
    Z = (((b[0] * 128 + b[1]) & 0xFFFFFFFF) << 35) & MASK64
    Z = (Z + b[2] * (1 << 28)) & MASK64
    Z = (Z + b[3] * (1 << 21)) & MASK64
    Z = (Z + b[4] * (1 << 14)) & MASK64
    Z = (Z + b[5] * (1 << 7)) & MASK64
    Z = (Z + b[6] + b[7]) & MASK64
    K = ((magic_bits(0) << 42) + (magic_bits(7) << 35) + (magic_bits(14) << 28) + (magic_bits(21) << 21)
         + (magic_bits(28) << 14) + (magic_bits(35) << 7) + 2 * magic_bits(42)) & MASK64
    return int_to_f64_scaled((Z - K) & MASK64, scale)


def oz_dot(x, R_row):
    """One real output: sum_k R_row[k] x[k] the kernel's way."""
    E, G = max_exp(x), max_exp(R_row)
    A = np.array([digits8(float(v), E) for v in x])      # [k][i]
    B = np.array([digits8(float(v), G) for v in R_row])  # [k][j]
    c = []
    for t in range(8):                                   # every order exact (summed in float64, exact here)
        acc = 0.0
        for i in range(t + 1):
            acc += float(np.dot(A[:, i].astype(np.float64), B[:, t - i].astype(np.float64)))
        assert float(np.float32(acc)) == acc             # representable: FP32 accumulation is exact
        c.append(np.float32(acc))
    return recombine(c, E + G - 2100), E, G


def exact_dot(x, r):
    return sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, r))


def align(E):
    return 2.0 ** (E - 1022)      # |v| < 2^(e_v - 1022) <= this for every value aligned to E


def test_digits_reassemble_the_rounded_value():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        v = float(rng.standard_normal() * 10.0 ** rng.uniform(-12, 2))
        E = fields(v)[1] + int(rng.integers(0, 20))
        d = digits8(v, E)
        back = sum(Fraction(float(t)) for t in d) * Fraction(2) ** (E - 1078 + 49)
        assert abs(back - Fraction(v)) <= Fraction(2) ** (E - 1078 - 1)   # half a unit of 2^(E-1078)
        for i, t in enumerate(d):
            q = abs(float(t)) * 2.0 ** (7 * i)
            assert q == int(q) and q < 128                                 # a 7-bit digit, exact in BF16


def test_exact_orders_stay_below_the_magic_range():
    # worst case: every digit 127 (all values at the top of the alignment)
    x = np.full(32, np.nextafter(2.0, 0.0))
    d = digits8(float(x[0]), fields(float(x[0]))[1])
    # a 53-bit significand shifted by 3: the last digit keeps 4 bits
    assert [round(abs(float(t)) * 2.0 ** (7 * i)) for i, t in enumerate(d)] == [127] * 7 + [120]
    for t in range(8):
        assert (t + 1) * 32 * 127 * 127 < 2 ** 22


def test_recombined_dot_products_are_fp64_accurate():
    rng = np.random.default_rng(2)
    worst = 0.0
    for trial in range(300):
        scale_x = 10.0 ** rng.uniform(-6, 0)
        x = rng.standard_normal(32) * scale_x * 10.0 ** rng.uniform(-3, 0, 32)
        x[rng.integers(0, 32, 4)] = 0.0                   # exact zeros occur in density matrices
        r = rng.standard_normal(32) * 10.0 ** rng.uniform(-2, 0, 32)
        if trial % 5 == 0:
            r[rng.integers(0, 32, 20)] = 0.0              # structured superoperator rows
        y, E, G = oz_dot(x, r)
        err = abs(Fraction(y) - exact_dot(x, r))
        worst = max(worst, float(err) / (align(E) * align(G)))
    # 32 operand pairs, each rounded at 2^-57 of its alignment, dropped orders
    # and one final rounding: below 2^-51 of the product of the alignments
    assert worst < 2.0 ** -51, worst / 2.0 ** -53


def test_zero_rows_and_groups_give_exact_zeros():
    x = np.zeros(32)
    r = np.random.default_rng(3).standard_normal(32)
    assert oz_dot(x, r)[0] == 0.0
    assert oz_dot(r, np.zeros(32))[0] == 0.0


def test_signs_and_an_identity_row():
    rng = np.random.default_rng(4)
    x = rng.standard_normal(32)
    for k in (0, 5, 31):
        e = np.zeros(32)
        e[k] = 1.0
        y, _, _ = oz_dot(x, e)
        assert abs(y - x[k]) <= 2.0 ** -52 * align(max_exp(x))   # the identity reproduces the entry
        e[k] = -1.0
        y, _, _ = oz_dot(x, e)
        assert abs(y + x[k]) <= 2.0 ** -52 * align(max_exp(x))


def test_integer_conversion_rounds_to_nearest():
    rng = np.random.default_rng(5)
    for _ in range(5000):
        z = int(rng.integers(-(1 << 62), 1 << 62))
        s = int(rng.integers(-60, 60))
        got = int_to_f64_scaled(z & MASK64, s)
        want = Fraction(z) * Fraction(2) ** s
        # within half a unit in the last place of the result
        assert abs(Fraction(got) - want) <= abs(want) * Fraction(1, 2 ** 53)
    assert int_to_f64_scaled(0, 5) == 0.0
    assert int_to_f64_scaled((1 << 53) + 1, 0) == float((1 << 53) + 2)   # a tie rounds away from zero
    assert int_to_f64_scaled((-(1 << 53) - 1) & MASK64, 0) == -float((1 << 53) + 2)
    assert int_to_f64_scaled(1, -1075) == 0.0                             # below the normal range
