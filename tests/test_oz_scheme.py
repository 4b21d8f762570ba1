"""CPU pins of the arithmetic of the FP64-accurate tensor-core pass
(csrc/tq_apply_oz.cu), emulated bit by bit in numpy: every FP64 operand's
significand aligned to the largest exponent of its group (inputs) or row
(superoperator), at least 64, rounded to nearest (54 bits), cut into seven
balanced 8-bit digits (the bytes of F + 0x0080808080808080, minus 128, signed
by one FP16 multiply-add), the digit products
summed exactly per order t = i + j (orders 0..7, each in its own FP32
accumulator), each accumulator turned into its integer by the 1.5 * 2^23
float addition (orders 6 and 7 rounded to units of 2^8 and 2^16), the
integers combined in wrapped 64-bit arithmetic and converted to FP64 with
integer operations only, the exponent placed directly. The exact reference is
the dot product in rational arithmetic. These pin the digit layout, the
orders, the magic constants and the scaling; the GPU tests hold the kernel
itself to the oracle."""
from fractions import Fraction

import numpy as np

MASK64 = (1 << 64) - 1
OFFSET = 0x0080808080808080


def fields(v: float):
    b = int(np.array([v], dtype=np.float64).view(np.uint64)[0])
    return b >> 63, (b >> 52) & 0x7FF, b & ((1 << 52) - 1)


def aligned_offset(v: float, E: int) -> int:
    """F + 0x0080808080808080 the kernel's way: M2 = the significand (implicit
    bit set) times 4, T = M2 >> (E - e_v) (0 for shifts of 64 or more),
    (T + 0x0101010101010101) >> 1."""
    _, ev, frac = fields(v)
    sh = E - ev
    M2 = ((1 << 52) | frac) << 2
    T = M2 >> sh if sh < 64 else 0
    out = (T + 0x0101010101010101) >> 1
    # the same as v's significand (times 2: 54 bits) aligned to E and
    # rounded to nearest, ties away from zero (zeros and subnormals: 0), plus
    # the offset
    M1 = 0 if ev == 0 else ((1 << 52) | frac) << 1
    F = int(Fraction(M1, 2 ** sh) + Fraction(1, 2)) if M1 else 0
    assert out == F + OFFSET and F < (1 << 54)
    return out


def fp16_digit(byte: int, neg: bool) -> float:
    """The kernel's FP16 arithmetic on one half: the byte placed in the low
    mantissa byte of FP16 1024, times s = -1 or +1, plus -1152 s (one
    multiply-add; every intermediate is exact in FP16)."""
    w = np.array([0x6400 | byte], dtype=np.uint16).view(np.float16)[0]
    s = np.float16(-1.0 if neg else 1.0)
    d = np.float16(np.float32(w) * np.float32(s) + np.float32(-1152.0) * np.float32(s))
    assert float(d) == (byte - 128) * (-1 if neg else 1)
    return float(d)


def digits7(v: float, E: int):
    """The seven digits of v (sign applied): integers in [-128, 128]."""
    sgn = fields(v)[0]
    Fp = aligned_offset(v, E)
    assert Fp >> 56 == 0                                   # the offset never carries out of byte 6
    return [fp16_digit((Fp >> (8 * (6 - i))) & 0xFF, bool(sgn)) for i in range(7)]


def max_exp(vals):
    """The alignment exponent: the largest biased exponent, at least 64."""
    return max(64, max(fields(float(v))[1] for v in vals))


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
    b = [magic_int(a, 0) for a in c[:6]] + [magic_int(c[6], -8), magic_int(c[7], -16)]
    Z = (((b[0] * 256 + b[1]) & 0xFFFFFFFF) << 32) & MASK64
    Z = (Z + b[2] * (1 << 24)) & MASK64
    Z = (Z + b[3] * (1 << 16)) & MASK64
    Z = (Z + b[4] * (1 << 8)) & MASK64
    Z = (Z + b[5] + b[6] + b[7]) & MASK64
    K = (sum(magic_bits(0) << (8 * s) for s in range(6)) + magic_bits(-8) + magic_bits(-16)) & MASK64
    return int_to_f64_scaled((Z - K) & MASK64, scale)


def oz_dot(x, R_row):
    """One real output: sum_k R_row[k] x[k] the kernel's way."""
    E, G = max_exp(x), max_exp(R_row)
    A = np.array([digits7(float(v), E) for v in x])      # [k][i]
    B = np.array([digits7(float(v), G) for v in R_row])  # [k][j]
    c = []
    for t in range(8):                                   # orders 0..7, each exact
        acc = 0.0
        for i in range(7):
            if 0 <= t - i < 7:
                acc += float(np.dot(A[:, i], B[:, t - i]))
        assert abs(acc) < 2 ** 22 and float(np.float32(acc)) == acc   # FP32 accumulation is exact
        c.append(np.float32(acc))
    return recombine(c, E + G - 2096), E, G


def exact_dot(x, r):
    return sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, r))


def align(E):
    return 2.0 ** (E - 1022)      # |v| < 2^(e_v - 1022) <= this for every value aligned to E


def test_digits_reassemble_the_rounded_value():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        v = float(rng.standard_normal() * 10.0 ** rng.uniform(-12, 2))
        E = fields(v)[1] + int(rng.integers(0, 20))
        d = digits7(v, E)
        back = sum(Fraction(int(t)) * 256 ** (6 - i) for i, t in enumerate(d)) * Fraction(2) ** (E - 1076)
        assert abs(back - Fraction(v)) <= Fraction(2) ** (E - 1076 - 1)   # half a unit of 2^(E-1076)
        assert all(abs(t) <= 128 and t == int(t) for t in d)              # integers, exact in FP16 (sign applied)
        assert abs(d[0]) <= 64                                           # F < 2^54: the top digit stays small


def test_exact_orders_stay_below_the_magic_range():
    # the largest digit magnitudes: every order's integer stays below 2^22,
    # where the 1.5 * 2^23 addition extracts it exactly
    for t in range(8):
        pairs = min(t + 1, 7, 14 - t)
        assert pairs * 32 * 128 * 128 < 2 ** 22
    x = np.full(32, np.nextafter(2.0, 0.0))
    r = -x
    y, _, _ = oz_dot(x, r)
    assert abs(Fraction(y) - exact_dot(x, r)) <= abs(exact_dot(x, r)) * Fraction(1, 2 ** 52)


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
    # 32 operand pairs, each rounded at 2^-55 of its alignment, dropped orders,
    # the rounding of orders 6 and 7 and one final rounding: below 2^-51 of
    # the product of the alignments (measured: ~2 x 2^-53)
    assert worst < 2.0 ** -51, worst / 2.0 ** -53


def test_tiny_groups_are_aligned_to_the_floor_exponent():
    # a group whose largest entry is below 2^-959 is aligned to 2^-959: the
    # result stays within 2^-51 of that alignment times the row's
    rng = np.random.default_rng(6)
    x = rng.standard_normal(32) * 1e-300
    r = rng.standard_normal(32)
    y, E, G = oz_dot(x, r)
    assert E == 64
    assert abs(Fraction(y) - exact_dot(x, r)) < Fraction(align(E) * align(G)) * Fraction(1, 2 ** 51)


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
        assert abs(Fraction(got) - want) <= abs(want) * Fraction(1, 2 ** 53)   # half an ulp of the result
    assert int_to_f64_scaled(0, 5) == 0.0
    assert int_to_f64_scaled((1 << 53) + 1, 0) == float((1 << 53) + 2)   # a tie rounds away from zero
    assert int_to_f64_scaled((-(1 << 53) - 1) & MASK64, 0) == -float((1 << 53) + 2)
    assert int_to_f64_scaled(1, -1075) == 0.0                             # below the normal range
