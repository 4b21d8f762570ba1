"""CPU pins of the arithmetic the split-precision tensor-core pass uses
(csrc/tq_tc.cuh), emulated in numpy: a width-2 superoperator S real-ified
with entries interleaved (Re, Im) into a 32 x 32 matrix R, the identity
taken out, every FP32 operand split into three BF16 terms (round to nearest
even), and the six term products with orders i + j <= 2 summed. These pin
the layout and signs of R and the accuracy the scheme can reach; the GPU
tests hold the kernel itself to the oracle."""
import numpy as np


def bf16_rn(x):
    """Round float32 values to bfloat16 (round to nearest, ties to even),
    returned as float32."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return rounded.astype(np.uint32).view(np.float32)


def split3(x):
    x = np.asarray(x, dtype=np.float32)
    t0 = bf16_rn(x)
    r = (x - t0).astype(np.float32)
    t1 = bf16_rn(r)
    r = (r - t1).astype(np.float32)
    t2 = bf16_rn(r)
    return t0, t1, t2


def realify(S):
    """R[n][k] with n = 2o + (0: Re, 1: Im) of output o and k = 2l + (0: Re,
    1: Im) of input l, so that y = S x is R applied to the interleaved x."""
    D = S.shape[0]
    R = np.zeros((2 * D, 2 * D))
    R[0::2, 0::2] = S.real
    R[0::2, 1::2] = -S.imag
    R[1::2, 0::2] = S.imag
    R[1::2, 1::2] = S.real
    return R


def interleave(x):
    v = np.empty(2 * x.shape[-1])
    v[0::2], v[1::2] = x.real, x.imag
    return v


def random_superop(rng):
    # a CPTP width-2 superoperator: sum_i conj(K_i) (x) K_i of a random Kraus set
    G = rng.standard_normal((3, 4, 4)) + 1j * rng.standard_normal((3, 4, 4))
    M = sum(g.conj().T @ g for g in G)
    w, V = np.linalg.eigh(M)
    Ks = [g @ V @ np.diag(w ** -0.5) @ V.conj().T for g in G]
    return sum(np.kron(K.conj(), K) for K in Ks)


def test_realified_product_equals_the_complex_one():
    rng = np.random.default_rng(1)
    S = random_superop(rng)
    x = rng.standard_normal(16) + 1j * rng.standard_normal(16)
    assert np.allclose(realify(S) @ interleave(x), interleave(S @ x), atol=1e-12)
    # with the identity taken out, y = x + (R - I) x
    R = realify(S)
    assert np.allclose(interleave(x) + (R - np.eye(32)) @ interleave(x), interleave(S @ x), atol=1e-12)


def test_three_bf16_terms_represent_fp32_to_2_pow_minus_24():
    rng = np.random.default_rng(2)
    x = (rng.standard_normal(200000) * 10.0 ** rng.uniform(-8, 2, 200000)).astype(np.float32)
    t0, t1, t2 = split3(x)
    for t in (t0, t1, t2):
        assert np.array_equal(t, bf16_rn(t))        # each term is a BF16 value
    err = np.abs(x.astype(np.float64) - (t0.astype(np.float64) + t1 + t2))
    assert np.all(err <= 2.0 ** -24 * np.abs(x.astype(np.float64)))
    # terms shrink by >= 2^8 each (so dropping t_i t_j with i + j > 2 loses ~2^-24)
    nz = t1 != 0
    assert np.all(np.abs(t1[nz]) <= 2.0 ** -8 * np.abs(t0[nz]))


def test_six_term_products_reach_fp32_accuracy_on_a_density_matrix_group():
    # emulates the kernel's order of rounding: twelve MMAs (six term
    # products x two K-halves of 16, smallest first), each adding its
    # 16-term dot product to an FP32 accumulator (one FP32 rounding per MMA),
    # then the FP32 add y = x + D on the CUDA cores
    rng = np.random.default_rng(3)
    worst = 0.0
    for trial in range(50):
        S = random_superop(rng)
        E = (realify(S) - np.eye(32)).astype(np.float32)
        x = interleave((rng.standard_normal(16) + 1j * rng.standard_normal(16)) / 64).astype(np.float32)
        a, b = split3(x), split3(E)
        d = np.zeros(32, dtype=np.float32)
        for i, j in ((2, 0), (1, 1), (0, 2), (1, 0), (0, 1), (0, 0)):   # the kept products, smallest first
            for kh in (slice(0, 16), slice(16, 32)):
                part = b[j][:, kh].astype(np.float64) @ a[i][kh].astype(np.float64)
                d = (d.astype(np.float64) + part).astype(np.float32)
        y = (x + d).astype(np.float64)                                  # FP32 add, rounded to nearest
        exact = x.astype(np.float64) + E.astype(np.float64) @ x.astype(np.float64)
        scale = np.abs(E.astype(np.float64)) @ np.abs(x.astype(np.float64)) + np.abs(x)
        worst = max(worst, float(np.max(np.abs(y - exact) / scale)))
    # the final FP32 rounding (half a unit of 2^-23 of |y|), the
    # accumulator's roundings of the smaller change and the dropped products
    # stay below one unit of 2^-23 of the scale (measured: 0.72 x 2^-24)
    assert worst < 2.0 ** -23, worst
