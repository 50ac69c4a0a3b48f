"""The split arithmetic the tensor-core kernels rely on, emulated on the CPU with
numpy's IEEE half precision: a value x carried as hi + lo with hi = fp16(x) and
lo = fp16(x - hi) holds x to about 2^-22 relative when |x| sits in FP16's normal
range with room for lo, and the product a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi
(three MMAs, FP32 accumulation) then stays within a few 2^-22 of the exact product.
A single FP16 term (2^-11) or the TF32 two-term split with one MMA would not meet
the 1e-4 / 1e-5 parity tolerances; the split-TF32 scheme gets about 2^-21."""
import numpy as np

RS = np.random.default_rng(31)


def split16(x):
    hi = x.astype(np.float16)
    lo = (x - hi.astype(np.float64)).astype(np.float16)
    return hi.astype(np.float64), lo.astype(np.float64)


def tf32(x):
    """Round to nearest, ties away, to 10 explicit mantissa bits (the TF32 format)."""
    m, e = np.frexp(x)
    return np.ldexp(np.sign(m) * np.floor(np.abs(m) * 2 ** 11 + 0.5) / 2 ** 11, e)


def split32(x):
    hi = tf32(x)
    return hi, tf32(x - hi)


def test_fp16_split_holds_22_bits_in_the_scaled_range():
    # the kernels scale every operand into [2^-3, 1) (row maxima in [1/2, 1))
    x = RS.uniform(0.125, 1.0, 200000) * RS.choice([-1, 1], 200000)
    hi, lo = split16(x)
    rel = np.abs(x - (hi + lo)) / np.abs(x)
    assert rel.max() < 2.0 ** -21
    assert (np.abs(x - hi) / np.abs(x)).max() > 2.0 ** -13  # one term alone: ~2^-12


def test_fp16_split_error_is_absolute_below_the_range():
    # small entries of a scaled row lose relative bits but keep the absolute error
    # under 2^-24 of the row maximum (1): what the residual and update see
    x = RS.uniform(-1e-4, 1e-4, 100000)
    hi, lo = split16(x)
    assert np.abs(x - (hi + lo)).max() <= 2.0 ** -24


def test_three_term_product_fp16_and_tf32():
    a = RS.uniform(0.125, 1.0, 100000) * RS.choice([-1, 1], 100000)
    b = RS.uniform(0.125, 1.0, 100000) * RS.choice([-1, 1], 100000)
    exact = a * b
    for split, bound in ((split16, 2.0 ** -20), (split32, 2.0 ** -19)):
        ah, al = split(a)
        bh, bl = split(b)
        # FP32 accumulation of the three terms, lo terms first as in the kernels
        acc = (np.float32(ah * bl) + np.float32(al * bh)).astype(np.float32)
        acc = (acc + np.float32(ah * bh)).astype(np.float32)
        rel = np.abs(acc - exact) / np.abs(exact)
        assert rel.max() < bound, (split.__name__, rel.max())
    # one MMA on single-term operands is far outside the parity tolerances
    assert (np.abs(split16(a)[0] * split16(b)[0] - exact) / np.abs(exact)).max() > 1e-4
