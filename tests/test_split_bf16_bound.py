"""The error bound of the split-BF16 products (the tensor-core complex64 GEMM) pinned on
the host against exact arithmetic, independently of the device code.

Each FP32 operand is split as a_hi = bf16(a) (round to nearest, ties to even: BF16 keeps the
sign, the 8 exponent bits and the top 7 fraction bits of the FP32 word) and
a_lo = bf16(a - a_hi); the product is taken as a_hi b_hi + a_hi b_lo + a_lo b_hi.  Claimed:
|a b - (a_hi b_hi + a_hi b_lo + a_lo b_hi)| <= 3 * 2^-16 |a| |b| for every pair of normal
FP32 numbers (the bound the GPU tests of the product use, with the FP32 accumulation term
added).  Checked in FP64, where the three partial products of BF16 values are exact.
"""
import numpy as np


def bf16_rn(x):
    """Round float32 values to the nearest BF16 value (ties to even), returned as float32."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def split(a):
    hi = bf16_rn(a)
    lo = bf16_rn(a.astype(np.float32) - hi)  # the FP32 difference is exact (Sterbenz)
    return hi, lo


def test_bf16_rounding_is_exact_on_representable_values_and_halves_ulp():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(100000) * np.exp(rng.uniform(-20, 20, 100000))).astype(np.float32)
    h = bf16_rn(x)
    # a BF16 value is a float32 whose low 16 bits are zero, and rounding it is the identity
    assert np.all((h.view(np.uint32) & 0xFFFF) == 0)
    assert np.array_equal(bf16_rn(h), h)
    # nearest rounding: the error is at most half a BF16 ulp = 2^-8 of the value's binade
    e = np.abs(x.astype(np.float64) - h.astype(np.float64))
    assert np.all(e <= 2.0 ** -8 * np.abs(x.astype(np.float64)))


def test_split_product_error_is_within_three_times_two_to_the_minus_sixteen():
    rng = np.random.default_rng(1)
    n = 400000
    a = (rng.standard_normal(n) * np.exp(rng.uniform(-10, 10, n))).astype(np.float32)
    b = (rng.standard_normal(n) * np.exp(rng.uniform(-10, 10, n))).astype(np.float32)
    ah, al = split(a)
    bh, bl = split(b)
    A, B = a.astype(np.float64), b.astype(np.float64)
    approx = ah.astype(np.float64) * bh + ah.astype(np.float64) * bl + al.astype(np.float64) * bh
    err = np.abs(A * B - approx) / (np.abs(A) * np.abs(B))
    assert err.max() <= 3 * 2.0 ** -16, err.max()
    # and the bound is not loose by orders of magnitude: the dropped a_lo b_lo term alone
    # reaches a sizeable fraction of it
    assert err.max() >= 2.0 ** -18


def test_split_parts_reconstruct_the_operand_to_two_to_the_minus_sixteen():
    rng = np.random.default_rng(2)
    a = (rng.standard_normal(100000) * 10.0 ** rng.uniform(-5, 5, 100000)).astype(np.float32)
    hi, lo = split(a)
    rem = np.abs(a.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64))
    assert np.all(rem <= 2.0 ** -16 * np.abs(a.astype(np.float64)))
    assert np.all(np.abs(lo.astype(np.float64)) <= 2.0 ** -8 * np.abs(a.astype(np.float64)))
