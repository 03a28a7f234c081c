"""The arithmetic behind the exact Gram in base-64 digits, checked on the host.

The FP32 paths sum G = C C^H exactly: C^H's columns are scaled to integers
|q| <= 2^23, and on the tensor cores every integer is split into four signed
base-64 digits whose products are summed in FP32.  Two facts make that exact:
the digits reproduce the integers, and a sum of n2 <= 4096 digit products
(|d| <= 63) stays below 2^24, so FP32 accumulation in any order adds exact
integers.  These tests check both with an FP32 BLAS product (whose summation
order is not ours) against the integer Gram, including the worst case of
every digit at 63.
"""
import numpy as np
import pytest

DIGITS, DBITS = 4, 6


def digits(q):
    """Signed base-64 digits of integers |q| < 2^24: q = sum_s d_s 64^(3-s)."""
    mag, sgn = np.abs(q), np.sign(q)
    return [sgn * ((mag >> (DBITS * (DIGITS - 1 - s))) & 63) for s in range(DIGITS)]


def deinterleave(re, im):
    """(n2 x m) real and imaginary parts -> rows 2i (real) and 2i+1 (imaginary) of length n2."""
    n2, m = re.shape
    D = np.empty((2 * m, n2), dtype=re.dtype)
    D[0::2] = re.T
    D[1::2] = im.T
    return D


def gram_exact(re, im):
    """sum_l conj(q_li) q_lj in 64-bit integers."""
    a, b = re.astype(np.int64), im.astype(np.int64)
    return a.T @ a + b.T @ b, a.T @ b - b.T @ a


def gram_digits(re, im):
    """The same from FP32 products of the de-interleaved digit rows, pairs combined in int64."""
    m = re.shape[1]
    dre, dim = digits(re), digits(im)
    Ds = [deinterleave(dre[s], dim[s]).astype(np.float32) for s in range(DIGITS)]
    gre = np.zeros((m, m), dtype=np.int64)
    gim = np.zeros((m, m), dtype=np.int64)
    for s in range(DIGITS):
        for t in range(DIGITS):
            P = Ds[s] @ Ds[t].T  # FP32 accumulation, BLAS order
            Pi = P.astype(np.int64)
            assert np.array_equal(Pi.astype(np.float32), P)  # every entry an integer
            w = np.int64(1) << (DBITS * (2 * DIGITS - 2 - s - t))
            gre += (Pi[0::2, 0::2] + Pi[1::2, 1::2]) * w
            gim += (Pi[0::2, 1::2] - Pi[1::2, 0::2]) * w
    return gre, gim


def test_digits_reproduce_the_integers():
    rng = np.random.default_rng(1)
    q = rng.integers(-(1 << 23), (1 << 23) + 1, size=10000)
    q[:4] = [0, 1 << 23, -(1 << 23), (1 << 24) - 1]
    d = digits(q)
    assert all(np.abs(x).max() <= 63 for x in d)
    back = sum(d[s] * (64 ** (DIGITS - 1 - s)) for s in range(DIGITS))
    np.testing.assert_array_equal(back, q)


def test_worst_case_digit_sums_stay_below_two_to_24():
    n2 = 4096
    assert n2 * 63 * 63 < (1 << 24)
    a = np.full((1, n2), 63.0, dtype=np.float32)
    assert (a @ a.T)[0, 0] == n2 * 63 * 63


@pytest.mark.parametrize("n2,m,seed", [(4096, 12, 0), (2048, 20, 1), (129, 7, 2)])
def test_digit_gram_equals_integer_gram(n2, m, seed):
    rng = np.random.default_rng(seed)
    re = rng.integers(-(1 << 23), (1 << 23) + 1, size=(n2, m))
    im = rng.integers(-(1 << 23), (1 << 23) + 1, size=(n2, m))
    re[:, 0] = (1 << 23) - 1  # a column of the largest magnitudes (digits 31, 63, 63, 63)
    im[:, 0] = -((1 << 23) - 1)
    er, ei = gram_exact(re, im)
    dr, di = gram_digits(re, im)
    np.testing.assert_array_equal(dr, er)
    np.testing.assert_array_equal(di, ei)
