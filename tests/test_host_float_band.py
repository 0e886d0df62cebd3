"""The real-X verification sums Y'_i X'_ij X'_ik first in float and sends a
candidate to the double sum when its float sum lies within
(n + 64) 2^-23 ||Y'||_1 of the threshold.  That is safe when the float sum
is never farther than the band from the exact sum.  This models the
kernel's float summation on the host -- eight lanes, lane l adding the
terms of the pieces q = l, l + 8, ... (four terms per 16-byte piece) with
fused multiply-adds of Y' rounded to float and the rounded float product
X'_ij X'_ik, then a three-level shuffle tree -- and checks the error
against the exact (double) sum, with |X'| <= 1 as the row scaling makes it,
for random data and for data built to make the rounding errors add up.
"""
import numpy as np
import pytest


def f32(x):
    return np.float32(x)


def kernel_float_sum(y, a, b):
    """Float sum in the kernel's order: fmaf(y, a*b, part) per term."""
    n = len(y)
    nq = n // 4
    parts = []
    for lane in range(8):
        part = np.float32(0.0)
        for q in range(lane, nq, 8):
            for c in range(4):
                i = 4 * q + c
                prod = f32(np.float32(a[i]) * np.float32(b[i]))
                # fused multiply-add: one rounding of y * prod + part
                part = f32(float(np.float32(y[i])) * float(prod) + float(part))
        parts.append(part)
    # shuffle tree: xor 4, 2, 1
    for o in (4, 2, 1):
        parts = [f32(parts[l] + parts[l ^ o]) for l in range(8)]
    return float(parts[0])


def exact_sum(y, a, b):
    return float(np.sum(np.asarray(y, np.float64) * (np.asarray(a, np.float64) * np.asarray(b, np.float64))))


def band(y):
    return (len(y) + 64) * 2.0 ** -23 * float(np.sum(np.abs(y)))


@pytest.mark.parametrize("n,seed", [(64, 1), (512, 2), (2000, 3), (4096, 4)])
def test_float_sum_within_band_random(n, seed):
    rng = np.random.default_rng(seed)
    for _ in range(20):
        a = rng.uniform(-1, 1, n).astype(np.float32)
        b = rng.uniform(-1, 1, n).astype(np.float32)
        y = rng.standard_normal(n) * rng.uniform(0.1, 10.0, n)
        err = abs(kernel_float_sum(y, a, b) - exact_sum(y, a, b))
        # the analysis gives (n/8 + 6) 2^-24 ||Y'||_1; the kernel's band is
        # eight times that and more
        assert err <= (n / 8 + 6) * 2.0 ** -24 * float(np.sum(np.abs(y)))
        assert err <= band(y)


@pytest.mark.parametrize("n", [256, 2000])
def test_float_sum_within_band_adversarial(n):
    # every term of the same sign and near its largest magnitude, with
    # values chosen to round poorly: the errors add up rather than cancel
    rng = np.random.default_rng(n)
    for _ in range(5):
        a = (1.0 - rng.uniform(0, 2.0 ** -20, n)).astype(np.float32)
        b = (1.0 - rng.uniform(0, 2.0 ** -20, n)).astype(np.float32)
        y = 1.0 + rng.uniform(0, 1e-3, n) + 1.0 / 3.0
        err = abs(kernel_float_sum(y, a, b) - exact_sum(y, a, b))
        assert err <= (n / 8 + 6) * 2.0 ** -24 * float(np.sum(np.abs(y)))
        assert err <= band(y)
