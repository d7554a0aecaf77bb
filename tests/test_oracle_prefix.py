"""Pins of the fixed summation order of the resampling weights.

Sec. II.B needs the normalisation S = sum_i w_i and, for the multinomial draws,
cumulative weights P_i to search.  The oracle sums in a fixed hierarchical
order (runs of 32 summed left to right, recursively over the run totals) and
takes a running maximum so that P never decreases.  These tests pin it to
what does not depend on the order:
  * on inputs whose partial sums are exact in FP64 (small integers, dyadic
    fractions) every order gives the exact prefix, for lengths across several
    levels and ragged runs;
  * up to 32 entries the order is the plain left-to-right sum;
  * P is non-decreasing, equals the running maximum of the raw prefix, and
    its last entry is within the error bound of a sum of that depth of the
    correctly rounded total (math.fsum).
"""
import math

import numpy as np
import pytest


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 64, 65, 1000, 1024, 1025, 32 * 32 * 32 + 17, 70001])
def test_exact_inputs_give_the_exact_prefix(oracle, n):
    rng = np.random.default_rng(n)
    k = rng.integers(0, 1000, n)
    P, pre = oracle.weight_prefix(k.astype(np.float64))
    want = np.cumsum(k).astype(np.float64)  # integers below 2^53: exact
    np.testing.assert_array_equal(P, want)
    np.testing.assert_array_equal(pre, want)
    d = rng.integers(0, 1 << 20, n).astype(np.float64) * 2.0 ** -30  # dyadic, exact partial sums
    P, _ = oracle.weight_prefix(d)
    np.testing.assert_array_equal(P, np.cumsum(d))


@pytest.mark.parametrize("n", [1, 5, 32])
def test_short_inputs_are_summed_left_to_right(oracle, n):
    rng = np.random.default_rng(100 + n)
    w = np.exp(-rng.uniform(0, 30, n))
    P, pre = oracle.weight_prefix(w)
    acc, want = 0.0, []
    for j, v in enumerate(w):
        acc = float(v) if j == 0 else acc + float(v)
        want.append(acc)
    np.testing.assert_array_equal(pre, want)
    np.testing.assert_array_equal(P, want)


@pytest.mark.parametrize("n,scale", [(5000, 1.0), (33 * 33 * 33, 40.0), (100000, 700.0)])
def test_monotone_running_maximum_and_error_bound(oracle, n, scale):
    rng = np.random.default_rng(n)
    w = np.exp(-rng.uniform(0, scale, n))  # weights in (0, 1], many orders of magnitude
    w[rng.integers(0, n, n // 50)] = 0.0   # dead replicas
    P, pre = oracle.weight_prefix(w)
    assert np.all(np.diff(P) >= 0)
    np.testing.assert_array_equal(P, np.maximum.accumulate(pre))
    depth = 1
    m = n
    while m > 32:
        m = (m + 31) // 32
        depth += 1
    # every partial sum takes at most 32 additions per level of the hierarchy
    eps = 2.0 ** -53
    bound = 32 * depth * eps * math.fsum(w) * (1 + 1e-6)
    assert abs(P[-1] - math.fsum(w)) <= bound
    # every raw prefix is within the same bound of the exact partial sum (extended-precision
    # reference, whose own error n 2^-63 sum w is added to the bound)
    ref = np.cumsum(w.astype(np.longdouble))
    err = np.abs(pre.astype(np.longdouble) - ref)
    assert np.all(err <= 32 * depth * eps * ref * (1 + 1e-6) + n * 2.0 ** -63 * math.fsum(w))
