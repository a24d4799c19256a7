"""Pins for the oracle's sum and dotproduct intrinsics (arXiv 2409.18824 Sec.
5.3-5.4, Table 3).  No GPU.

Checked against exact arithmetic: integer-valued data whose sums are exactly
representable (so any order gives the same bits), closed forms, Python's
correctly rounded math.fsum with the textbook error bound of recursive
summation, |computed - exact| <= (n - 1) u sum|x_i| (u = 2^-53), and a
library routine (numpy.dot).
"""
import math

import numpy as np
import pytest

import oracle
import stencil_inputs as si

U = 2.0 ** -53


def test_sum_closed_forms():
    n = 1_000_001
    x = np.arange(n, dtype=np.float64)
    assert oracle.sum_(x) == n * (n - 1) / 2          # exact below 2^53
    assert oracle.sum_(np.full(12345, 0.5)) == 6172.5
    assert oracle.sum_(np.zeros(0)) == 0.0
    assert oracle.sum_(np.array([-3.25])) == -3.25


def test_dot_closed_forms():
    n = 100_000
    i = np.arange(n, dtype=np.float64)
    assert oracle.dot(i, i) == (n - 1) * n * (2 * n - 1) / 6  # sum of squares, exact
    x = si.rng(3).random(777)
    assert oracle.dot(x, np.ones(777)) == oracle.sum_(x)
    assert oracle.dot(np.zeros(0), np.zeros(0)) == 0.0


@pytest.mark.parametrize("n", [1, 17, 10_000, 1_000_003])
def test_integer_data_is_exact(n):
    """Integer-valued data: every partial sum is an exactly representable integer,
    so the result is the exact sum (checked with Python integers)."""
    g = si.rng(n)
    a = g.integers(-1000, 1001, size=n)
    b = g.integers(-1000, 1001, size=n)
    assert oracle.sum_(a.astype(np.float64)) == float(int(a.sum()))
    assert oracle.dot(a.astype(np.float64), b.astype(np.float64)) == float(int(np.dot(a, b)))


@pytest.mark.parametrize("n,seed", [(1000, 1), (100_000, 2)])
def test_sum_within_recursive_summation_bound(n, seed):
    x = si.rng(seed).standard_normal(n)
    exact = math.fsum(x)
    bound = (n - 1) * U * float(np.abs(x).sum())
    assert abs(oracle.sum_(x) - exact) <= bound


def test_dot_within_bound_and_matches_numpy():
    n = 50_000
    g = si.rng(9)
    x, y = g.standard_normal(n), g.standard_normal(n)
    exact = math.fsum(x * y) # products rounded once each: one more u per term
    bound = n * U * float(np.abs(x * y).sum()) * 2
    assert abs(oracle.dot(x, y) - exact) <= bound
    assert abs(oracle.dot(x, y) - float(np.dot(x, y))) <= bound


def test_order_is_sequential():
    """1 + 2^-53 + 2^-53 + ...: a sequential sum from the left loses every tiny
    term (each addition rounds back to 1), unlike a pairwise sum."""
    x = np.full(1001, 2.0 ** -53)
    x[0] = 1.0
    assert oracle.sum_(x) == 1.0
    assert math.fsum(x) > 1.0
