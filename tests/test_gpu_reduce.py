"""Parity of the sum and dotproduct intrinsics (Sec. 5.4, Table 3) with the
oracle, through the C ABI.

The GPU adds in a blocked order and the oracle left to right, so real-valued
results are compared within the recursive-summation bound both satisfy,
|s - exact| <= n u sum|x_i| (u = 2^-53; for dot products sum|x_i y_i| with one
more u per term).  Integer-valued data are exact in any order and are
compared bitwise, including at the paper's full sizes (2^30 and 2^27
elements) against closed forms.
"""
import numpy as np
import pytest

import oracle
import stencil_inputs as si

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


SIZES = [0, 1, 2, 3, 17, 2047, 4096 * 8 + 5, 1_000_003, 1 << 22]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("offset", [0, 1])
def test_sum_matches_oracle(lib, cuda, n, offset):
    """offset 1 starts the array 8 bytes past a 16-byte boundary."""
    x = si.rng(n + 7).standard_normal(n + offset)
    d = dev(x)[offset:]
    got = lib.reduce_sum_f64(d)
    ref = oracle.sum_(np.ascontiguousarray(x[offset:]))
    assert abs(got - ref) <= 2 * n * U * float(np.abs(x[offset:]).sum())


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("ox,oy", [(0, 0), (1, 1), (0, 1), (1, 0)])
def test_dot_matches_oracle(lib, cuda, n, ox, oy):
    g = si.rng(n + 11)
    x, y = g.standard_normal(n + ox), g.standard_normal(n + oy)
    got = lib.dot_f64(dev(x)[ox:], dev(y)[oy:])
    xs, ys = np.ascontiguousarray(x[ox:]), np.ascontiguousarray(y[oy:])
    ref = oracle.dot(xs, ys)
    assert abs(got - ref) <= 4 * (n + 1) * U * float(np.abs(xs * ys).sum())


@pytest.mark.parametrize("n", [5, 4096 * 8 + 3, 3_000_001])
def test_integer_data_bitwise(lib, cuda, n):
    g = si.rng(n)
    a = g.integers(-1000, 1001, size=n).astype(np.float64)
    b = g.integers(-1000, 1001, size=n).astype(np.float64)
    assert lib.reduce_sum_f64(dev(a)) == oracle.sum_(a)
    assert lib.dot_f64(dev(a), dev(b)) == oracle.dot(a, b)


def test_host_arrays_and_repeatability(lib, cuda):
    x = si.rng(5).random(1_234_567)
    s1 = lib.reduce_sum_f64(x)
    s2 = lib.reduce_sum_f64(dev(x))
    assert s1 == s2 == lib.reduce_sum_f64(dev(x))
    assert abs(s1 - oracle.sum_(x)) <= 2 * x.size * U * x.sum()


def test_paper_sizes_exact(lib, cuda):
    """The paper's sizes: sum over a 32768 x 32768 array (2^30 doubles) and a dot
    product of two 2^27-element vectors, on periodic integer data whose exact
    results follow from one period."""
    import torch
    n = 32768 * 32768
    x = (torch.arange(n, device="cuda", dtype=torch.int64) % 1001 - 500).to(torch.float64)
    per = np.arange(1001) - 500
    full, rest = divmod(n, 1001)
    exact = full * int(per.sum()) + int(per[:rest].sum())
    assert lib.reduce_sum_f64(x) == float(exact)
    del x
    n = 1 << 27
    i = torch.arange(n, device="cuda", dtype=torch.int64)
    a = (i % 7 - 3).to(torch.float64)
    b = (i % 11 - 5).to(torch.float64)
    del i
    k = np.arange(77)
    prod = (k % 7 - 3) * (k % 11 - 5)
    full, rest = divmod(n, 77)
    exact = full * int(prod.sum()) + int(prod[:rest].sum())
    assert lib.dot_f64(a, b) == float(exact)
