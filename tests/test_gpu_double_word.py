"""The opt-in double sweep in double-word float arithmetic (knob
fp64_double_word = 1) against the CPU oracle's canonical double sweep.

It is not bitwise: every value is a float pair of about 48 bits.  Its error
per sweep is at most about 40 * 2^-48 of the largest magnitude in the
neighbourhood (split of the six neighbours, five double-word additions and
the product with c1, each within the published double-word bounds, and the
final rounding to double), and the 7-point Jacobi update with weights 1/6 is
non-expansive in the max norm, so after n sweeps the error is at most
n * 40 * 2^-48 * max|u0|.  Points whose neighbours lie outside the range
the float split handles take the canonical double update, bit for bit.
"""
import numpy as np
import pytest

import oracle
import stencil_inputs as si

pytestmark = pytest.mark.gpu

L7 = si.LAPLACE7
PER_SWEEP = 40.0 * 2.0 ** -48


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def to_host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture
def double_word(lib):
    lib.stencil_tune_set("fp64_double_word", 1)
    yield
    lib.stencil_tune_set("fp64_double_word", 0)


def run(lib, u0, iters):
    d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
    lib.stencil_sweep_f64(d_in, d_out, L7, 1, iters)
    return to_host(d_out)


@pytest.mark.parametrize("shape", [(64, 64, 64), (37, 19, 11), (130, 7, 40), (1, 1, 1), (33, 40, 3)])
@pytest.mark.parametrize("iters", [1, 10])
def test_double_word_within_bound(lib, cuda, double_word, shape, iters):
    nx, ny, nz = shape
    rng = np.random.Generator(np.random.PCG64(nx + ny + nz))
    u0 = rng.uniform(-1.0, 1.0, si.padded_shape(nx, ny, nz, 1))  # non-zero halo, mixed signs
    ref = oracle.stencil_sweep(u0, L7, 1, iters)
    got = run(lib, u0, iters)
    err = np.max(np.abs(got - ref))
    assert err <= iters * PER_SWEEP * np.max(np.abs(u0)), err
    # the halo stays the input's
    assert np.array_equal(got[0], u0[0]) and np.array_equal(got[:, 0], u0[:, 0])


def test_double_word_out_of_range_points_are_exact(lib, cuda, double_word):
    """Zeros are split exactly; values below 2^-74 or at or above 2^127 send
    their neighbours to the canonical double update."""
    nx, ny, nz = 40, 30, 20
    u0 = si.uniform_interior(nx, ny, nz, 1, seed=3, lo=0.5, hi=1.0)
    u0[5:9, 5:9, 5:9] = 1e-30
    u0[12, 12, 12] = 3e38 * 1e5  # beyond the float range
    ref = oracle.stencil_sweep(u0, L7, 1, 1)
    got = run(lib, u0, 1)
    # neighbours of the out-of-range cells: bitwise the oracle's
    mask = np.zeros(u0.shape, dtype=bool)
    for (k, j, i) in [(k, j, i) for k in range(5, 9) for j in range(5, 9) for i in range(5, 9)] + [(12, 12, 12)]:
        for dk, dj, di in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            mask[k + dk, j + dj, i + di] = True
    mask[0, :, :] = mask[-1, :, :] = mask[:, 0, :] = mask[:, -1, :] = mask[:, :, 0] = mask[:, :, -1] = False
    assert np.array_equal(got[mask].view(np.uint64), ref[mask].view(np.uint64))
    rest = ~mask
    assert np.max(np.abs(got[rest] - ref[rest])) <= PER_SWEEP * 1.0


def test_double_word_eigenmode_1000_sweeps(lib, cuda, double_word):
    """1000 sweeps of the (1,1,1) sine mode on 128 x 96 x 80: within the
    accumulated bound of the oracle's canonical result, which the closed form
    pins (lambda^1000 times the mode)."""
    nx, ny, nz = 128, 96, 80
    u0 = si.sine_mode(nx, ny, nz, 1)
    ref = oracle.stencil_sweep(u0, L7, 1, 1000)
    got = run(lib, u0, 1000)
    err = np.max(np.abs(got - ref))
    assert err <= 1000 * PER_SWEEP * np.max(np.abs(u0)), err
