"""Sweeps of small 3-D grids in one cooperative launch (knob resident3d = 1,
the default for grids of up to 2^18 interior points).

Every sweep is the canonical update, so the result must be the oracle's bit
for bit, for double and float, radius 1 and 2, with a c0 term, non-zero
halos and odd and even sweep counts, and the same bits with the resident
path switched off.  A host-side fault (fault_withhold_3d: one block never
arrives at the grid barrier) makes the other blocks' bounded waits run out:
the next synchronising call on the stream reports STN_ETIMEOUT and the call
after it is correct again on the same context.
"""
import numpy as np
import pytest

import oracle
import stencil_inputs as si

pytestmark = pytest.mark.gpu

L7 = si.LAPLACE7


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def to_host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def bitwise(a, b):
    ut = f"u{a.itemsize}"
    return a.shape == b.shape and np.array_equal(a.view(ut), b.view(ut))


def grid(nx, ny, nz, r, seed, dtype):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, si.padded_shape(nx, ny, nz, r)).astype(dtype)  # halo included


@pytest.fixture
def resident(lib):
    def use(v):
        lib.stencil_tune_set("resident3d", v)
    yield use
    lib.stencil_tune_set("resident3d", 1)
    lib.stencil_tune_set("fault_withhold_3d", 0)


CASES = [((64, 64, 64), 1, L7, 100), ((37, 19, 11), 1, L7, 7), ((1, 1, 1), 1, L7, 4), ((130, 7, 9), 2, (0.2, 0.1, 0.05), 6),
         ((33, 40, 21), 2, (0.0, 0.15, 0.0417), 5), ((5, 300, 4), 1, (0.1, 0.15, 0.0), 2), ((64, 64, 65), 1, L7, 3)]


@pytest.mark.parametrize("shape,r,c,iters", CASES)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_resident_sweeps_bitwise_oracle(lib, cuda, resident, shape, r, c, iters, dtype):
    nx, ny, nz = shape
    u0 = grid(nx, ny, nz, r, seed=nx + 3 * ny + 7 * nz, dtype=dtype)
    ref = oracle.stencil_sweep(u0, c, r, iters)
    sweep = lib.stencil_sweep_f64 if dtype == np.float64 else lib.stencil_sweep_f32
    outs = []
    for v in (1, 0):
        resident(v)
        d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
        sweep(d_in, d_out, c, r, iters)
        outs.append(to_host(d_out))
    assert bitwise(outs[0], ref)
    assert bitwise(outs[1], ref)


def test_c1_configuration_resident(lib, cuda, resident):
    """64^3 FP64, U[0,1) seed 1, 100 sweeps then the residual norm: the
    resident path's result is the oracle's, bit for bit, and the norm within
    1e-12."""
    resident(1)
    u0 = si.uniform_interior(64, 64, 64, 1, seed=1)
    ref = oracle.stencil_sweep(u0, L7, 1, 100)
    d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
    lib.stencil_sweep_f64(d_in, d_out, L7, 1, 100)
    assert bitwise(to_host(d_out), ref)
    n_ref = oracle.residual_norm(ref, L7, 1)
    assert abs(lib.residual_norm_f64(d_out, L7, 1) - n_ref) <= 1e-12 * n_ref


def test_withheld_block_times_out_and_context_survives(lib, cuda, resident):
    resident(1)
    u0 = si.uniform_interior(40, 30, 20, 1, seed=3)
    d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
    lib.stencil_tune_set("fault_withhold_3d", 1)
    lib.stencil_sweep_f64(d_in, d_out, L7, 1, 10)  # asynchronous: returns before the waits run out
    lib.stencil_tune_set("fault_withhold_3d", 0)
    with pytest.raises(lib.StencilError) as ei:
        lib.residual_norm_f64(d_out, L7, 1)          # the next synchronising call on the stream
    assert ei.value.code == lib.STN_ETIMEOUT and "grid barrier" in lib.last_error()
    # the status was reported once; the same context sweeps correctly again
    ref = oracle.stencil_sweep(u0, L7, 1, 10)
    d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
    lib.stencil_sweep_f64(d_in, d_out, L7, 1, 10)
    assert bitwise(to_host(d_out), ref)
    n_ref = oracle.residual_norm(ref, L7, 1)
    assert abs(lib.residual_norm_f64(d_out, L7, 1) - n_ref) <= 1e-12 * n_ref
