"""The TMA-staged variable-coefficient float sweep (radius 2) against the CPU
oracle, bitwise.

The kernel can run when the padded rows are a multiple of 16 bytes (nx + 4
divisible by 4) and the grids are aligned, and runs by default on grids of
at least four waves of its blocks (the knob var_variant = 2 makes it run
wherever it applies, as most tests here do); it stages 64 x 16-column tiles
with their radius-2 halo through a ring of shared-memory planes.  Shapes
here cover one and several tiles in i and j, ragged last tiles in both,
k chunks of every length the plan makes, a single plane, and odd sweep
counts (ping-pong ending in either buffer).  Halos are random and non-zero:
the sweep reads them and must leave them as they were.
"""
import numpy as np
import pytest

import oracle
import stencil_inputs as si

pytestmark = pytest.mark.gpu

W = si.VARCOEF_W
R = 2


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def to_host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def assert_bitwise(got, ref):
    assert got.shape == ref.shape and got.dtype == ref.dtype
    ut = f"u{got.itemsize}"
    bad = np.argwhere(got.view(ut) != ref.view(ut))
    assert bad.size == 0, f"{len(bad)} mismatches, first at {bad[0]}: {got[tuple(bad[0])]} vs {ref[tuple(bad[0])]}"


def inputs(nx, ny, nz, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (nz + 2 * R, ny + 2 * R, nx + 2 * R)
    u = rng.uniform(-1.0, 1.0, shape).astype(np.float32)      # halo included: non-zero Dirichlet values
    a = rng.uniform(0.5, 1.5, shape).astype(np.float32)
    f = rng.standard_normal(shape).astype(np.float32)
    return u, a, f


@pytest.fixture
def tma_forced(lib):
    lib.stencil_tune_set("var_variant", 2)
    yield
    lib.stencil_tune_set("var_variant", -1)


# nx % 4 == 0 so that rows of nx + 4 floats are a multiple of 16 bytes
TMA_SHAPES = [(64, 16, 8), (128, 32, 40), (68, 17, 5), (4, 1, 1), (196, 50, 23), (60, 15, 130),
              (8, 100, 2), (132, 7, 64), (256, 33, 17)]


@pytest.mark.parametrize("shape", TMA_SHAPES)
@pytest.mark.parametrize("sweeps", [1, 3])
def test_tma_float_sweep_bitwise(lib, cuda, tma_forced, shape, sweeps):
    nx, ny, nz = shape
    q = lib.stencil_plan_query("varcoef_sweep", nx, ny, nz, 4, R)
    assert q["variant"] == 2, q  # forced: the TMA-staged kernel wherever it applies
    u, a, f = inputs(nx, ny, nz, seed=nx * 7 + ny * 3 + nz)
    ref = u
    for _ in range(sweeps):
        ref = oracle.varcoef_sweep(ref, a, f, W, R)
    d_in, d_out = to_dev(u), to_dev(np.zeros_like(u))
    lib.varcoef_sweep_f32(d_in, d_out, to_dev(a), to_dev(f), W, R, sweeps)
    assert_bitwise(to_host(d_out), ref)


def test_tma_equals_column_kernel(lib, cuda):
    """Same bits as the column kernel on a grid of many tiles and chunks."""
    nx, ny, nz = 384, 96, 200
    u, a, f = inputs(nx, ny, nz, seed=11)
    outs = []
    for v in (2, 1):
        lib.stencil_tune_set("var_variant", v)
        try:
            q = lib.stencil_plan_query("varcoef_sweep", nx, ny, nz, 4, R)
            assert q["variant"] == v
            d_in, d_out = to_dev(u), to_dev(np.zeros_like(u))
            lib.varcoef_sweep_f32(d_in, d_out, to_dev(a), to_dev(f), W, R, 4)
            outs.append(to_host(d_out))
        finally:
            lib.stencil_tune_set("var_variant", -1)
    assert_bitwise(outs[0], outs[1])


@pytest.mark.parametrize("shape", [(63, 20, 9), (66, 18, 7), (65, 5, 4)])
def test_unaligned_rows_take_the_column_kernel(lib, cuda, tma_forced, shape):
    """Rows that are not a multiple of 16 bytes cannot be described by a tensor
    map: the column kernel runs instead, with the same bits."""
    nx, ny, nz = shape
    assert lib.stencil_plan_query("varcoef_sweep", nx, ny, nz, 4, R)["variant"] == 1
    u, a, f = inputs(nx, ny, nz, seed=5)
    ref = oracle.varcoef_sweep(oracle.varcoef_sweep(u, a, f, W, R), a, f, W, R)
    d_in, d_out = to_dev(u), to_dev(np.zeros_like(u))
    lib.varcoef_sweep_f32(d_in, d_out, to_dev(a), to_dev(f), W, R, 2)
    assert_bitwise(to_host(d_out), ref)


def test_misaligned_grid_pointer_takes_the_column_kernel(lib, cuda):
    """A u grid that starts 4 bytes past a 16-byte boundary cannot be a tensor
    map's base: the launch falls back to the column kernel (same bits)."""
    import torch
    nx, ny, nz = 64, 12, 6
    u, a, f = inputs(nx, ny, nz, seed=9)
    n = u.size
    buf = torch.zeros(n + 4, dtype=torch.float32, device="cuda")
    d_in = buf[1:1 + n].view(u.shape)
    d_in.copy_(torch.from_numpy(u))
    d_out = to_dev(np.zeros_like(u))
    lib.varcoef_sweep_f32(d_in, d_out, to_dev(a), to_dev(f), W, R, 1)
    assert_bitwise(to_host(d_out), oracle.varcoef_sweep(u, a, f, W, R))


def test_refined_solve_through_tma_sweeps(lib, cuda, tma_forced):
    """The refined solve on an aligned grid runs its float inner sweeps through
    the TMA kernel; it must match the oracle's refinement bitwise and meet tol
    on the oracle's independent double residual."""
    nx, ny, nz = 28, 20, 12
    assert lib.stencil_plan_query("varcoef_sweep", nx, ny, nz, 4, R)["variant"] == 2
    a = si.uniform_full(nx, ny, nz, R, seed=3)
    ustar = si.sine_mode(nx, ny, nz, R)
    f = oracle.varcoef_apply(ustar, a, W, R)
    tol, inner, outer = 1e-10, 400, 30
    u_ref, o_ref, rel_ref, st_ref = oracle.varcoef_refined_solve(a, f, np.zeros_like(f), W, R, tol, inner, outer)
    d_u = to_dev(np.zeros_like(f))
    rc, info = lib.jacobi_solve_varcoef_refined(to_dev(a), to_dev(f), d_u, W, R, tol, inner, outer)
    assert rc == st_ref == 0 and info["outer"] == o_ref
    got = to_host(d_u)
    assert_bitwise(got, u_ref)
    assert oracle.varcoef_residual_norm(got, a, f, W, R) / oracle.interior_norm(f, R) <= tol
