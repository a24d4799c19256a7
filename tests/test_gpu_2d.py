"""Parity of the 2-D sweeps (the paper's jacobi benchmark, Sec. 4) with the CPU
oracle, through the C ABI.

Both paths are covered: shared-memory resident bands (one CTA per SM, boundary
rows exchanged every sweep) and per-sweep launches through HBM.  Double and
float sweeps follow the canonical order on both sides and are compared
BITWISE; norms at 1e-12 relative.  Shapes are ragged against the 32 x 8 tile
and against the band partition (fewer rows than SMs, bands of exactly R rows,
single-band grids), and halos are non-zero.
"""
import math

import numpy as np
import pytest

import oracle
import stencil_inputs as si

pytestmark = pytest.mark.gpu

L5 = si.LAPLACE5
C2 = (0.1, 0.15, 0.075)
NORM_RTOL = 1e-12


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def to_host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def assert_bitwise(got, ref):
    assert got.shape == ref.shape and got.dtype == ref.dtype
    bad = np.argwhere(got.view(f"u{got.itemsize}") != ref.view(f"u{ref.itemsize}"))
    assert bad.size == 0, f"{len(bad)} mismatches, first at {bad[0]}: {got[tuple(bad[0])]} vs {ref[tuple(bad[0])]}"


@pytest.fixture(params=["auto", "regs", "hbm", "2band", "3band-regs"])
def path(request, lib):
    """auto: resident, halo rows by bulk copy where rows are 16-byte multiples;
    regs: resident, halo rows through registers; hbm: per-sweep launches;
    2band / 3band-regs: resident with 2 or 3 bands per SM where they fit."""
    lib.stencil_tune_set("sweep2d_resident", 0 if request.param == "hbm" else -1)
    lib.stencil_tune_set("sweep2d_tma", 0 if "regs" in request.param else 1)
    lib.stencil_tune_set("sweep2d_ctas_per_sm", {"2band": 2, "3band-regs": 3}.get(request.param, 1))
    yield request.param
    lib.stencil_tune_set("sweep2d_resident", -1)
    lib.stencil_tune_set("sweep2d_tma", 1)
    lib.stencil_tune_set("sweep2d_ctas_per_sm", 1)


SHAPES2D = [(1024, 1024), (37, 19), (1, 1), (1, 50), (50, 1), (130, 7), (2000, 3), (33, 1000),
            (300, 152), (300, 153), (64, 304), (17, 4)]


@pytest.mark.parametrize("shape", SHAPES2D)
@pytest.mark.parametrize("r,c", [(1, L5), (2, C2)])
def test_sweep2d_f64_bitwise(lib, cuda, path, shape, r, c):
    nx, ny = shape
    u0 = si.uniform_full2d(nx, ny, r, seed=nx + ny, lo=-1, hi=1)
    for iters in (1, 2, 5):
        ref = oracle.stencil_sweep2d(u0, c, r, iters)
        d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
        lib.stencil_sweep2d_f64(d_in, d_out, c, r, iters)
        assert_bitwise(to_host(d_out), ref)


@pytest.mark.parametrize("shape", [(1024, 1024), (37, 19), (300, 153), (2000, 3)])
@pytest.mark.parametrize("r,c", [(1, L5), (2, (0.0, 0.2, 0.05))])
def test_sweep2d_f32_bitwise(lib, cuda, path, shape, r, c):
    nx, ny = shape
    u0 = si.uniform_full2d(nx, ny, r, seed=3 * nx + ny, lo=-1, hi=1, dtype=np.float32)
    ref = oracle.stencil_sweep2d(u0, c, r, 4)
    d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
    lib.stencil_sweep2d_f32(d_in, d_out, c, r, 4)
    assert_bitwise(to_host(d_out), ref)


def test_sweep2d_paper_grid_20_sweeps(lib, cuda):
    """The paper's 1024 x 1024 grid, 20 sweeps, resident path: bitwise; `in` untouched."""
    u0 = si.uniform_interior2d(1024, 1024, 1, seed=7)
    ref = oracle.stencil_sweep2d(u0, L5, 1, 20)
    d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
    lib.stencil_sweep2d_f64(d_in, d_out, L5, 1, 20)
    assert_bitwise(to_host(d_out), ref)
    assert_bitwise(to_host(d_in), u0)


def test_sweep2d_paper_length_eigenmode(lib, cuda):
    """The paper's full run (1024 x 1024, 100000 iterations) on the slowest sine
    mode: the result is cos(pi/1025)^100000 times the start, to within the
    rounding of 1e5 sweeps."""
    u0 = si.sine_mode2d(1024, 1024, 1)
    d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
    lib.stencil_sweep2d_f64(d_in, d_out, L5, 1, 100000)
    lam = math.cos(math.pi / 1025) ** 100000
    got = to_host(d_out)
    assert np.max(np.abs(got - lam * u0)) <= 1e-9 * lam
    assert np.all(got[0] == 0) and np.all(got[-1] == 0) and np.all(got[:, 0] == 0) and np.all(got[:, -1] == 0)


@pytest.mark.parametrize("chunk", [1, 2, 7, 16])
def test_sweep2d_several_launches(lib, cuda, path, chunk):
    """Runs longer than one resident launch continue in place, bit for bit."""
    try:
        lib.stencil_tune_set("sweep2d_chunk", chunk)
        for (nx, ny), r, c in (((100, 333), 1, L5), ((41, 600), 2, C2)):
            u0 = si.uniform_full2d(nx, ny, r, seed=chunk + r, lo=-1, hi=1)
            ref = oracle.stencil_sweep2d(u0, c, r, 30)
            d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
            lib.stencil_sweep2d_f64(d_in, d_out, c, r, 30)
            assert_bitwise(to_host(d_out), ref)
    finally:
        lib.stencil_tune_set("sweep2d_chunk", 32768)


def test_sweep2d_zero_iters_and_host_buffers(lib, cuda):
    u0 = si.uniform_full2d(70, 45, 1, seed=9)
    d_out = to_dev(np.zeros_like(u0))
    lib.stencil_sweep2d_f64(to_dev(u0), d_out, L5, 1, 0)
    assert_bitwise(to_host(d_out), u0)
    h_in, h_out = u0.copy(), np.zeros_like(u0)
    lib.stencil_sweep2d_f64(h_in, h_out, L5, 1, 6)
    assert_bitwise(h_out, oracle.stencil_sweep2d(u0, L5, 1, 6))


@pytest.mark.parametrize("shape", [(1024, 1024), (37, 19), (2000, 3), (1, 1)])
@pytest.mark.parametrize("r,c", [(1, L5), (2, C2)])
def test_residual2d_matches_oracle(lib, cuda, shape, r, c):
    nx, ny = shape
    u = si.uniform_full2d(nx, ny, r, seed=nx, lo=-1, hi=1)
    b = si.uniform_interior2d(nx, ny, r, seed=ny, lo=-1, hi=1)
    for bb in (None, b):
        nref = oracle.residual_norm2d(u, c, r, bb)
        got = lib.residual_norm2d_f64(to_dev(u), c, r, b=None if bb is None else to_dev(bb))
        assert abs(got - nref) <= NORM_RTOL * nref
    u32 = u.astype(np.float32)
    nref = oracle.residual_norm2d(u32, c, r)
    assert abs(lib.residual_norm2d_f32(to_dev(u32), c, r) - nref) <= NORM_RTOL * nref


@pytest.mark.parametrize("tma", [1, 0])
def test_resident_wait_times_out_and_context_survives(lib, cuda, tma):
    """The last band withholds its rows: its neighbour's bounded wait gives up
    (about 2 s), the call returns STN_ETIMEOUT, and the next call is correct."""
    u0 = si.uniform_interior2d(256, 400, 1, seed=11)
    d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
    try:
        lib.stencil_tune_set("sweep2d_tma", tma)
        lib.stencil_tune_set("fault_withhold_2d", 1)
        with pytest.raises(lib.StencilError) as e:
            lib.stencil_sweep2d_f64(d_in, d_out, L5, 1, 50)
        assert e.value.code == lib.STN_ETIMEOUT
    finally:
        lib.stencil_tune_set("fault_withhold_2d", 0)
    lib.stencil_sweep2d_f64(d_in, d_out, L5, 1, 50)
    lib.stencil_tune_set("sweep2d_tma", 1)
    assert_bitwise(to_host(d_out), oracle.stencil_sweep2d(u0, L5, 1, 50))
