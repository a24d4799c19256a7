"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Double sweeps follow the same canonical operation order on both sides, so they
are compared BITWISE; float sweeps likewise against the float oracle.  Norms,
whose reduction order differs, are compared at 1e-12 relative.  Grids are
non-cubic and ragged against the 32 x 8 tile so that partial tiles, partial
k-chunks and every halo duty are exercised.
"""
import math

import numpy as np
import pytest

import oracle
import stencil_inputs as si

pytestmark = pytest.mark.gpu

L7 = si.LAPLACE7
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
    bad = np.argwhere(got.view(np.uint8 if got.itemsize == 1 else f"u{got.itemsize}") !=
                      ref.view(f"u{ref.itemsize}"))
    assert bad.size == 0, f"{len(bad)} mismatches, first at {bad[0]}: {got[tuple(bad[0])]} vs {ref[tuple(bad[0])]}"


# odd NX (scalar kernel) and even NX (two-points-per-lane kernel), partial tiles in i and j
SHAPES = [(64, 64, 64), (37, 19, 11), (33, 9, 70), (1, 1, 1), (1, 50, 3), (65, 8, 5), (31, 17, 4),
          (36, 19, 11), (62, 9, 70), (2, 3, 2), (130, 7, 9), (126, 17, 5)]


# ------------------------------------------------------------------ sweeps --
def test_c1_config_64cubed_100_sweeps_and_norm(lib, cuda):
    """64^3 FP64, U[0,1) interior (seed 1), zero halo, c = {0, 1/6}, 100 sweeps,
    then the L2 norm of the residual."""
    u0 = si.uniform_interior(64, 64, 64, 1, seed=1)
    ref = oracle.stencil_sweep(u0, L7, 1, 100)
    d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
    lib.stencil_sweep_f64(d_in, d_out, L7, 1, 100)
    got = to_host(d_out)
    assert_bitwise(got, ref)
    n_ref = oracle.residual_norm(ref, L7, 1)
    n_gpu = lib.residual_norm_f64(d_out, L7, 1)
    assert abs(n_gpu - n_ref) <= NORM_RTOL * n_ref


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("r,c", [(1, (0.0, 1 / 6)), (1, (0.25, 0.125)), (2, (0.0, 0.125, 1 / 24)),
                                 (2, (0.2, 0.1, 0.0333))])
@pytest.mark.parametrize("iters", [1, 2, 5])
def test_sweep_f64_bitwise(lib, cuda, shape, r, c, iters):
    nx, ny, nz = shape
    u0 = si.uniform_interior(nx, ny, nz, r, seed=7, lo=-1, hi=1)
    # non-zero halo: it must be read and carried to out unchanged
    halo = np.ones_like(u0, dtype=bool)
    halo[r:r + nz, r:r + ny, r:r + nx] = False
    u0[halo] = si.rng(8).random(int(halo.sum()))
    ref = oracle.stencil_sweep(u0, c, r, iters)
    d_in, d_out = to_dev(u0), to_dev(np.full_like(u0, np.nan))
    lib.stencil_sweep_f64(d_in, d_out, c, r, iters)
    assert_bitwise(to_host(d_out), ref)
    if iters == 1:
        assert_bitwise(to_host(d_in), u0)  # in untouched for a single sweep


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("r,c", [(1, (0.0, 1 / 6)), (2, (0.1, 0.1, 0.05))])
def test_sweep_f32_bitwise(lib, cuda, shape, r, c):
    nx, ny, nz = shape
    u0 = si.uniform_interior(nx, ny, nz, r, seed=17, dtype=np.float32)
    ref = oracle.stencil_sweep(u0, c, r, 3)
    d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
    lib.stencil_sweep_f32(d_in, d_out, c, r, 3)
    assert_bitwise(to_host(d_out), ref)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_sweep_misaligned_grids_use_scalar_path(lib, cuda, dtype):
    """Grids that start one element past an aligned address cannot take the
    vector kernel; the scalar kernel must give the same bitwise result."""
    import torch
    nx, ny, nz, r = 62, 9, 13, 1
    u0 = si.uniform_interior(nx, ny, nz, r, seed=41, dtype=dtype)
    ref = oracle.stencil_sweep(u0, L7, r, 3)
    n = u0.size
    base_in = torch.zeros(n + 1, dtype=torch.from_numpy(u0).dtype, device="cuda")
    base_out = torch.zeros(n + 1, dtype=base_in.dtype, device="cuda")
    d_in = base_in[1:].view(u0.shape)
    d_out = base_out[1:].view(u0.shape)
    d_in.copy_(torch.from_numpy(u0))
    (lib.stencil_sweep_f64 if dtype == np.float64 else lib.stencil_sweep_f32)(d_in, d_out, L7, r, 3)
    assert_bitwise(to_host(d_out), ref)
    if dtype == np.float64:
        nref = oracle.residual_norm(ref, L7, r)
        assert abs(lib.residual_norm_f64(d_out, L7, r) - nref) <= NORM_RTOL * nref


@pytest.mark.parametrize("repeat", [1, 0])
@pytest.mark.parametrize("n_iters", [16, 37, 100])
def test_graph_repeated_sweeps_bitwise(lib, cuda, repeat, n_iters):
    """Sweep loops run as a device-repeated CUDA graph (repeat_graph 1: 16 sweeps
    per repetition plus a host-launched remainder) or as stream launches (0):
    the same bits as the oracle either way, for stencil and variable-coefficient
    sweeps and for the refined solver's inner loop."""
    try:
        lib.stencil_tune_set("repeat_graph", repeat)
        for (nx, ny, nz), r, c in (((64, 64, 64), 1, L7), ((37, 19, 11), 2, (0.2, 0.1, 0.0333))):
            u0 = si.uniform_interior(nx, ny, nz, r, seed=n_iters, lo=-1, hi=1)
            ref = oracle.stencil_sweep(u0, c, r, n_iters)
            d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
            lib.stencil_sweep_f64(d_in, d_out, c, r, n_iters)
            assert_bitwise(to_host(d_out), ref)
            u32 = u0.astype(np.float32)
            d_in, d_out = to_dev(u32), to_dev(np.zeros_like(u32))
            lib.stencil_sweep_f32(d_in, d_out, c, r, n_iters)
            assert_bitwise(to_host(d_out), oracle.stencil_sweep(u32, c, r, n_iters))
        nx, ny, nz, R = 21, 13, 9, 2
        a = si.uniform_full(nx, ny, nz, R, seed=3)
        f = si.normal_interior(nx, ny, nz, R, seed=5)
        u = si.uniform_interior(nx, ny, nz, R, seed=6)
        ref = u
        for _ in range(n_iters):
            ref = oracle.varcoef_sweep(ref, a, f, VW, R)
        d_in, d_out = to_dev(u), to_dev(np.zeros_like(u))
        lib.varcoef_sweep_f64(d_in, d_out, to_dev(a), to_dev(f), VW, R, n_iters)
        assert_bitwise(to_host(d_out), ref)
    finally:
        lib.stencil_tune_set("repeat_graph", 1)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("r,c", [(1, (0.0, 1 / 6)), (2, (0.2, 0.1, 0.0333))])
def test_every_kernel_variant_bitwise(lib, cuda, variant, r, c):
    """The one-point-per-thread kernel, both register-blocked kernels and the
    staged (shared-memory ring) kernel give the same bits (forced through the
    tuning knob), for sweeps, residuals and a solve, on shapes ragged against
    every tile size."""
    try:
        lib.stencil_tune_set("star_variant", variant)
        for shape in [(64, 64, 64), (37, 19, 11), (130, 33, 9), (62, 70, 5), (2, 1, 3)]:
            nx, ny, nz = shape
            u0 = si.uniform_interior(nx, ny, nz, r, seed=nx, lo=-1, hi=1)
            b = si.normal_interior(nx, ny, nz, r, seed=ny)
            ref = oracle.stencil_sweep(u0, c, r, 3)
            d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
            lib.stencil_sweep_f64(d_in, d_out, c, r, 3)
            assert_bitwise(to_host(d_out), ref)
            u32 = u0.astype(np.float32)
            d_in, d_out = to_dev(u32), to_dev(np.zeros_like(u32))
            lib.stencil_sweep_f32(d_in, d_out, c, r, 3)
            assert_bitwise(to_host(d_out), oracle.stencil_sweep(u32, c, r, 3))
            nref = oracle.residual_norm(u0, c, r, b)
            assert abs(lib.residual_norm_f64(to_dev(u0), c, r, b=to_dev(b)) - nref) <= NORM_RTOL * nref
        b = si.normal_interior(33, 17, 9, 1, seed=5)
        u_ref, it_ref, _, _ = oracle.jacobi_solve(b, np.zeros_like(b), L7, 1, 1e-8, 20000, 20)
        d_u = to_dev(np.zeros_like(b))
        rc, info = lib.jacobi_solve_f64(to_dev(b), d_u, L7, 1, 1e-8, 20000, 20)
        assert rc == 0 and info["iters"] == it_ref
        assert_bitwise(to_host(d_u), u_ref)
    finally:
        lib.stencil_tune_set("star_variant", -1)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_forced_chunk_counts_bitwise(lib, cuda, variant):
    """Forcing the number of k chunks (one block per tile and chunk: ragged last
    chunks, chunks shorter than the radius ring, more chunks than allowed) leaves
    every sweep bit unchanged and the residual within the norm tolerance."""
    c = (0.2, 0.1, 0.0333)
    try:
        lib.stencil_tune_set("star_variant", variant)
        for chunks in (1, 2, 3, 5, 7, 1000):
            lib.stencil_tune_set("star_chunks", chunks)
            assert lib.stencil_tune_get("star_chunks") == chunks
            for (nx, ny, nz), r, cf in (((37, 19, 29), 1, L7), ((64, 40, 33), 2, c)):
                u0 = si.uniform_interior(nx, ny, nz, r, seed=chunks, lo=-1, hi=1)
                d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
                lib.stencil_sweep_f64(d_in, d_out, cf, r, 2)
                assert_bitwise(to_host(d_out), oracle.stencil_sweep(u0, cf, r, 2))
                u32 = u0.astype(np.float32)
                d_in, d_out = to_dev(u32), to_dev(np.zeros_like(u32))
                lib.stencil_sweep_f32(d_in, d_out, cf, r, 2)
                assert_bitwise(to_host(d_out), oracle.stencil_sweep(u32, cf, r, 2))
                nref = oracle.residual_norm(u0, cf, r)
                assert abs(lib.residual_norm_f64(to_dev(u0), cf, r) - nref) <= NORM_RTOL * nref
    finally:
        lib.stencil_tune_set("star_chunks", 0)
        lib.stencil_tune_set("star_variant", -1)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("offset", [1, 2, 3])
def test_staged_variant_on_unaligned_grids(lib, cuda, dtype, offset):
    """The staged kernel copies 16-byte chunks of the aligned span around each
    plane's rows and falls back to single elements where a chunk would reach
    outside the grid: grids starting 1-3 elements past a 16-byte boundary, and
    ending off one, give the oracle's bits; long rows that leave no room for a
    ring stage fall back to another kernel."""
    import torch
    try:
        lib.stencil_tune_set("star_variant", 3)
        for (nx, ny, nz), r, c in (((37, 19, 11), 1, L7), ((29, 13, 9), 2, (0.2, 0.1, 0.0333))):
            u0 = si.uniform_interior(nx, ny, nz, r, seed=offset, lo=-1, hi=1, dtype=dtype)
            n = u0.size
            flat_in = torch.zeros(n + 8, dtype=torch.float64 if dtype == np.float64 else torch.float32,
                                  device="cuda")
            flat_out = torch.zeros_like(flat_in)
            d_in = flat_in[offset:offset + n].view(u0.shape)
            d_out = flat_out[(offset + 1) % 4:(offset + 1) % 4 + n].view(u0.shape)
            d_in.copy_(torch.from_numpy(u0))
            fn = lib.stencil_sweep_f64 if dtype == np.float64 else lib.stencil_sweep_f32
            fn(d_in, d_out, c, r, 3)
            assert lib.stencil_tune_get("last_star_variant") == 3
            assert_bitwise(to_host(d_out), oracle.stencil_sweep(u0, c, r, 3))
            # the elements around the views are untouched
            assert not flat_out[:(offset + 1) % 4].any() and not flat_out[(offset + 1) % 4 + n:].any()
        # rows too long for a ring stage: another kernel runs, same bits
        u0 = si.uniform_interior(12000, 2, 3, 2, seed=9, dtype=dtype)
        d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
        fn(d_in, d_out, (0.2, 0.1, 0.0333), 2, 2)
        assert lib.stencil_tune_get("last_star_variant") != 3
        assert_bitwise(to_host(d_out), oracle.stencil_sweep(u0, (0.2, 0.1, 0.0333), 2, 2))
    finally:
        lib.stencil_tune_set("star_variant", -1)


@pytest.mark.parametrize("depth", [2, 3, 4])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("r,c", [(1, (0.0, 1 / 6)), (2, (0.2, 0.1, 0.0333))])
def test_temporal_blocking_bitwise(lib, cuda, depth, dtype, r, c):
    """depth sweeps fused per pass (temporal blocking) equal depth separate
    sweeps bit for bit, including a remainder of single sweeps, non-zero halos,
    ragged tiles (62 x 16 output tiles) and grids thinner than the fused depth."""
    try:
        lib.stencil_tune_set("temporal_depth", depth)
        for shape, iters in [((64, 64, 64), 2 * depth + 1), ((37, 19, 11), depth), ((125, 33, 40), 7),
                             ((3, 2, 1), depth + 2), ((62, 16, 2), 2 * depth), ((70, 45, 100), depth + 1)]:
            nx, ny, nz = shape
            u0 = si.uniform_interior(nx, ny, nz, r, seed=nx + 3, lo=-1, hi=1, dtype=dtype)
            halo = np.ones_like(u0, dtype=bool)
            halo[r:r + nz, r:r + ny, r:r + nx] = False
            u0[halo] = si.rng(9).random(int(halo.sum())).astype(dtype)
            ref = oracle.stencil_sweep(u0, c, r, iters)
            d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
            fn = lib.stencil_sweep_f64 if dtype == np.float64 else lib.stencil_sweep_f32
            fn(d_in, d_out, c, r, iters)
            assert_bitwise(to_host(d_out), ref)
    finally:
        lib.stencil_tune_set("temporal_depth", 0)


def test_sweep_iters_zero_copies(lib, cuda):
    u0 = si.uniform_interior(9, 8, 7, 1, seed=3)
    d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
    lib.stencil_sweep_f64(d_in, d_out, L7, 1, 0)
    assert_bitwise(to_host(d_out), u0)


def test_sweep_host_buffers(lib, cuda):
    """Host (numpy) grids are staged through device memory by the library."""
    u0 = si.uniform_interior(40, 21, 13, 1, seed=5)
    ref = oracle.stencil_sweep(u0, L7, 1, 4)
    h_in, h_out = u0.copy(), np.zeros_like(u0)
    lib.stencil_sweep_f64(h_in, h_out, L7, 1, 4)
    assert_bitwise(h_out, ref)


def test_host_grids_through_the_abi(lib, cuda):
    """The calls that stage host grids (the path the bench's e2e figures time)
    give the device calls' bits: residual norm, Jacobi solve, and the
    variable-coefficient apply, sweep, residual, solve and refined solve; the
    constant-coefficient refined solve's scheduler engine takes device grids
    only."""
    nx, ny, nz, r = 29, 17, 13, 1
    b = si.normal_interior(nx, ny, nz, r, seed=71)
    u = si.uniform_interior(nx, ny, nz, r, seed=72, lo=-1, hi=1)
    assert lib.residual_norm_f64(u, L7, r, b=b) == lib.residual_norm_f64(to_dev(u), L7, r, b=to_dev(b))
    uh = np.zeros_like(b)
    rc_h, info_h = lib.jacobi_solve_f64(b, uh, L7, r, 1e-8, 20000, 25)
    ud = to_dev(np.zeros_like(b))
    rc_d, info_d = lib.jacobi_solve_f64(to_dev(b), ud, L7, r, 1e-8, 20000, 25)
    assert rc_h == rc_d == 0 and info_h["iters"] == info_d["iters"]
    assert_bitwise(uh, to_host(ud))
    R, W = 2, si.VARCOEF_W
    a = si.uniform_full(nx, ny, nz, R, seed=73)
    f = si.normal_interior(nx, ny, nz, R, seed=74)
    v = si.uniform_interior(nx, ny, nz, R, seed=75)
    oh = np.zeros_like(v)
    lib.varcoef_apply_f64(v, a, oh, W, R)
    od = to_dev(np.zeros_like(v))
    lib.varcoef_apply_f64(to_dev(v), to_dev(a), od, W, R)
    assert_bitwise(oh, to_host(od))
    oh = np.zeros_like(v)
    lib.varcoef_sweep_f64(v.copy(), oh, a, f, W, R, 3)
    od = to_dev(np.zeros_like(v))
    lib.varcoef_sweep_f64(to_dev(v), od, to_dev(a), to_dev(f), W, R, 3)
    assert_bitwise(oh, to_host(od))
    assert lib.varcoef_residual_norm_f64(v, a, f, W, R) == lib.varcoef_residual_norm_f64(
        to_dev(v), to_dev(a), to_dev(f), W, R)
    for solve, args in ((lib.jacobi_solve_varcoef_f64, (1e-8, 200000, 50)),
                        (lib.jacobi_solve_varcoef_refined, (1e-10, 300, 40))):
        uh = np.zeros_like(f)
        rc_h, info_h = solve(a, f, uh, W, R, *args)
        ud = to_dev(np.zeros_like(f))
        rc_d, info_d = solve(to_dev(a), to_dev(f), ud, W, R, *args)
        assert rc_h == rc_d == 0 and info_h["iters"] == info_d["iters"], (solve, info_h, info_d)
        assert_bitwise(uh, to_host(ud))
    # the constant-coefficient refined solve: host grids are staged like the
    # others on the full-grid engine (the default); the scheduler engine takes
    # device grids only
    uh = np.zeros_like(b)
    rc_h, info_h = lib.jacobi_solve_refined_f64(b, uh, L7, r, 1e-8, 100, 0.0, 10, 5)
    ud = to_dev(np.zeros_like(b))
    rc_d, info_d = lib.jacobi_solve_refined_f64(to_dev(b), ud, L7, r, 1e-8, 100, 0.0, 10, 5)
    assert rc_h == rc_d and info_h["outer"] == info_d["outer"]
    assert_bitwise(uh, to_host(ud))
    lib.stencil_tune_set("refined_engine", 0)
    try:
        with pytest.raises(lib.StencilError) as ei:
            lib.jacobi_solve_refined_f64(b, np.zeros_like(b), L7, r, 1e-8, 100, 0.0, 10, 5)
        assert ei.value.code == lib.STN_EINVAL
    finally:
        lib.stencil_tune_set("refined_engine", 1)


def test_eigenmode_decay_1000_sweeps_128(lib, cuda):
    """Property that holds at any size: the (1,1,1) sine mode decays by exactly
    lambda = (cos tx + cos ty + cos tz)/3 per sweep."""
    nx, ny, nz = 128, 96, 80
    u0 = si.sine_mode(nx, ny, nz, 1)
    lam = sum(math.cos(math.pi / (n + 1)) for n in (nx, ny, nz)) / 3
    d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
    lib.stencil_sweep_f64(d_in, d_out, L7, 1, 1000)
    got = to_host(d_out)
    expect = lam ** 1000 * u0
    assert np.max(np.abs(got - expect)) / np.max(np.abs(expect)) < 1e-12


def test_full_size_512_1000_sweeps_closed_form(lib, cuda):
    """The bench workload's size and launch configuration (512^3, 1000 sweeps,
    the default kernel and plan): the (1,1,1) sine mode ends at lambda^1000 times
    the start, and the fused residual norm at |1 - lambda| lambda^1000 ||u0||
    with ||u0||^2 = (513/2)^3."""
    n = 512
    u0 = si.sine_mode(n, n, n, 1)
    lam = math.cos(math.pi / (n + 1))
    d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
    lib.stencil_sweep_f64(d_in, d_out, L7, 1, 1000)
    norm = lib.residual_norm_f64(d_out, L7, 1)
    got = to_host(d_out)
    assert np.max(np.abs(got - lam ** 1000 * u0)) <= 1e-12 * lam ** 1000
    expect = abs(1 - lam) * lam ** 1000 * math.sqrt((n + 1) / 2) ** 3
    assert abs(norm - expect) <= 1e-9 * expect


# -------------------------------------------------------------- residuals --
@pytest.mark.parametrize("shape", SHAPES[:5] + SHAPES[7:9])
@pytest.mark.parametrize("r,c", [(1, (0.0, 1 / 6)), (2, (0.2, 0.1, 0.0333))])
def test_residual_norm_with_source(lib, cuda, shape, r, c):
    nx, ny, nz = shape
    u = si.uniform_interior(nx, ny, nz, r, seed=23)
    b = si.normal_interior(nx, ny, nz, r, seed=24)
    for bb in (None, b):
        ref = oracle.residual_norm(u, c, r, bb)
        got = lib.residual_norm_f64(to_dev(u), c, r, b=None if bb is None else to_dev(bb))
        assert abs(got - ref) <= NORM_RTOL * ref
    u32, b32 = u.astype(np.float32), b.astype(np.float32)
    ref32 = oracle.residual_norm(u32, c, r, b32)
    got32 = lib.residual_norm_f32(to_dev(u32), c, r, b=to_dev(b32))
    assert abs(got32 - ref32) <= NORM_RTOL * ref32


def test_residual_norm_deterministic(lib, cuda):
    u = to_dev(si.uniform_interior(130, 70, 90, 1, seed=29))
    vals = {lib.residual_norm_f64(u, L7, 1) for _ in range(5)}
    assert len(vals) == 1


# ------------------------------------------------------------------ solves --
@pytest.fixture(params=[1, 0], ids=["graph", "hostloop"])
def solve_mode(request, lib):
    """Both iteration drivers: the CUDA graph with a device-side while node and
    the host loop; they launch the same kernels, so they give the same bits."""
    lib.stencil_tune_set("solve_graph", request.param)
    yield request.param
    lib.stencil_tune_set("solve_graph", 1)


@pytest.mark.parametrize("shape,K", [((12, 9, 7), 5), ((33, 17, 9), 20), ((5, 4, 6), 1), ((20, 20, 20), 7)])
def test_jacobi_solve_matches_oracle(lib, cuda, shape, K, solve_mode):
    nx, ny, nz = shape
    b = si.normal_interior(nx, ny, nz, 1, seed=5)
    u0 = np.zeros_like(b)
    tol = 1e-8
    u_ref, it_ref, rel_ref, st_ref = oracle.jacobi_solve(b, u0, L7, 1, tol, 20000, K)
    d_u = to_dev(u0)
    rc, info = lib.jacobi_solve_f64(to_dev(b), d_u, L7, 1, tol, 20000, K)
    assert rc == st_ref == 0
    assert info["iters"] == it_ref
    assert abs(info["rel_res"] - rel_ref) <= NORM_RTOL * rel_ref
    assert_bitwise(to_host(d_u), u_ref)


def test_jacobi_solve_not_converged_and_zero_iters(lib, cuda, solve_mode):
    b = si.normal_interior(10, 10, 10, 1, seed=6)
    d_u = to_dev(np.zeros_like(b))
    rc, info = lib.jacobi_solve_f64(to_dev(b), d_u, L7, 1, 1e-14, 30, 7)
    assert rc == lib.STN_NOT_CONVERGED and info["iters"] == 30  # 4 full groups (graph) + a remainder of 2
    u_ref, it_ref, rel_ref, _ = oracle.jacobi_solve(b, np.zeros_like(b), L7, 1, 1e-14, 30, 7)
    assert_bitwise(to_host(d_u), u_ref)
    assert abs(info["rel_res"] - rel_ref) <= NORM_RTOL * rel_ref
    rc0, info0 = lib.jacobi_solve_f64(to_dev(b), to_dev(np.zeros_like(b)), L7, 1, 1e-3, 0, 7)
    assert rc0 == lib.STN_NOT_CONVERGED and info0["iters"] == 0
    assert abs(info0["rel_res"] - 1.0) < 1e-12  # u = 0: rho = b


# ---------------------------------------------------- variable coefficient --
VW = si.VARCOEF_W


@pytest.fixture(params=[-1, 0, 1])
def var_variant(request, lib):
    """-1: automatic (the TMA-staged kernel for float radius-2 sweeps on rows of
    a multiple of 16 bytes, else the column kernel with shared face
    coefficients); 0: the plane kernel; 1: the column kernel."""
    lib.stencil_tune_set("var_variant", request.param)
    yield request.param
    lib.stencil_tune_set("var_variant", -1)


@pytest.mark.parametrize("shape", [(21, 13, 9), (40, 7, 12), (1, 3, 2), (60, 37, 19), (29, 5, 33)])
@pytest.mark.parametrize("R", [1, 2])
def test_varcoef_apply_sweep_residual(lib, cuda, var_variant, shape, R):
    nx, ny, nz = shape
    a = si.uniform_full(nx, ny, nz, R, seed=3)
    f = si.normal_interior(nx, ny, nz, R, seed=5)
    u = si.uniform_interior(nx, ny, nz, R, seed=6)
    w = VW[:R + 1]
    # apply
    d_out = to_dev(np.zeros_like(u))
    lib.varcoef_apply_f64(to_dev(u), to_dev(a), d_out, w, R)
    assert_bitwise(to_host(d_out), oracle.varcoef_apply(u, a, w, R))
    # sweeps (double and float)
    ref = u
    for _ in range(3):
        ref = oracle.varcoef_sweep(ref, a, f, w, R)
    d_in, d_out = to_dev(u), to_dev(np.zeros_like(u))
    lib.varcoef_sweep_f64(d_in, d_out, to_dev(a), to_dev(f), w, R, 3)
    assert_bitwise(to_host(d_out), ref)
    u32, a32, f32 = u.astype(np.float32), a.astype(np.float32), f.astype(np.float32)
    ref32 = u32
    for _ in range(3):
        ref32 = oracle.varcoef_sweep(ref32, a32, f32, w, R)
    d_in, d_out = to_dev(u32), to_dev(np.zeros_like(u32))
    lib.varcoef_sweep_f32(d_in, d_out, to_dev(a32), to_dev(f32), w, R, 3)
    assert_bitwise(to_host(d_out), ref32)
    # residual
    nref = oracle.varcoef_residual_norm(u, a, f, w, R)
    assert abs(lib.varcoef_residual_norm_f64(to_dev(u), to_dev(a), to_dev(f), w, R) - nref) <= NORM_RTOL * nref


def test_varcoef_jacobi_solve_matches_oracle(lib, cuda, var_variant):
    nx, ny, nz, R = 14, 9, 11, 2
    a = si.uniform_full(nx, ny, nz, R, seed=3)
    f = si.normal_interior(nx, ny, nz, R, seed=5)
    u_ref, it_ref, rel_ref, st = oracle.varcoef_jacobi_solve(a, f, np.zeros_like(f), VW, R, 1e-9, 50000, 25)
    d_u = to_dev(np.zeros_like(f))
    rc, info = lib.jacobi_solve_varcoef_f64(to_dev(a), to_dev(f), d_u, VW, R, 1e-9, 50000, 25)
    assert rc == st == 0 and info["iters"] == it_ref
    assert abs(info["rel_res"] - rel_ref) <= NORM_RTOL * rel_ref
    assert_bitwise(to_host(d_u), u_ref)


@pytest.fixture(params=[1, 0])
def repeat_graph(request, lib):
    lib.stencil_tune_set("repeat_graph", request.param)
    yield request.param
    lib.stencil_tune_set("repeat_graph", 1)


def test_refined_solve_matches_oracle(lib, cuda, var_variant, repeat_graph):
    """Manufactured (1,1,1) sine-mode solution: f = A u* by the oracle.  The float
    inner sweeps and the double residual/update are bitwise on both sides, so
    the refined iterate must agree bitwise while the outer-step counts agree."""
    nx, ny, nz, R = 24, 20, 12, 2
    a = si.uniform_full(nx, ny, nz, R, seed=3)
    ustar = si.sine_mode(nx, ny, nz, R)
    f = oracle.varcoef_apply(ustar, a, VW, R)
    tol, inner, outer = 1e-10, 400, 30
    u_ref, o_ref, rel_ref, st_ref = oracle.varcoef_refined_solve(a, f, np.zeros_like(f), VW, R, tol, inner, outer)
    d_u = to_dev(np.zeros_like(f))
    rc, info = lib.jacobi_solve_varcoef_refined(to_dev(a), to_dev(f), d_u, VW, R, tol, inner, outer)
    assert rc == st_ref == 0 and info["outer"] == o_ref
    got = to_host(d_u)
    assert_bitwise(got, u_ref)
    # independent double residual of the returned u
    assert oracle.varcoef_residual_norm(got, a, f, VW, R) / oracle.interior_norm(f, R) <= tol


def test_extents_beyond_the_launch_grid_are_rejected_before_launch(lib, cuda):
    """A double sweep of 1 x ny x 1 runs the plane kernel, 8 rows per tile:
    ny = 65535 x 8 needs exactly CUDA's 65535 blocks in y and runs (bitwise
    the oracle); one row more would need 65536 and is STN_EINVAL, from the
    sweep and from the plan query alike, before anything is launched."""
    ny = 65535 * 8
    u0 = si.uniform_interior(1, ny, 1, 1, seed=41)
    d_out = to_dev(np.zeros_like(u0))
    lib.stencil_sweep_f64(to_dev(u0), d_out, L7, 1, 2)
    assert_bitwise(to_host(d_out), oracle.stencil_sweep(u0, L7, 1, 2))
    assert lib.stencil_plan_query("sweep", 1, ny, 1, 8, 1)["grid_y"] == 65535
    u1 = si.uniform_interior(1, ny + 1, 1, 1, seed=42)
    d1 = to_dev(np.zeros_like(u1))
    with pytest.raises(lib.StencilError) as e:
        lib.stencil_sweep_f64(to_dev(u1), d1, L7, 1, 1)
    assert e.value.code == -1 and "launch grid" in lib.last_error()
    with pytest.raises(lib.StencilError):
        lib.stencil_plan_query("sweep", 1, ny + 1, 1, 8, 1)
    # the context is unaffected
    lib.stencil_sweep_f64(to_dev(u0), d_out, L7, 1, 1)
    assert_bitwise(to_host(d_out), oracle.stencil_sweep(u0, L7, 1, 1))
