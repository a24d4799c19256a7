"""jacobi_solve_refined_f64 on the full-grid kernels (knob refined_engine = 1,
the default) against the CPU oracle's refinement.

With a fixed number of float sweeps per outer step the refinement is a fixed
sequence of roundings (double sweep, t - u, max |t - u|, float((t - u) / s),
float sweeps from e = 0, u + s * e), so the returned u must equal the
oracle's bit for bit, on grids that take each float kernel (column, staged,
two-plane at radius 2) and the device-repeated graph loop.  With an adaptive
inner stop the result must reach tol on the oracle's independent double
residual.  The scheduler's batch-of-one path (refined_engine = 0) computes
the same steps: with a fixed inner count both engines give the same bits.
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
    return a.shape == b.shape and np.array_equal(a.view(np.uint64), b.view(np.uint64))


@pytest.fixture
def engine(lib):
    def use(v):
        lib.stencil_tune_set("refined_engine", v)
    yield use
    lib.stencil_tune_set("refined_engine", 1)


@pytest.mark.parametrize("shape,r,c,inner", [
    ((20, 14, 9), 1, L7, 150),          # small: device-repeated graph inner loop
    ((37, 19, 11), 1, L7, 37),          # odd inner count: graph body + host remainder
    ((130, 70, 40), 1, L7, 64),         # column float kernel, many tiles
    ((24, 22, 18), 2, (0.1, 0.1, 0.025), 80),  # radius 2 with c0: two-plane float kernel
])
def test_direct_fixed_inner_bitwise_oracle(lib, cuda, engine, shape, r, c, inner):
    nx, ny, nz = shape
    b = si.normal_interior(nx, ny, nz, r, seed=nx + ny + nz)
    tol, outer_max = 1e-10, 40
    u_ref, o_ref, rel_ref, st = oracle.refined_solve(b, np.zeros_like(b), c, r, tol, inner, outer_max)
    engine(1)
    d_u = to_dev(np.zeros_like(b))
    rc, info = lib.jacobi_solve_refined_f64(to_dev(b), d_u, c, r, tol, inner, 0.0, 50, outer_max)
    assert rc == st and info["outer"] == o_ref and info["iters"] == o_ref * inner, (info, o_ref, st)
    got = to_host(d_u)
    assert bitwise(got, u_ref)
    assert abs(info["rel_res"] - rel_ref) <= 1e-12 * rel_ref
    if st == 0:
        assert oracle.residual_norm(got, c, r, b) / oracle.interior_norm(b, r) <= tol


def test_direct_fixed_inner_staged_kernel(lib, cuda, engine):
    """A grid of over 3e7 points: the float sweeps take the staged kernel; two
    outer steps of 6 float sweeps against the oracle, bitwise."""
    nx, ny, nz = 320, 320, 300
    b = si.normal_interior(nx, ny, nz, 1, seed=3)
    assert lib.stencil_plan_query("sweep", nx, ny, nz, 4, 1)["variant"] == 3
    u_ref, o_ref, rel_ref, st = oracle.refined_solve(b, np.zeros_like(b), L7, 1, 1e-30, 6, 2)
    engine(1)
    d_u = to_dev(np.zeros_like(b))
    rc, info = lib.jacobi_solve_refined_f64(to_dev(b), d_u, L7, 1, 1e-30, 6, 0.0, 50, 2)
    assert rc == lib.STN_NOT_CONVERGED == st and info["outer"] == o_ref == 2
    assert bitwise(to_host(d_u), u_ref)


def test_engines_agree_with_fixed_inner(lib, cuda, engine):
    sizes = [(33, 21, 17), (64, 9, 40)]
    for i, (nx, ny, nz) in enumerate(sizes):
        b = si.normal_interior(nx, ny, nz, 1, seed=70 + i)
        outs = []
        for v in (0, 1):
            engine(v)
            d_u = to_dev(np.zeros_like(b))
            rc, info = lib.jacobi_solve_refined_f64(to_dev(b), d_u, L7, 1, 1e-9, 120, 0.0, 40, 30)
            assert rc == 0
            outs.append((to_host(d_u), info["outer"], info["iters"]))
        assert bitwise(outs[0][0], outs[1][0]) and outs[0][1:] == outs[1][1:]


@pytest.mark.parametrize("solve_graph", [1, 0])
def test_direct_adaptive_inner_reaches_tolerance(lib, cuda, engine, solve_graph):
    engine(1)
    lib.stencil_tune_set("solve_graph", solve_graph)
    try:
        for i, (nx, ny, nz) in enumerate([(40, 30, 20), (16, 16, 16), (12, 50, 7), (90, 64, 48)]):
            b = si.normal_interior(nx, ny, nz, 1, seed=21 + i)
            for tol in (1e-8, 1e-10):
                d_u = to_dev(np.zeros_like(b))
                rc, info = lib.jacobi_solve_refined_f64(to_dev(b), d_u, L7, 1, tol, 200000, 1e-2, 50, 40)
                assert rc == 0 and info["status"] == 0
                got = to_host(d_u)
                rel = oracle.residual_norm(got, L7, 1, b) / oracle.interior_norm(b, 1)
                assert rel <= tol and abs(rel - info["rel_res"]) <= 1e-6 * tol
                # the inner loop stops on whole groups of check_every sweeps
                assert info["iters"] % 50 == 0
    finally:
        lib.stencil_tune_set("solve_graph", 1)


def test_direct_host_grids(lib, cuda, engine):
    """Host (numpy) grids are staged through device copies: same bits."""
    engine(1)
    nx, ny, nz = 26, 18, 13
    b = si.normal_interior(nx, ny, nz, 1, seed=5)
    u_h = np.zeros_like(b)
    rc, info = lib.jacobi_solve_refined_f64(b, u_h, L7, 1, 1e-9, 90, 0.0, 30, 30)
    d_u = to_dev(np.zeros_like(b))
    rc2, info2 = lib.jacobi_solve_refined_f64(to_dev(b), d_u, L7, 1, 1e-9, 90, 0.0, 30, 30)
    assert rc == rc2 == 0 and info["outer"] == info2["outer"]
    assert bitwise(u_h, to_host(d_u))
