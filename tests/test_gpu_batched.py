"""Batched persistent solves (one cluster launch over many problems) and the
mixed-precision refinement, against the CPU oracle.

A batched problem's sweeps are the single-problem path's sweeps (same tile
code, same canonical order), so its iterate must agree bitwise with the
oracle's Jacobi solve whenever the iteration counts agree; and a problem's
result must not depend on which other problems share the launch.
"""
import numpy as np
import pytest

import oracle
import stencil_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(params=[0, 1, 2], ids=["scheduler", "clusters", "pool"])
def engine(request, lib):
    """The batched engines: the dynamic work-unit scheduler, one cluster per
    problem, and worker streams running the one-problem solves; they must give
    the same bits."""
    lib.stencil_tune_set("batch_engine", request.param)
    yield request.param
    lib.stencil_tune_set("batch_engine", 0)

L7 = si.LAPLACE7
NORM_RTOL = 1e-12


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def to_host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def bitwise(a, b):
    return a.shape == b.shape and np.array_equal(a.view(np.uint64), b.view(np.uint64))


SIZES = [(16, 16, 16), (23, 17, 40), (40, 9, 11), (8, 30, 12), (33, 33, 5), (5, 6, 7), (1, 1, 1), (64, 20, 9)]


def make_batch(sizes, seed0=5):
    rhs = [si.normal_interior(nx, ny, nz, 1, seed=seed0 + i) for i, (nx, ny, nz) in enumerate(sizes)]
    return rhs


def test_batched_f64_matches_oracle_and_is_composition_independent(lib, cuda, engine):
    rhs = make_batch(SIZES)
    tol, K, maxit = 1e-8, 10, 40000
    d_u = [to_dev(np.zeros_like(b)) for b in rhs]
    d_b = [to_dev(b) for b in rhs]
    rc, infos = lib.jacobi_solve_batched_f64(d_u, d_b, L7, 1, tol, maxit, K)
    assert rc == 0
    got = [to_host(u) for u in d_u]
    for i, b in enumerate(rhs):
        u_ref, it_ref, rel_ref, st = oracle.jacobi_solve(b, np.zeros_like(b), L7, 1, tol, maxit, K)
        assert st == 0 and infos[i]["status"] == 0
        assert infos[i]["iters"] == it_ref, (i, infos[i], it_ref)
        assert abs(infos[i]["rel_res"] - rel_ref) <= NORM_RTOL * rel_ref
        assert bitwise(got[i], u_ref), i
    # the same problem alone, and in a different mix, gives the same bits
    for pick in ([3], [6, 3, 0]):
        d_u2 = [to_dev(np.zeros_like(rhs[i])) for i in pick]
        d_b2 = [to_dev(rhs[i]) for i in pick]
        rc2, infos2 = lib.jacobi_solve_batched_f64(d_u2, d_b2, L7, 1, tol, maxit, K)
        assert rc2 == 0
        for j, i in enumerate(pick):
            assert bitwise(to_host(d_u2[j]), got[i])
            assert infos2[j]["iters"] == infos[i]["iters"] and infos2[j]["rel_res"] == infos[i]["rel_res"]


def test_batched_not_converged_and_empty(lib, cuda, engine):
    rhs = make_batch(SIZES[:3])
    d_u = [to_dev(np.zeros_like(b)) for b in rhs]
    rc, infos = lib.jacobi_solve_batched_f64(d_u, [to_dev(b) for b in rhs], L7, 1, 1e-14, 25, 10)
    assert rc == lib.STN_NOT_CONVERGED and all(i["iters"] == 25 and i["status"] == 1 for i in infos)
    for i, b in enumerate(rhs):
        u_ref, _, rel_ref, _ = oracle.jacobi_solve(b, np.zeros_like(b), L7, 1, 1e-14, 25, 10)
        assert bitwise(to_host(d_u[i]), u_ref)
    assert lib.jacobi_solve_batched_f64([], [], L7, 1, 1e-8, 10, 10) == (0, [])


def test_batched_rejects_host_grids(lib, cuda):
    b = si.normal_interior(4, 4, 4, 1, seed=1)
    with pytest.raises(lib.StencilError):
        lib.jacobi_solve_batched_f64([np.zeros_like(b)], [b], L7, 1, 1e-8, 10, 10)


def test_batched_radius2_with_center_term_matches_oracle(lib, cuda, engine):
    """A radius-2 star with a centre coefficient (c0 + 6 c1 + 6 c2 = 0.85, a
    contraction) on problems of every scheduler tile shape: the 16 x 16, 48 x 9
    and 12 x 30 problems take 16 x 16 tiles, 64 x 20 and 30 x 3 take 32 x 8,
    8 x 60 and 7 x 33 take 8 x 32; bitwise the oracle's solve, with its sweep
    count."""
    c = (0.1, 0.1, 0.025)
    sizes = [(16, 16, 6), (48, 9, 7), (12, 30, 5), (64, 20, 4), (30, 3, 9), (8, 60, 5), (7, 33, 6)]
    rhs = [si.normal_interior(nx, ny, nz, 2, seed=40 + i) for i, (nx, ny, nz) in enumerate(sizes)]
    tol, K, maxit = 1e-10, 7, 5000
    d_u = [to_dev(np.zeros_like(b)) for b in rhs]
    rc, infos = lib.jacobi_solve_batched_f64(d_u, [to_dev(b) for b in rhs], c, 2, tol, maxit, K)
    assert rc == 0
    for i, b in enumerate(rhs):
        u_ref, it_ref, rel_ref, st = oracle.jacobi_solve(b, np.zeros_like(b), c, 2, tol, maxit, K)
        assert st == 0 and infos[i]["status"] == 0
        assert infos[i]["iters"] == it_ref, (i, infos[i], it_ref)
        assert abs(infos[i]["rel_res"] - rel_ref) <= NORM_RTOL * rel_ref
        assert bitwise(to_host(d_u[i]), u_ref), i


@pytest.mark.parametrize("batched", [False, True])
def test_refined_fixed_inner_matches_oracle(lib, cuda, engine, batched):
    """With a fixed number of float sweeps per outer step the refinement is a
    fixed sequence of roundings: bitwise equal to the oracle's refinement."""
    sizes = [(20, 14, 9), (9, 9, 9), (31, 7, 12)]
    rhs = make_batch(sizes, seed0=11)
    tol, inner, outer_max = 1e-10, 150, 40
    refs = [oracle.refined_solve(b, np.zeros_like(b), L7, 1, tol, inner, outer_max) for b in rhs]
    if batched:
        d_u = [to_dev(np.zeros_like(b)) for b in rhs]
        rc, infos = lib.jacobi_solve_batched_refined(d_u, [to_dev(b) for b in rhs], L7, 1, tol, inner, 0.0, 50,
                                                     outer_max)
        assert rc == 0
    else:
        d_u, infos = [], []
        for b in rhs:
            u = to_dev(np.zeros_like(b))
            rc, info = lib.jacobi_solve_refined_f64(to_dev(b), u, L7, 1, tol, inner, 0.0, 50, outer_max)
            assert rc == 0
            d_u.append(u)
            infos.append(info)
    for i, (u_ref, o_ref, rel_ref, st) in enumerate(refs):
        assert st == 0 and infos[i]["outer"] == o_ref and infos[i]["iters"] == o_ref * inner
        got = to_host(d_u[i])
        assert bitwise(got, u_ref), i
        # independent double residual of the returned iterate
        assert oracle.residual_norm(got, L7, 1, rhs[i]) / oracle.interior_norm(rhs[i], 1) <= tol


def test_refined_adaptive_inner_reaches_tolerance(lib, cuda, engine):
    sizes = [(40, 30, 20), (16, 16, 16), (12, 50, 7)]
    rhs = make_batch(sizes, seed0=21)
    tol = 1e-10
    d_u = [to_dev(np.zeros_like(b)) for b in rhs]
    rc, infos = lib.jacobi_solve_batched_refined(d_u, [to_dev(b) for b in rhs], L7, 1, tol, 20000, 1e-3, 25, 50)
    assert rc == 0
    for i, b in enumerate(rhs):
        got = to_host(d_u[i])
        rel = oracle.residual_norm(got, L7, 1, b) / oracle.interior_norm(b, 1)
        assert rel <= tol and abs(rel - infos[i]["rel_res"]) <= 1e-6 * tol
        u_ref, _, _, _ = oracle.jacobi_solve(b, np.zeros_like(b), L7, 1, 1e-13, 200000, 100)
        assert np.max(np.abs(got - u_ref)) / np.max(np.abs(u_ref)) < 1e-6


def test_device_wait_times_out_and_context_survives(lib, cuda):
    """Failure detection without a GPU fault: the last problem is never queued,
    so every CTA runs out of work while the batch is unfinished; the bounded
    idle wait ends the launch with STN_ETIMEOUT, and the next call works."""
    rhs = make_batch(SIZES[:4])
    try:
        lib.stencil_tune_set("sched_idle_ms", 200)
        lib.stencil_tune_set("fault_withhold_last", 1)
        d_u = [to_dev(np.zeros_like(b)) for b in rhs]
        with pytest.raises(lib.StencilError) as ei:
            lib.jacobi_solve_batched_f64(d_u, [to_dev(b) for b in rhs], L7, 1, 1e-8, 40000, 10)
        assert ei.value.code == lib.STN_ETIMEOUT
        assert "idle" in str(ei.value)
    finally:
        lib.stencil_tune_set("fault_withhold_last", 0)
        lib.stencil_tune_set("sched_idle_ms", 2000)
    d_u = [to_dev(np.zeros_like(b)) for b in rhs]
    rc, infos = lib.jacobi_solve_batched_f64(d_u, [to_dev(b) for b in rhs], L7, 1, 1e-8, 40000, 10)
    assert rc == 0 and all(i["status"] == 0 for i in infos)


def test_full_2048_mix_sampled_parity(lib, cuda):
    """The batched workload at full size, in the launch configuration the
    benchmark times: 2048 solves (per-axis sizes log-uniform in [16,128], seed
    4; b ~ N(0,1) from seed 5 * 1000003 + i; tol 1e-8, residual every 100
    sweeps) in one persistent launch.  Every solve must converge; a sample of
    eight (the six smallest and two mid-size problems) must agree with the
    oracle's Jacobi solve bitwise, with the same sweep count."""
    import torch
    sizes = [tuple(int(v) for v in s) for s in si.log_uniform_sizes(2048, 16, 128, 4)]
    tol, maxit, K = 1e-8, 10 ** 7, 100
    counts = [(nx + 2) * (ny + 2) * (nz + 2) for nx, ny, nz in sizes]
    offs = np.concatenate([[0], np.cumsum(counts)])
    d_b = torch.empty(int(offs[-1]), dtype=torch.float64, device="cuda")
    for i, (nx, ny, nz) in enumerate(sizes):
        d_b[offs[i]:offs[i + 1]] = torch.from_numpy(si.normal_interior(nx, ny, nz, 1, seed=5 * 1000003 + i).ravel())
    d_u = torch.zeros_like(d_b)
    us = [d_u[offs[i]:offs[i + 1]].view(nz + 2, ny + 2, nx + 2) for i, (nx, ny, nz) in enumerate(sizes)]
    bs = [d_b[offs[i]:offs[i + 1]].view(nz + 2, ny + 2, nx + 2) for i, (nx, ny, nz) in enumerate(sizes)]
    rc, infos = lib.jacobi_solve_batched_f64(us, bs, L7, 1, tol, maxit, K)
    assert rc == 0
    assert all(i["status"] == 0 and i["rel_res"] <= tol for i in infos)
    pts = np.array([nx * ny * nz for nx, ny, nz in sizes])
    order = np.argsort(pts, kind="stable")
    mid = [int(i) for i in order if 30_000 <= pts[i] <= 60_000][:2]
    for i in [int(j) for j in order[:6]] + mid:
        b = to_host(bs[i])
        u_ref, it_ref, rel_ref, st = oracle.jacobi_solve(b, np.zeros_like(b), L7, 1, tol, maxit, K)
        assert st == 0 and infos[i]["iters"] == it_ref, (i, sizes[i])
        assert bitwise(to_host(us[i]), u_ref), (i, sizes[i])
        assert abs(infos[i]["rel_res"] - rel_ref) <= NORM_RTOL * rel_ref


def test_graph_and_plain_launch_give_the_same_bits(lib, cuda):
    """The scheduler's persistent launch captured in a CUDA graph (knob
    batch_graph = 1, the default) and launched plainly (0): same results."""
    rhs = make_batch(SIZES, seed0=61)
    outs = []
    try:
        for v in (1, 0):
            lib.stencil_tune_set("batch_graph", v)
            d_u = [to_dev(np.zeros_like(b)) for b in rhs]
            rc, infos = lib.jacobi_solve_batched_refined(d_u, [to_dev(b) for b in rhs], L7, 1, 1e-8, 200000, 1e-2, 50,
                                                         40)
            assert rc == 0
            outs.append(([to_host(u) for u in d_u], [(i["iters"], i["outer"]) for i in infos]))
    finally:
        lib.stencil_tune_set("batch_graph", 1)
    assert outs[0][1] == outs[1][1]
    assert all(bitwise(a, b) for a, b in zip(outs[0][0], outs[1][0]))


def test_small_half_of_the_mix_refined_completes(lib, cuda):
    """The 1150 problems of the 2048-solve mix with at most 48^3 points, refined
    (tol 1e-8, inner 1e-2 every 50 sweeps), in one scheduler launch.  Their
    passes have one to a few units, so a CTA that goes back to the slot of its
    last unit often finds the next pass already published; the unit it then
    holds belongs to that pass and must be run (dropping it stalled the batch
    until the idle limit).  Every solve must converge; for a sample, the
    oracle's own residual of the result must be within tol and agree with the
    reported one, and the same problems solved on their own must give the
    same bits."""
    import torch
    sizes = [tuple(int(v) for v in s) for s in si.log_uniform_sizes(2048, 16, 128, 4)]
    pick = [i for i, (nx, ny, nz) in enumerate(sizes) if nx * ny * nz <= 48 ** 3]
    assert len(pick) == 1150
    bs = [torch.from_numpy(si.normal_interior(*sizes[i], 1, seed=5 * 1000003 + i)).cuda() for i in pick]
    us = [torch.zeros_like(b) for b in bs]
    tol, inner_tol, K, outer = 1e-8, 1e-2, 50, 40
    rc, infos = lib.jacobi_solve_batched_refined(us, bs, L7, 1, tol, 200000, inner_tol, K, outer)
    assert rc == 0
    assert all(i["status"] == 0 and i["rel_res"] <= tol for i in infos)
    sample = (0, 1, len(pick) // 2, len(pick) - 1)
    for j in sample:
        b, got = to_host(bs[j]), to_host(us[j])
        rel = oracle.residual_norm(got, L7, 1, b) / oracle.interior_norm(b, 1)
        assert rel <= tol and abs(rel - infos[j]["rel_res"]) <= 1e-6 * tol, (j, sizes[pick[j]])
    alone = [torch.zeros_like(bs[j]) for j in sample]
    rc2, infos2 = lib.jacobi_solve_batched_refined(alone, [bs[j] for j in sample], L7, 1, tol, 200000, inner_tol, K,
                                                   outer)
    assert rc2 == 0
    for n, j in enumerate(sample):
        assert bitwise(to_host(alone[n]), to_host(us[j])), (j, sizes[pick[j]])
        assert (infos2[n]["iters"], infos2[n]["outer"]) == (infos[j]["iters"], infos[j]["outer"])


def test_full_2048_mix_refined_sampled(lib, cuda):
    """The refined batched workload at full size, in the configuration the
    benchmark times: 2048 solves (the mix above), FP32 sweeps with FP64
    refinement to 1e-8 (inner tolerance 1e-2, residual every 50 inner sweeps,
    at most 40 outer steps), one persistent launch.  Every solve converges;
    for a sample (the smallest, the largest and every 256th) the oracle's own
    FP64 residual of the returned solution is within tol and matches the
    reported one, and the smallest and largest solved alone give the same
    bits."""
    import torch
    sizes = [tuple(int(v) for v in s) for s in si.log_uniform_sizes(2048, 16, 128, 4)]
    tol = 1e-8
    counts = [(nx + 2) * (ny + 2) * (nz + 2) for nx, ny, nz in sizes]
    offs = np.concatenate([[0], np.cumsum(counts)])
    d_b = torch.empty(int(offs[-1]), dtype=torch.float64, device="cuda")
    for i, (nx, ny, nz) in enumerate(sizes):
        d_b[offs[i]:offs[i + 1]] = torch.from_numpy(si.normal_interior(nx, ny, nz, 1, seed=5 * 1000003 + i).ravel())
    d_u = torch.zeros_like(d_b)
    us = [d_u[offs[i]:offs[i + 1]].view(nz + 2, ny + 2, nx + 2) for i, (nx, ny, nz) in enumerate(sizes)]
    bs = [d_b[offs[i]:offs[i + 1]].view(nz + 2, ny + 2, nx + 2) for i, (nx, ny, nz) in enumerate(sizes)]
    rc, infos = lib.jacobi_solve_batched_refined(us, bs, L7, 1, tol, 200000, 1e-2, 50, 40)
    assert rc == 0
    assert all(i["status"] == 0 and i["rel_res"] <= tol for i in infos)
    pts = np.array([nx * ny * nz for nx, ny, nz in sizes])
    small, large = int(np.argmin(pts)), int(np.argmax(pts))
    for i in sorted({small, large, *range(0, 2048, 256)}):
        b, got = to_host(bs[i]), to_host(us[i])
        rel = oracle.residual_norm(got, L7, 1, b) / oracle.interior_norm(b, 1)
        assert rel <= tol and abs(rel - infos[i]["rel_res"]) <= 1e-6 * tol, (i, sizes[i])
    alone = [torch.zeros_like(bs[i]) for i in (small, large)]
    rc2, infos2 = lib.jacobi_solve_batched_refined(alone, [bs[small], bs[large]], L7, 1, tol, 200000, 1e-2, 50, 40)
    assert rc2 == 0
    for n, i in enumerate((small, large)):
        assert bitwise(to_host(alone[n]), to_host(us[i])), (i, sizes[i])
        assert (infos2[n]["iters"], infos2[n]["outer"]) == (infos[i]["iters"], infos[i]["outer"])
