"""The sweep autotuner and its cache on the GPU.

A cache entry must steer the launches of sweeps on its extents (the plan in
effect is read back through the read-only knobs), every configuration it can
name must give the oracle's iterates bitwise, the knobs must take precedence
over it, and the autotuner must return a configuration at least as fast as
the built-in plan in its own timing.
"""
import numpy as np
import pytest

import oracle
import stencil_inputs as si

pytestmark = pytest.mark.gpu


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def to_host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def bitwise(a, b):
    return a.shape == b.shape and np.array_equal(a.view(f"u{a.itemsize}"), b.view(f"u{b.itemsize}"))


@pytest.fixture(autouse=True)
def clean_cache(lib):
    lib.stencil_tune_cache_clear()
    yield
    lib.stencil_tune_cache_clear()


def plan_in_effect(lib):
    return (lib.stencil_tune_get("last_star_variant"), lib.stencil_tune_get("last_star_chunks"),
            lib.stencil_tune_get("last_temporal_depth"))


def sweep(lib, u0, coeffs, r, iters):
    d_out = to_dev(np.zeros_like(u0))
    fn = lib.stencil_sweep_f64 if u0.dtype == np.float64 else lib.stencil_sweep_f32
    fn(to_dev(u0), d_out, coeffs, r, iters)
    return to_host(d_out)


@pytest.mark.parametrize("variant,chunks,depth", [(0, 1, 1), (0, 7, 1), (1, 2, 1), (1, 25, 1), (2, 4, 1),
                                                  (2, 13, 1), (3, 1, 1), (3, 13, 1), (0, 4, 2), (1, 3, 3),
                                                  (2, 5, 4), (3, 4, 2)])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_cache_entry_steers_the_plan_and_keeps_the_bits(lib, cuda, variant, chunks, depth, dtype):
    nx, ny, nz, r, iters = 70, 45, 100, 1, 7
    u0 = si.uniform_interior(nx, ny, nz, r, seed=21, dtype=dtype)
    lib.stencil_tune_cache_put(nx, ny, nz, np.dtype(dtype).itemsize, r, variant, chunks, depth)
    got = sweep(lib, u0, si.LAPLACE7, r, iters)
    # 7 sweeps: whole temporal passes, then single sweeps on the entry's kernel
    # (the last launch is a single sweep unless depth divides 7)
    v, c, d = plan_in_effect(lib)
    assert d == depth
    if iters % depth:
        assert (v, c) == (variant, chunks)
    assert bitwise(got, oracle.stencil_sweep(u0, si.LAPLACE7, r, iters))


@pytest.mark.parametrize("variant,chunks", [(0, 3), (1, 5), (2, 9), (3, 4)])
def test_cache_entry_radius2_norm_and_solve(lib, cuda, variant, chunks):
    """Radius 2 with a centre term: sweeps bitwise, the fused norm within
    1e-12 of the oracle's, and a Jacobi solve with the oracle's sweep count."""
    nx, ny, nz, r = 33, 40, 50, 2
    c = (0.1, 0.1, 0.025)
    lib.stencil_tune_cache_put(nx, ny, nz, 8, r, variant, chunks, 1)
    u0 = si.uniform_interior(nx, ny, nz, r, seed=22)
    got = sweep(lib, u0, c, r, 5)
    assert plan_in_effect(lib)[:2] == (variant, chunks)
    assert bitwise(got, oracle.stencil_sweep(u0, c, r, 5))
    norm = lib.residual_norm_f64(to_dev(got), c, r)
    ref = oracle.residual_norm(got, c, r)
    assert abs(norm - ref) <= 1e-12 * ref
    b = si.normal_interior(nx, ny, nz, r, seed=23)
    d_u = to_dev(np.zeros_like(b))
    rc, info = lib.jacobi_solve_f64(to_dev(b), d_u, c, r, 1e-10, 5000, 7)
    u_ref, it_ref, rel_ref, st = oracle.jacobi_solve(b, np.zeros_like(b), c, r, 1e-10, 5000, 7)
    assert rc == 0 and st == 0 and info["iters"] == it_ref
    assert bitwise(to_host(d_u), u_ref)


def test_knobs_take_precedence_over_the_cache(lib, cuda):
    nx, ny, nz, r = 40, 40, 40, 1
    u0 = si.uniform_interior(nx, ny, nz, r, seed=24)
    lib.stencil_tune_cache_put(nx, ny, nz, 8, r, 2, 4, 2)
    try:
        lib.stencil_tune_set("star_variant", 1)
        lib.stencil_tune_set("star_chunks", 3)
        lib.stencil_tune_set("temporal_depth", 1)
        got = sweep(lib, u0, si.LAPLACE7, r, 3)
        assert plan_in_effect(lib) == (1, 3, 1)
    finally:
        lib.stencil_tune_set("star_variant", -1)
        lib.stencil_tune_set("star_chunks", 0)
        lib.stencil_tune_set("temporal_depth", 0)
    assert bitwise(got, oracle.stencil_sweep(u0, si.LAPLACE7, r, 3))
    # other extents are not affected by the entry
    u1 = si.uniform_interior(nx, ny, nz + 1, r, seed=24)
    sweep(lib, u1, si.LAPLACE7, r, 1)
    assert plan_in_effect(lib)[2] == 1


@pytest.mark.parametrize("dtype,r,coeffs", [(np.float64, 1, None), (np.float32, 2, (0.1, 0.1, 0.025))])
def test_autotune_picks_a_configuration_and_the_sweeps_use_it(lib, cuda, dtype, r, coeffs):
    nx, ny, nz = 96, 80, 72
    esize = np.dtype(dtype).itemsize
    e = lib.stencil_autotune_sweep(nx, ny, nz, esize, r, coeffs)
    assert 0 <= e["variant"] <= 3 and e["chunks"] >= 1 and 1 <= e["depth"] <= 4
    assert e["glups"] > 0 and e["default_glups"] > 0 and e["glups"] >= e["default_glups"]
    assert (e["nx"], e["ny"], e["nz"], e["esize"], e["radius"]) == (nx, ny, nz, esize, r)
    cached = lib.stencil_tune_cache_get(nx, ny, nz, esize, r)
    assert cached is not None and (cached["variant"], cached["chunks"], cached["depth"]) == (
        e["variant"], e["chunks"], e["depth"])
    c = coeffs if coeffs is not None else si.LAPLACE7
    u0 = si.uniform_interior(nx, ny, nz, r, seed=25, dtype=dtype)
    iters = 12 * e["depth"] + 1  # ends on a single sweep
    got = sweep(lib, u0, c, r, iters)
    assert plan_in_effect(lib) == (e["variant"], e["chunks"], e["depth"])
    assert bitwise(got, oracle.stencil_sweep(u0, c, r, iters))


def test_autotune_writes_the_cache_file(lib, cuda, tmp_path, monkeypatch):
    path = tmp_path / "tuned.json"
    monkeypatch.setenv("STN_TUNE_CACHE", str(path))
    e = lib.stencil_autotune_sweep(48, 40, 30, 8, 1)
    lib.stencil_tune_cache_clear()
    assert lib.stencil_tune_cache_load(str(path)) == 1
    got = lib.stencil_tune_cache_get(48, 40, 30, 8, 1)
    assert (got["variant"], got["chunks"], got["depth"]) == (e["variant"], e["chunks"], e["depth"])
