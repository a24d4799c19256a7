"""The multi-core host path (libstencil_host.so) against the oracle, on CPU.

Sweeps and advection tendencies follow the canonical order, so they must equal
the oracle bitwise for every thread count; residual norms sum per-row partials
in row order, so they must be the same bits for every thread count and within
the recursive summation bound of the oracle's own norm.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import stencil_inputs as si

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def host():
    import paper_2409_18824_gb300.host as h
    return h


def bitwise(a, b):
    return a.shape == b.shape and np.array_equal(a.view(np.uint64), b.view(np.uint64))


def declared_host_functions():
    src = open(os.path.join(ROOT, "include", "stencil_host.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:int|char|double)\s*\**\s*(\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_symbol(host):
    names = declared_host_functions()
    assert "stencil_host_sweep2d_f64" in names and "stencil_host_sweep_f64" in names
    missing = [n for n in names if not hasattr(host.lib(), n)]
    assert not missing and set(names) <= set(host.SIGNATURES)
    assert host.threads() >= 1


def test_gpu_library_does_not_call_the_host_path():
    """libstencil.so must not reach the host library (it is no fallback)."""
    import glob
    srcs = glob.glob(os.path.join(ROOT, "paper_2409_18824_gb300", "csrc", "*"))
    for path in srcs:
        assert "stencil_host" not in open(path, errors="replace").read(), path


def nonzero_halo(u, r, seed):
    rng = np.random.default_rng(seed)
    v = u.copy()
    mask = np.ones(u.shape, dtype=bool)
    mask[tuple(slice(r, m - r) for m in u.shape)] = False
    v[mask] = rng.uniform(-1, 1, size=int(mask.sum()))
    return v


CASES3 = [((37, 19, 11), 1, si.LAPLACE7), ((20, 9, 30), 2, (0.1, 0.1, 0.025)), ((1, 1, 1), 1, (0.3, 0.1)),
          ((33, 17, 5), 2, (0.0, 0.125, 0.0625)), ((64, 3, 2), 1, (0.05, 0.15))]


@pytest.mark.parametrize("shape,r,c", CASES3)
@pytest.mark.parametrize("iters", [0, 1, 2, 7])
def test_sweep3d_bitwise_for_every_thread_count(host, shape, r, c, iters):
    nx, ny, nz = shape
    u0 = nonzero_halo(si.uniform_interior(nx, ny, nz, r, seed=31, lo=-1, hi=1), r, 32)
    ref = oracle.stencil_sweep(u0, c, r, iters)
    for T in (1, 2, 3, 8, 64):
        a, out = u0.copy(), np.zeros_like(u0)
        host.stencil_host_sweep_f64(a, out, c, r, iters, nthreads=T)
        assert bitwise(out, ref), (T, iters)


@pytest.mark.parametrize("shape,r,c", [((37, 19), 1, si.LAPLACE5), ((50, 23), 2, (0.1, 0.15, 0.05)),
                                       ((1, 1), 1, (0.2, 0.2)), ((128, 4), 1, si.LAPLACE5)])
@pytest.mark.parametrize("iters", [0, 1, 6, 13])
def test_sweep2d_bitwise_for_every_thread_count(host, shape, r, c, iters):
    nx, ny = shape
    u0 = nonzero_halo(si.uniform_interior2d(nx, ny, r, seed=33), r, 34)
    ref = oracle.stencil_sweep2d(u0, c, r, iters)
    for T in (1, 2, 5, 0):
        a, out = u0.copy(), np.zeros_like(u0)
        host.stencil_host_sweep2d_f64(a, out, c, r, iters, nthreads=T)
        assert bitwise(out, ref), (T, iters)


def test_the_papers_2d_jacobi_at_full_size(host):
    """The paper's jacobi grid (1024^2, c = {0, 1/4}), 50 sweeps on 16 threads,
    bitwise the oracle."""
    u0 = si.uniform_interior2d(1024, 1024, 1, seed=7)
    ref = oracle.stencil_sweep2d(u0, si.LAPLACE5, 1, 50)
    out = np.zeros_like(u0)
    host.stencil_host_sweep2d_f64(u0.copy(), out, si.LAPLACE5, 1, 50, nthreads=16)
    assert bitwise(out, ref)


@pytest.mark.parametrize("with_b", [False, True])
def test_norms_match_the_oracle_and_not_the_thread_count(host, with_b):
    nx, ny, nz, r, c = 45, 30, 21, 2, (0.1, 0.1, 0.025)
    u = nonzero_halo(si.uniform_interior(nx, ny, nz, r, seed=35, lo=-1, hi=1), r, 36)
    b = si.normal_interior(nx, ny, nz, r, seed=37) if with_b else None
    ref = oracle.residual_norm(u, c, r, b)
    n = nx * ny * nz
    got = [host.stencil_host_residual_norm_f64(u, c, r, b=b, nthreads=T) for T in (1, 2, 7, 0)]
    assert len({x.hex() for x in got}) == 1
    assert abs(got[0] - ref) <= n * 2.0 ** -53 * ref
    # 2-D
    u2 = si.uniform_interior2d(77, 41, 1, seed=38)
    b2 = si.normal_interior(77, 41, 1, 1, seed=39)[1] if with_b else None  # one plane of a 3-D draw
    ref2 = oracle.residual_norm2d(u2, si.LAPLACE5, 1, b2)
    got2 = [host.stencil_host_residual_norm2d_f64(u2, si.LAPLACE5, 1, b=b2, nthreads=T) for T in (1, 3, 16)]
    assert len({x.hex() for x in got2}) == 1
    assert abs(got2[0] - ref2) <= 77 * 41 * 2.0 ** -53 * ref2


def test_rejects_bad_arguments(host):
    so = host.lib()
    u = np.zeros((5, 5, 5))
    o = np.zeros_like(u)
    c = (ctypes.c_double * 3)(0.0, 1.0 / 6.0, 0.0)
    cp = ctypes.cast(c, ctypes.POINTER(ctypes.c_double))
    ptr, optr = u.ctypes.data, o.ctypes.data
    assert so.stencil_host_sweep_f64(ptr, optr, 3, 3, 3, cp, 1, 1, 0) == 0
    for args in ((None, optr, 3, 3, 3, cp, 1, 1, 0), (ptr, None, 3, 3, 3, cp, 1, 1, 0),
                 (ptr, optr, 0, 3, 3, cp, 1, 1, 0), (ptr, optr, 3, 3, 3, cp, 3, 1, 0),
                 (ptr, optr, 3, 3, 3, cp, 1, -1, 0), (ptr, optr, 3, 3, 3, cp, 1, 1, -2),
                 (ptr, optr, 3, 3, 3, None, 1, 1, 0), (ptr, ptr + 8, 3, 3, 3, cp, 1, 1, 0)):
        assert so.stencil_host_sweep_f64(*args) == -1, args
    assert "invalid argument" in so.stencil_host_last_error().decode()
    v = ctypes.c_double()
    assert so.stencil_host_residual_norm_f64(ptr, None, 3, 3, 3, cp, 1, None, 0) == -1
    assert so.stencil_host_residual_norm2d_f64(None, None, 3, 3, cp, 1, ctypes.byref(v), 0) == -1
    assert so.stencil_host_sweep2d_f64(ptr, optr, 3, 0, cp, 1, 1, 0) == -1


def random_grid(nx, ny, nz, seed):
    return np.random.default_rng(seed).uniform(-1, 1, size=(nz + 2, ny + 2, nx + 2))


@pytest.mark.parametrize("shape", [(37, 19, 11), (1, 1, 1), (64, 3, 2), (5, 40, 9)])
def test_advect_self_and_tracers_bitwise_for_every_thread_count(host, shape):
    """The host advection gives the oracle's bits (every value of every grid,
    halos included, random) in both modes, for any thread count; only the
    interior of each output is written."""
    nx, ny, nz = shape
    u, v, w = (random_grid(nx, ny, nz, 80 + m) for m in range(3))
    c = (0.25, 0.125, 0.375)
    ref_self = [oracle.advect(u, v, w, f, c) for f in (u, v, w)]
    tracers = [random_grid(nx, ny, nz, 90 + m) for m in range(5)]
    ref_tr = [oracle.advect(u, v, w, f, c) for f in tracers]
    for T in (1, 2, 3, 16):
        outs = [np.full_like(u, 7.0) for _ in range(3)]
        host.stencil_host_advect_f64(u, v, w, outs, c, nthreads=T)
        for o, ref in zip(outs, ref_self):
            assert bitwise(o[1:-1, 1:-1, 1:-1].copy(), ref[1:-1, 1:-1, 1:-1].copy())
            halo = np.ones(o.shape, dtype=bool)
            halo[1:-1, 1:-1, 1:-1] = False
            assert np.all(o[halo] == 7.0)
        outs = [np.zeros_like(u) for _ in tracers]
        host.stencil_host_advect_f64(u, v, w, outs, c, q=tracers, nthreads=T)
        for o, ref in zip(outs, ref_tr):
            assert bitwise(o, ref)


def test_advect_rejects_bad_arguments(host):
    u = np.zeros((4, 5, 6))
    v, w, q = np.zeros_like(u), np.zeros_like(u), np.zeros_like(u)
    s = [np.zeros_like(u) for _ in range(3)]
    c = (0.25, 0.25, 0.25)
    with pytest.raises(host.HostStencilError):
        host.stencil_host_advect_f64(u, v, w, s, c, q=[q] * 7)  # nq > 6
    with pytest.raises(host.HostStencilError):
        host.stencil_host_advect_f64(u, v, w, [u, s[1], s[2]], c)  # output = an input
    with pytest.raises(host.HostStencilError):
        host.stencil_host_advect_f64(u, v, w, [s[0], s[0], s[2]], c)  # two outputs alias
    with pytest.raises(host.HostStencilError):
        host.stencil_host_advect_f64(u, v, w, s, (0.25, float("nan"), 0.25))
    so = host.lib()
    assert so.stencil_host_advect_f64(None, None, None, None, 0, None, 4, 3, 2, None, 0) == -1


def test_binding_refuses_mismatched_grids(host):
    """Every grid of a call must have the first grid's shape (the extents come
    from it): a smaller output, source term or field is refused before the
    library could run past it."""
    u = np.zeros((6, 7, 8))
    c = (0.0, 1.0 / 6.0)
    with pytest.raises(ValueError):
        host.stencil_host_sweep_f64(u, np.zeros((6, 7, 7)), c, 1, 2)
    with pytest.raises(ValueError):
        host.stencil_host_residual_norm_f64(u, c, 1, b=np.zeros((5, 7, 8)))
    with pytest.raises(ValueError):
        host.stencil_host_sweep2d_f64(np.zeros((6, 7)), np.zeros((7, 6)), (0.0, 0.25), 1, 1)
    with pytest.raises(ValueError):
        host.stencil_host_advect_f64(u, u.copy(), np.zeros((6, 7, 9)), [np.zeros_like(u)] * 3, (0.1, 0.1, 0.1))
    with pytest.raises(TypeError):
        host.stencil_host_sweep_f64(u, np.zeros((6, 7, 8), dtype=np.float32), c, 1, 2)
