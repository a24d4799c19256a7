"""residual_norm_f64_noalloc: the residual norm for callers that cannot let
the library allocate device memory (a serving process whose memory is all
handed to its own pools, code that must not call cudaMalloc because it can
synchronise the device, loops with no way to report an allocation failure).
Its scratch is a fixed device array inside the library.

Checked here through the C ABI, on two calls in a row with different inputs
(the shared scratch keeps the last call's contents, which must not leak into
the next result):
  * the same bits as residual_norm_f64, which runs the same kernels in the same
    fixed reduction order;
  * within 1e-12 relative of the oracle's residual norm;
  * at the largest plan the array accepts (exactly 65536 partial sums) and one
    row past it, which is refused before any GPU work;
  * no device memory taken by a call on a stream the library has not seen.
This file is collected last so that, run with -x, every other test has
already run.
"""
import ctypes

import numpy as np
import pytest

import oracle
import stencil_inputs as si

NORM_RTOL = 1e-12
SCRATCH_PARTIALS = 65536


def _abi_call(lib, u, b, nx, ny, nz, coeffs, r, stream=None):
    arr = (ctypes.c_double * len(coeffs))(*coeffs)
    out = ctypes.c_double(-1.0)
    rc = lib.lib().residual_norm_f64_noalloc(u, b, nx, ny, nz, ctypes.cast(arr, ctypes.POINTER(ctypes.c_double)),
                                             r, ctypes.byref(out), stream)
    return rc, out.value


def _check_case(lib, nx, ny, nz, r, c, with_b, seed):
    import torch
    uh = si.uniform_interior(nx, ny, nz, r, seed=seed)
    bh = si.normal_interior(nx, ny, nz, r, seed=seed + 1) if with_b else None
    want = oracle.residual_norm(uh, c, r, b=bh)
    u = torch.from_numpy(uh).cuda()
    b = torch.from_numpy(bh).cuda() if with_b else None
    ref = lib.residual_norm_f64(u, c, r, b=b)
    for _ in range(2):  # two calls in a row on the shared scratch
        torch.cuda.synchronize()
        rc, got = _abi_call(lib, u.data_ptr(), None if b is None else b.data_ptr(), nx, ny, nz, c, r)
        assert rc == lib.STN_OK, lib.last_error()
        assert got == ref, (got, ref)
        assert abs(got - want) <= NORM_RTOL * want, (got, want)
    return u, b


@pytest.mark.gpu
def test_noalloc_matches_residual_norm_and_oracle_on_consecutive_calls(lib, cuda):
    cases = [((96, 40, 33), 1, si.LAPLACE7, True), ((37, 19, 11), 2, (0.2, 0.1, 0.0333), False),
             ((64, 64, 64), 1, si.LAPLACE7, False), ((130, 7, 300), 2, (0.1, 0.15, 0.05), True)]
    for (nx, ny, nz), r, c, with_b in cases:
        _check_case(lib, nx, ny, nz, r, c, with_b, seed=nx + ny)


@pytest.mark.gpu
def test_noalloc_python_binding(lib, cuda):
    import torch
    nx, ny, nz = 50, 21, 17
    uh = si.uniform_interior(nx, ny, nz, 1, seed=11)
    u = torch.from_numpy(uh).cuda()
    got = lib.residual_norm_f64_noalloc(u, si.LAPLACE7, 1)
    assert got == lib.residual_norm_f64(u, si.LAPLACE7, 1)
    want = oracle.residual_norm(uh, si.LAPLACE7, 1)
    assert abs(got - want) <= NORM_RTOL * want


@pytest.mark.gpu
def test_noalloc_at_the_scratch_limit(lib, cuda):
    # A single-plane grid of 4096 x ny: one block per 32 x 8 tile of the
    # (i, j) plane and one k chunk.  Find the largest ny whose plan fits the
    # array exactly or just under it, run it, then one tile row more.
    nx, nz = 4096, 1
    best = None
    for ny in range(4000, 4200):
        q = lib.stencil_plan_query("sweep", nx, ny, nz, 8, 1)
        nb = q["grid_x"] * q["grid_y"] * q["grid_z"]
        if nb <= SCRATCH_PARTIALS:
            best = (ny, nb)
        else:
            over = ny
            break
    assert best is not None and best[1] > SCRATCH_PARTIALS - 600, best
    ny, nb = best
    _check_case(lib, nx, ny, nz, 1, si.LAPLACE7, True, seed=5)
    # past the limit: refused before any GPU work (a dummy address is never read)
    rc, _ = _abi_call(lib, 0x7F0000000000, None, nx, over, nz, si.LAPLACE7, 1)
    assert rc == lib.STN_EINVAL and "65536" in lib.last_error()


@pytest.mark.gpu
def test_noalloc_takes_no_device_memory_on_a_new_stream(lib, cuda):
    # residual_norm_f64 keeps a workspace per (device, stream); this call must
    # take none, so a stream it has never seen costs no device memory.
    import torch
    nx, ny, nz = 200, 180, 160
    u = torch.from_numpy(si.uniform_interior(nx, ny, nz, 1, seed=3)).cuda()
    ref = lib.residual_norm_f64(u, si.LAPLACE7, 1)
    torch.cuda.synchronize()
    for _ in range(2):
        s = torch.cuda.Stream()
        free0, _ = torch.cuda.mem_get_info()
        rc, got = _abi_call(lib, u.data_ptr(), None, nx, ny, nz, si.LAPLACE7, 1, ctypes.c_void_p(s.cuda_stream))
        free1, _ = torch.cuda.mem_get_info()
        assert rc == lib.STN_OK, lib.last_error()
        assert got == ref
        assert free1 == free0, (free0, free1)


@pytest.mark.gpu
def test_noalloc_rejects_host_grids_and_oversize(lib, cuda):
    u = si.uniform_interior(8, 8, 8, 1, seed=1)
    rc, _ = _abi_call(lib, u.ctypes.data, None, 8, 8, 8, si.LAPLACE7, 1)
    assert rc == lib.STN_EINVAL and "device grids only" in lib.last_error()
    # 8192 x 8200 plane: more partial sums than the scratch holds; rejected before any GPU work
    rc, _ = _abi_call(lib, 0x7F0000000000, None, 8192, 8200, 4, si.LAPLACE7, 1)
    assert rc == lib.STN_EINVAL and "65536" in lib.last_error()
