"""residual_norm_f64_noalloc: the residual norm for callers that cannot let
the library allocate (its scratch is a fixed device array inside the library).

It must give the same norm as residual_norm_f64 on the same device grids, on
consecutive calls with different inputs (the shared scratch keeps the last
call's contents, which must not leak into the next result).  This file is
collected last so that, run with -x, every other test has already run.
"""
import ctypes

import numpy as np
import pytest

import stencil_inputs as si

NORM_RTOL = 1e-12


def _abi_call(lib, u, b, nx, ny, nz, coeffs, r):
    arr = (ctypes.c_double * len(coeffs))(*coeffs)
    out = ctypes.c_double(-1.0)
    rc = lib.lib().residual_norm_f64_noalloc(u, b, nx, ny, nz, ctypes.cast(arr, ctypes.POINTER(ctypes.c_double)),
                                             r, ctypes.byref(out), None)
    return rc, out.value


@pytest.mark.gpu
def test_noalloc_matches_residual_norm_on_consecutive_calls(lib, cuda):
    import torch
    cases = [((96, 40, 33), 1, si.LAPLACE7, True), ((37, 19, 11), 2, (0.2, 0.1, 0.0333), False),
             ((64, 64, 64), 1, si.LAPLACE7, False)]
    for (nx, ny, nz), r, c, with_b in cases:
        u = torch.from_numpy(si.uniform_interior(nx, ny, nz, r, seed=nx + ny)).cuda()
        b = torch.from_numpy(si.normal_interior(nx, ny, nz, r, seed=nz)).cuda() if with_b else None
        ref = lib.residual_norm_f64(u, c, r, b=b)
        for _ in range(2):  # two calls in a row on the shared scratch
            torch.cuda.synchronize()
            rc, got = _abi_call(lib, u.data_ptr(), None if b is None else b.data_ptr(), nx, ny, nz, c, r)
            assert rc == lib.STN_OK, lib.last_error()
            assert abs(got - ref) <= NORM_RTOL * ref, (got, ref)


@pytest.mark.gpu
def test_noalloc_rejects_host_grids_and_oversize(lib, cuda):
    u = si.uniform_interior(8, 8, 8, 1, seed=1)
    rc, _ = _abi_call(lib, u.ctypes.data, None, 8, 8, 8, si.LAPLACE7, 1)
    assert rc == lib.STN_EINVAL and "device grids only" in lib.last_error()
    # 8192 x 8200 plane: more partial sums than the scratch holds; rejected before any GPU work
    rc, _ = _abi_call(lib, 0x7F0000000000, None, 8192, 8200, 4, si.LAPLACE7, 1)
    assert rc == lib.STN_EINVAL and "65536" in lib.last_error()
