"""Parity of the multi-field advection stand-in with the oracle (bitwise:
both follow the same operation order, and a face flux shared by two cells is
the same number from either side)."""
import numpy as np
import pytest

import oracle
import stencil_inputs as si

pytestmark = pytest.mark.gpu

C = (0.25, 0.2, 0.125)


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def bitwise(a, b):
    return a.shape == b.shape and np.array_equal(a.view(f"u{a.itemsize}"), b.view(f"u{b.itemsize}"))


SHAPES = [(64, 40, 33), (37, 19, 11), (1, 1, 1), (31, 9, 70), (30, 8, 5), (61, 17, 130), (2, 3, 2)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_self_advection_bitwise(lib, cuda, shape, dtype):
    """The pw-like case: (u, v, w) advect themselves."""
    nx, ny, nz = shape
    u, v, w = (si.uniform_full(nx, ny, nz, 1, seed=nx + i, lo=-1, hi=1, dtype=dtype) for i in range(3))
    outs = [dev(np.zeros_like(u)) for _ in range(3)]
    fn = lib.advect_f64 if dtype == np.float64 else lib.advect_f32
    fn(dev(u), dev(v), dev(w), outs, C)
    for m, q in enumerate((u, v, w)):
        assert bitwise(host(outs[m]), oracle.advect(u, v, w, q, C)), m


@pytest.mark.parametrize("nq", [1, 2, 3, 5, 6])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_tracer_advection_bitwise(lib, cuda, nq, dtype):
    """The tra-adv-like case: nq tracer fields (groups of up to three per launch)."""
    nx, ny, nz = 45, 23, 38
    u, v, w = (si.uniform_full(nx, ny, nz, 1, seed=7 + i, lo=-1, hi=1, dtype=dtype) for i in range(3))
    qs = [si.uniform_full(nx, ny, nz, 1, seed=20 + m, lo=0, hi=2, dtype=dtype) for m in range(nq)]
    outs = [dev(np.full_like(u, 7.0)) for _ in range(nq)]
    fn = lib.advect_f64 if dtype == np.float64 else lib.advect_f32
    fn(dev(u), dev(v), dev(w), outs, C, q=[dev(q) for q in qs])
    for m, q in enumerate(qs):
        got = host(outs[m])
        ref = oracle.advect(u, v, w, q, C)
        assert bitwise(got[1:-1, 1:-1, 1:-1].copy(), ref[1:-1, 1:-1, 1:-1].copy()), m
        # the output halo is not written
        halo = np.ones(got.shape, dtype=bool)
        halo[1:-1, 1:-1, 1:-1] = False
        assert np.all(got[halo] == 7.0)


def test_linear_field_exact_on_gpu(lib, cuda):
    """u = 3 x (halo included), v = w = 0: the tendency of u is -8 * 9 * x / 4."""
    nx, ny, nz = 50, 9, 7
    k, j, i = np.meshgrid(np.arange(nz + 2), np.arange(ny + 2), np.arange(nx + 2), indexing="ij")
    u = 3.0 * i.astype(np.float64)
    z = np.zeros_like(u)
    outs = [dev(np.zeros_like(u)) for _ in range(3)]
    lib.advect_f64(dev(u), dev(z), dev(z), outs, (0.25, 0.25, 0.25))
    got = host(outs[0])
    assert np.array_equal(got[1:-1, 1:-1, 1:-1], (0.25 * (-8 * 9.0 * i))[1:-1, 1:-1, 1:-1])
    assert np.all(host(outs[1]) == 0) and np.all(host(outs[2]) == 0)
