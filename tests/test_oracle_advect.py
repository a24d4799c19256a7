"""Pins for the oracle's multi-field advection stand-in (flux-form centred
advection of a field q by the velocity (u, v, w); a synthetic stand-in for
the paper's pw-advection / tra-adv workloads, whose formulas the paper does
not give).  No GPU.

Checked against: an independent numpy evaluation of the definition
(array slicing, same operation order, so bitwise), exact results for linear
fields (the centred flux form differentiates u^2 exactly), conservation (the
interior sum telescopes to the boundary fluxes), and the symmetry of the
three axes (a transposed problem gives the transposed tendency).
"""
import numpy as np
import pytest

import oracle
import stencil_inputs as si


def numpy_advect(u, v, w, q, c):
    """The definition with numpy slicing (z, y, x array axes)."""
    s = np.zeros_like(u)
    core = (slice(1, -1),) * 3
    t = []
    vel = {2: u, 1: v, 0: w}           # array axis -> velocity component
    coef = {2: c[0], 1: c[1], 0: c[2]}
    for ax in (2, 1, 0):
        V = vel[ax]

        def sh(a, d):
            idx = [slice(1, -1)] * 3
            idx[ax] = slice(1 + d, a.shape[ax] - 1 + d)
            return a[tuple(idx)]
        fm = (sh(V, -1) + sh(V, 0)) * (sh(q, -1) + sh(q, 0))
        fp = (sh(V, 0) + sh(V, 1)) * (sh(q, 0) + sh(q, 1))
        t.append(coef[ax] * (fm - fp))
    s[core] = (t[0] + t[1]) + t[2]
    return s


def fields(nx, ny, nz, seed, dtype=np.float64):
    g = [si.uniform_full(nx, ny, nz, 1, seed=seed + i, lo=-1.0, hi=1.0, dtype=dtype) for i in range(4)]
    return g


@pytest.mark.parametrize("shape", [(5, 4, 3), (7, 6, 9), (1, 1, 1), (12, 3, 5)])
def test_matches_numpy_definition(shape):
    u, v, w, q = fields(*shape, seed=sum(shape))
    c = (0.25, 0.3, 0.15)
    got = oracle.advect(u, v, w, q, c)
    assert np.array_equal(got, numpy_advect(u, v, w, q, c))
    # the pw-like case: the velocity advecting itself
    assert np.array_equal(oracle.advect(u, v, w, u, c), numpy_advect(u, v, w, u, c))


def test_float_is_float_arithmetic():
    u, v, w, q = fields(6, 5, 4, seed=3, dtype=np.float32)
    c = (0.25, 0.25, 0.25)
    got = oracle.advect(u, v, w, q, c)
    assert got.dtype == np.float32
    assert np.array_equal(got, numpy_advect(u, v, w, q, np.float32(c)))


def test_constant_fields_have_no_tendency():
    shape = si.padded_shape(6, 5, 4, 1)
    u, v, w, q = (np.full(shape, x) for x in (0.7, -1.3, 2.1, 0.9))
    assert np.all(oracle.advect(u, v, w, q, (0.25, 0.25, 0.25)) == 0.0)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_linear_self_advection_is_exact(axis):
    """V_a = alpha * x_a (halo included), the other components 0, q = V_a: the
    tendency is c_a * (-8 alpha^2 x_a) exactly, i.e. -d(V^2)/dx with c = 1/4."""
    nx, ny, nz = 7, 6, 5
    alpha, c = 3.0, (0.25, 0.5, 0.125)
    k, j, i = np.meshgrid(np.arange(nz + 2), np.arange(ny + 2), np.arange(nx + 2), indexing="ij")
    x = (i, j, k)[axis].astype(np.float64)
    vel = [np.zeros_like(x) for _ in range(3)]
    vel[axis] = alpha * x
    s = oracle.advect(*vel, vel[axis], c)
    core = (slice(1, -1),) * 3
    assert np.array_equal(s[core], (c[axis] * (-8 * alpha ** 2 * x))[core])


def test_interior_sum_telescopes_to_boundary_fluxes():
    """Integer-valued fields keep every flux exact, so the sum of the tendency
    over the interior equals the boundary-face fluxes exactly."""
    nx, ny, nz = 6, 5, 4
    g = si.rng(7)
    u, v, w, q = (g.integers(-3, 4, size=si.padded_shape(nx, ny, nz, 1)).astype(np.float64) for _ in range(4))
    s = oracle.advect(u, v, w, q, (1.0, 1.0, 1.0))
    total = 0.0
    for V, ax in ((u, 2), (v, 1), (w, 0)):
        lo = [slice(1, -1)] * 3
        hi = [slice(1, -1)] * 3
        lo0, lo1, hi0, hi1 = list(lo), list(lo), list(hi), list(hi)
        lo0[ax], lo1[ax] = slice(0, 1), slice(1, 2)
        n = V.shape[ax]
        hi0[ax], hi1[ax] = slice(n - 2, n - 1), slice(n - 1, n)
        f_in = (V[tuple(lo0)] + V[tuple(lo1)]) * (q[tuple(lo0)] + q[tuple(lo1)])
        f_out = (V[tuple(hi0)] + V[tuple(hi1)]) * (q[tuple(hi0)] + q[tuple(hi1)])
        total += f_in.sum() - f_out.sum()
    assert s[1:-1, 1:-1, 1:-1].sum() == total


def test_axes_are_symmetric():
    """Transposing x and z (and swapping u with w, c_x with c_z) transposes the tendency."""
    u, v, w, q = fields(5, 4, 6, seed=11)
    c = (0.2, 0.3, 0.4)
    s = oracle.advect(u, v, w, q, c)
    tr = lambda a: np.ascontiguousarray(a.transpose(2, 1, 0))
    s_t = oracle.advect(tr(w), tr(v), tr(u), tr(q), (c[2], c[1], c[0]))
    # the per-axis terms are added in the order x, y, z, so compare within rounding
    assert np.allclose(tr(s), s_t, rtol=0, atol=1e-14)
