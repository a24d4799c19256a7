"""Property tests over random tiny grids (hypothesis; CPU only).

For random extents (1..6 per axis), radius, coefficients, halo values and
source terms: the oracle's sweep and residual norm equal the dense operator
assembled from the definition (brute force, written here independently of
the oracle), and the multi-core host library gives the oracle's bits for a
random thread count.
"""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402

extent = st.integers(min_value=1, max_value=6)
coef = st.floats(min_value=-1.0, max_value=1.0, allow_nan=False, allow_infinity=False, width=64)


def dense_S(nx, ny, nz, r, c):
    """Rows: interior points (k, j, i order); columns: padded points.  Row p
    holds c0 at p and c_d at the 6 points at distance d along the axes."""
    NX, NY, NZ = nx + 2 * r, ny + 2 * r, nz + 2 * r
    S = np.zeros((nx * ny * nz, NX * NY * NZ))
    row = 0
    for k in range(r, nz + r):
        for j in range(r, ny + r):
            for i in range(r, nx + r):
                p = (k * NY + j) * NX + i
                S[row, p] += c[0]
                for d in range(1, r + 1):
                    for q in (p - d, p + d, p - d * NX, p + d * NX, p - d * NX * NY, p + d * NX * NY):
                        S[row, q] += c[d]
                row += 1
    return S


@settings(max_examples=60, deadline=None)
@given(nx=extent, ny=extent, nz=extent, r=st.sampled_from([1, 2]), c=st.lists(coef, min_size=3, max_size=3),
       seed=st.integers(0, 2 ** 31 - 1), with_b=st.booleans())
def test_oracle_sweep_and_residual_equal_the_dense_operator(nx, ny, nz, r, c, seed, with_b):
    c = c[:r + 1]
    rng = np.random.default_rng(seed)
    shape = (nz + 2 * r, ny + 2 * r, nx + 2 * r)
    u = rng.uniform(-1, 1, size=shape)  # random halo included
    b = None
    if with_b:
        b = np.zeros(shape)
        b[r:-r, r:-r, r:-r] = rng.normal(size=(nz, ny, nx))
    S = dense_S(nx, ny, nz, r, c)
    inner = (slice(r, nz + r), slice(r, ny + r), slice(r, nx + r))
    want = S @ u.ravel() + (b[inner].ravel() if with_b else 0.0)
    got = oracle.sweep(u, c, r, b)
    scale = 1.0 + np.abs(S).sum(axis=1).max() + (np.abs(b).max() if with_b else 0.0)
    assert np.max(np.abs(got[inner].ravel() - want)) <= 1e-14 * scale
    # the halo of the result is the input's
    mask = np.ones(shape, dtype=bool)
    mask[inner] = False
    assert np.array_equal(got[mask], u[mask])
    res = np.linalg.norm(want - u[inner].ravel())
    assert abs(oracle.residual_norm(u, c, r, b) - res) <= 1e-13 * (scale + res)


@settings(max_examples=40, deadline=None)
@given(nx=extent, ny=extent, nz=extent, r=st.sampled_from([1, 2]), c=st.lists(coef, min_size=3, max_size=3),
       seed=st.integers(0, 2 ** 31 - 1), iters=st.integers(0, 4), threads=st.integers(0, 9))
def test_host_library_is_the_oracle_bitwise(nx, ny, nz, r, c, seed, iters, threads):
    import paper_2409_18824_gb300.host as host
    c = c[:r + 1]
    u = np.random.default_rng(seed).uniform(-1, 1, size=(nz + 2 * r, ny + 2 * r, nx + 2 * r))
    ref = oracle.stencil_sweep(u, c, r, iters)
    out = np.zeros_like(u)
    host.stencil_host_sweep_f64(u.copy(), out, c, r, iters, nthreads=threads)
    assert np.array_equal(out.view(np.uint64), ref.view(np.uint64))


def dense_S2(nx, ny, r, c):
    NX = nx + 2 * r
    S = np.zeros((nx * ny, NX * (ny + 2 * r)))
    row = 0
    for j in range(r, ny + r):
        for i in range(r, nx + r):
            p = j * NX + i
            S[row, p] += c[0]
            for d in range(1, r + 1):
                for q in (p - d, p + d, p - d * NX, p + d * NX):
                    S[row, q] += c[d]
            row += 1
    return S


@settings(max_examples=60, deadline=None)
@given(nx=st.integers(1, 12), ny=st.integers(1, 12), r=st.sampled_from([1, 2]),
       c=st.lists(coef, min_size=3, max_size=3), seed=st.integers(0, 2 ** 31 - 1), with_b=st.booleans())
def test_oracle_2d_sweep_and_residual_equal_the_dense_operator(nx, ny, r, c, seed, with_b):
    c = c[:r + 1]
    rng = np.random.default_rng(seed)
    shape = (ny + 2 * r, nx + 2 * r)
    u = rng.uniform(-1, 1, size=shape)
    b = None
    if with_b:
        b = np.zeros(shape)
        b[r:-r, r:-r] = rng.normal(size=(ny, nx))
    S = dense_S2(nx, ny, r, c)
    inner = (slice(r, ny + r), slice(r, nx + r))
    want = S @ u.ravel() + (b[inner].ravel() if with_b else 0.0)
    got = oracle.sweep2d(u, c, r, b)
    scale = 1.0 + np.abs(S).sum(axis=1).max() + (np.abs(b).max() if with_b else 0.0)
    assert np.max(np.abs(got[inner].ravel() - want)) <= 1e-14 * scale
    res = np.linalg.norm(want - u[inner].ravel())
    assert abs(oracle.residual_norm2d(u, c, r, b) - res) <= 1e-13 * (scale + res)


@settings(max_examples=40, deadline=None)
@given(nx=st.integers(1, 5), ny=st.integers(1, 5), nz=st.integers(1, 5), R=st.sampled_from([1, 2]),
       w1=st.floats(0.1, 2.0), w2=st.floats(0.1, 2.0), seed=st.integers(0, 2 ** 31 - 1))
def test_oracle_varcoef_operator_equals_its_definition(nx, ny, nz, R, w1, w2, seed):
    """(A u)(p) = sum over the 6R neighbours q of w_d (a(p)+a(q))/2 (u(p) - u(q)),
    and one Jacobi sweep is u'(p) = (f(p) + sum w_d kappa u(q)) / sum w_d kappa."""
    w = (0.0, w1, w2)[:R + 1]
    rng = np.random.default_rng(seed)
    shape = (nz + 2 * R, ny + 2 * R, nx + 2 * R)
    NX, NY = nx + 2 * R, ny + 2 * R
    a = rng.uniform(0.5, 1.5, size=shape)
    u = rng.uniform(-1, 1, size=shape)
    f = np.zeros(shape)
    f[R:-R, R:-R, R:-R] = rng.normal(size=(nz, ny, nx))
    af, uf = a.ravel(), u.ravel()
    Au, sweep = [], []
    for k in range(R, nz + R):
        for j in range(R, ny + R):
            for i in range(R, nx + R):
                p = (k * NY + j) * NX + i
                D = N = 0.0
                for d in range(1, R + 1):
                    for q in (p - d, p + d, p - d * NX, p + d * NX, p - d * NX * NY, p + d * NX * NY):
                        t = w[d] * 0.5 * (af[p] + af[q])
                        D += t
                        N += t * uf[q]
                Au.append(D * uf[p] - N)
                sweep.append((f.ravel()[p] + N) / D)
    inner = (slice(R, nz + R), slice(R, ny + R), slice(R, nx + R))
    got_a = oracle.varcoef_apply(u, a, w, R)[inner].ravel()
    got_s = oracle.varcoef_sweep(u, a, f, w, R)[inner].ravel()
    assert np.max(np.abs(got_a - np.array(Au))) <= 1e-13 * (1 + np.max(np.abs(Au)))
    assert np.max(np.abs(got_s - np.array(sweep))) <= 1e-13 * (1 + np.max(np.abs(sweep)))
