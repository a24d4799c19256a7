"""Pins for the 2-D oracle (the paper's jacobi benchmark is a 2-D Laplace
Jacobi iteration, arXiv 2409.18824 Sec. 4).  No GPU.

As for the 3-D oracle, each test checks against something other than the
oracle itself: the closed-form eigenvalues of the zero-halo sine modes, the
1-D textbook reduction, invariants of a normalised stencil, a dense operator
assembled from the definition with numpy, and the independently pinned 3-D
oracle on a one-plane grid.  Grids are non-square wherever the two axes could
be confused (a swapped stride or a dropped neighbour fails a test).
"""
import math

import numpy as np
import pytest

import oracle
import stencil_inputs as si

L5 = si.LAPLACE5


def interior(g, r):
    return g[r:g.shape[0] - r, r:g.shape[1] - r]


def rel_inf(x, ref):
    return np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)), 1e-300)


def dense_operator2d(nx, ny, r, c):
    """Dense S (interior x padded): c0 at p, c_d at the 4 neighbours at distance d."""
    NX, NY = nx + 2 * r, ny + 2 * r
    rows = []
    for j in range(r, ny + r):
        for i in range(r, nx + r):
            row = np.zeros(NX * NY)
            p = np.ravel_multi_index((j, i), (NY, NX))
            row[p] += c[0]
            for d in range(1, r + 1):
                for dj, di in ((0, d), (0, -d), (d, 0), (-d, 0)):
                    row[np.ravel_multi_index((j + dj, i + di), (NY, NX))] += c[d]
            rows.append(row)
    return np.array(rows)


def interior_mask2d(nx, ny, r):
    m = np.zeros(si.padded_shape2d(nx, ny, r), dtype=bool)
    m[r:r + ny, r:r + nx] = True
    return m.ravel()


# ---------------------------------------------------- closed form: eigenmode
@pytest.mark.parametrize("n,m", [((64, 64), (1, 1)), ((13, 9), (2, 3)), ((40, 7), (5, 1)),
                                 ((1024, 1024), (1, 1))])
def test_sweep2d_eigenmode_decay(n, m):
    """A zero-halo sine mode is an eigenvector of the 5-point Jacobi sweep with
    eigenvalue (cos tx + cos ty)/2, t_a = m_a pi/(n_a+1)."""
    nx, ny = n
    u0 = si.sine_mode2d(nx, ny, 1, m)
    lam = sum(math.cos(ma * math.pi / (na + 1)) for ma, na in zip(m, n)) / 2.0
    sweeps = 3 if nx > 100 else 9
    u = oracle.stencil_sweep2d(u0, L5, 1, sweeps)
    assert rel_inf(interior(u, 1), lam ** sweeps * interior(u0, 1)) < 1e-13
    assert np.all(u[0] == 0) and np.all(u[-1] == 0) and np.all(u[:, 0] == 0) and np.all(u[:, -1] == 0)


def test_residual2d_closed_form():
    """||S u - u|| of lam^n u0 equals |1-lam| lam^n ||u0|| with ||u0||^2 = (nx+1)/2 (ny+1)/2."""
    nx, ny = 48, 30
    u0 = si.sine_mode2d(nx, ny, 1)
    lam = (math.cos(math.pi / (nx + 1)) + math.cos(math.pi / (ny + 1))) / 2
    u = oracle.stencil_sweep2d(u0, L5, 1, 50)
    expect = abs(1 - lam) * lam ** 50 * math.sqrt((nx + 1) / 2 * (ny + 1) / 2)
    assert abs(oracle.residual_norm2d(u, L5, 1) - expect) / expect < 1e-10


def test_paper_size_decay_factor():
    """The paper's grid (1024 x 1024, 100000 iterations): the slowest mode decays by
    cos(pi/1025)^100000; the value that full-length GPU runs are checked against."""
    lam = math.cos(math.pi / 1025)
    assert abs(lam ** 100000 - math.exp(-100000 * (math.pi / 1025) ** 2 / 2)) < 1e-6
    assert 0.62 < lam ** 100000 < 0.63


@pytest.mark.parametrize("c", [(0.1, 0.15, 0.075), (0.0, 0.2, 0.05)])
def test_radius2_2d_eigenvalue(c):
    """With the halo holding the odd extension of the sine, one radius-2 sweep
    multiplies the interior by c0 + sum_d c_d * 2 (cos d tx + cos d ty)."""
    nx, ny, r, m = 11, 8, 2, (1, 3)
    fx = np.sin(m[0] * np.pi * np.arange(1 - r, nx + r + 1) / (nx + 1))
    fy = np.sin(m[1] * np.pi * np.arange(1 - r, ny + r + 1) / (ny + 1))
    u = fy[:, None] * fx[None, :]
    th = (m[0] * math.pi / (nx + 1), m[1] * math.pi / (ny + 1))
    lam = c[0] + sum(c[d] * 2 * sum(math.cos(d * t) for t in th) for d in (1, 2))
    assert rel_inf(interior(oracle.sweep2d(u, c, 2), 2), lam * interior(u, 2)) < 1e-13


def test_one_dimensional_reduction_2d():
    """ny = 1, zero halo, c1 = 1/2: the textbook 1-D Jacobi sweep (u[i-1]+u[i+1])/2
    with eigenvalues cos(m pi/(n+1))."""
    n = 23
    for m in (1, 6, 17):
        u0 = si.sine_mode2d(n, 1, 1, (m, 1))
        lam = math.cos(m * math.pi / (n + 1))
        assert rel_inf(interior(oracle.sweep2d(u0, (0.0, 0.5), 1), 1), lam * interior(u0, 1)) < 1e-13


# ------------------------------------------------------------- invariants
@pytest.mark.parametrize("r,c", [(1, (0.0, 0.25)), (1, (0.2, 0.2)), (2, (0.2, 0.15, 0.05))])
def test_constant_and_linear_fields_fixed_2d(r, c):
    assert abs(c[0] + 4 * sum(c[1:]) - 1.0) < 1e-15
    u = np.full(si.padded_shape2d(9, 7, r), 0.37)
    assert rel_inf(oracle.sweep2d(u, c, r), u) < 8e-16
    lin = si.linear_field2d(9, 7, r, 0.3, -1.1, 2.0)
    assert rel_inf(oracle.sweep2d(lin, c, r), lin) < 1e-14


def test_quadratic_field_2d():
    """u = i^2 + 2 j^2: S u - u = sum_d c_d 2 d^2 (1 + 2) for a normalised stencil."""
    r, c = 2, (0.2, 0.15, 0.05)
    nx, ny = 7, 6
    j, i = np.meshgrid(np.arange(1, ny + 2 * r + 1), np.arange(1, nx + 2 * r + 1), indexing="ij")
    u = (i ** 2 + 2.0 * j ** 2).astype(np.float64)
    expect = sum(c[d] * 2 * d * d for d in (1, 2)) * 3
    assert np.max(np.abs(interior(oracle.sweep2d(u, c, r) - u, r) - expect)) < 1e-11


# ------------------------------------------------------------ brute force
@pytest.mark.parametrize("n,r,c", [((5, 4), 1, (0.0, 0.25)), ((4, 6), 1, (0.3, 0.11)),
                                   ((6, 5), 2, (0.2, 0.09, 0.04)), ((3, 7), 2, (-0.1, 0.2, -0.03))])
def test_sweep2d_matches_dense_operator(n, r, c):
    nx, ny = n
    u = si.uniform_full2d(nx, ny, r, seed=41, lo=-1, hi=1)  # non-zero halo: halo reads checked
    b = si.uniform_interior2d(nx, ny, r, seed=42, lo=-1, hi=1)
    S = dense_operator2d(nx, ny, r, c)
    mask = interior_mask2d(nx, ny, r)
    expect = S @ u.ravel() + b.ravel()[mask]
    got = oracle.sweep2d(u, c, r, b)
    assert np.max(np.abs(interior(got, r).ravel() - expect)) < 1e-14
    assert np.array_equal(got.ravel()[~mask], u.ravel()[~mask])
    rho = expect - u.ravel()[mask]
    assert abs(oracle.residual_norm2d(u, c, r, b) - np.linalg.norm(rho)) < 1e-13 * max(1, np.linalg.norm(rho))


def test_sweep2d_f32_is_float_arithmetic():
    nx, ny, r, c = 6, 5, 1, (0.0, 0.25)
    u = si.uniform_interior2d(nx, ny, r, seed=43, dtype=np.float32)
    S = dense_operator2d(nx, ny, r, np.array(c, dtype=np.float32).astype(np.float64))
    got = oracle.sweep2d(u, c, r)
    assert got.dtype == np.float32
    assert np.max(np.abs(interior(got, r).ravel().astype(np.float64) - S @ u.ravel().astype(np.float64))) \
        < 3 * 2.0 ** -24
    u3 = si.uniform_interior2d(nx, ny, r, seed=44, dtype=np.float32, lo=0.1, hi=0.9)
    assert not np.array_equal(oracle.sweep2d(u3, (0.0, 0.3), r).astype(np.float64),
                              oracle.sweep2d(u3.astype(np.float64), (0.0, np.float32(0.3)), r))


def test_stencil_sweep2d_iteration_composition():
    u = si.uniform_interior2d(9, 6, 1, seed=45)
    assert np.array_equal(oracle.stencil_sweep2d(u, L5, 1, 0), u)
    assert np.array_equal(oracle.stencil_sweep2d(u, L5, 1, 1), oracle.sweep2d(u, L5, 1))
    three = oracle.sweep2d(oracle.sweep2d(oracle.sweep2d(u, L5, 1), L5, 1), L5, 1)
    assert np.array_equal(oracle.stencil_sweep2d(u, L5, 1, 3), three)


@pytest.mark.parametrize("r,c", [(1, (0.0, 0.25)), (2, (0.1, 0.15, 0.075))])
def test_agrees_with_3d_oracle_on_one_plane(r, c):
    """nz = 1 with a zero z-halo: the 3-D sweep adds (0 + 0) to each neighbour sum,
    so its middle plane equals the 2-D sweep (compared with ==, so -0 == +0)."""
    nx, ny = 13, 10
    u2 = si.uniform_full2d(nx, ny, r, seed=46, lo=-1, hi=1)
    u3 = np.zeros(si.padded_shape(nx, ny, 1, r))
    u3[r] = u2
    got2 = oracle.stencil_sweep2d(u2, c, r, 4)
    got3 = oracle.stencil_sweep(u3, c, r, 4)
    assert np.all(got2 == got3[r])
