"""Pins for the CPU oracle (no GPU).

Each test checks the oracle against something other than itself: a closed
form, an invariant of the mathematics, a dense matrix assembled independently
from the definition, or a library routine (numpy.linalg.solve).  Grids are
non-cubic wherever axes could be confused, so that a swapped stride, a dropped
neighbour, a wrong sign or a wrong coefficient fails at least one test.
"""
import math

import numpy as np
import pytest

import oracle
import stencil_inputs as si

L7 = si.LAPLACE7


# ---------------------------------------------------------------- helpers
def interior(g, r):
    return g[r:g.shape[0] - r, r:g.shape[1] - r, r:g.shape[2] - r]


def dense_sweep_operator(nx, ny, nz, r, c):
    """Dense S (interior x padded) from the definition: row p has c0 at p and
    c_d at each of the 6 neighbours at distance d.  Written independently of
    the oracle (numpy index arithmetic over the padded grid)."""
    NX, NY, NZ = nx + 2 * r, ny + 2 * r, nz + 2 * r
    npad = NX * NY * NZ
    rows = []
    for k in range(r, nz + r):
        for j in range(r, ny + r):
            for i in range(r, nx + r):
                row = np.zeros(npad)
                p = np.ravel_multi_index((k, j, i), (NZ, NY, NX))
                row[p] += c[0]
                for d in range(1, r + 1):
                    for (dk, dj, di) in ((0, 0, d), (0, 0, -d), (0, d, 0), (0, -d, 0), (d, 0, 0), (-d, 0, 0)):
                        q = np.ravel_multi_index((k + dk, j + dj, i + di), (NZ, NY, NX))
                        row[q] += c[d]
                rows.append(row)
    return np.array(rows)


def dense_varcoef_operator(a, nx, ny, nz, R, w):
    """Dense A (interior x padded) from (A u)(p) = sum w_d kappa(p,q)(u(p)-u(q))."""
    NX, NY, NZ = nx + 2 * R, ny + 2 * R, nz + 2 * R
    af = a.ravel()
    rows = []
    for k in range(R, nz + R):
        for j in range(R, ny + R):
            for i in range(R, nx + R):
                row = np.zeros(NX * NY * NZ)
                p = np.ravel_multi_index((k, j, i), (NZ, NY, NX))
                for d in range(1, R + 1):
                    for (dk, dj, di) in ((0, 0, d), (0, 0, -d), (0, d, 0), (0, -d, 0), (d, 0, 0), (-d, 0, 0)):
                        q = np.ravel_multi_index((k + dk, j + dj, i + di), (NZ, NY, NX))
                        kap = 0.5 * (af[p] + af[q])
                        row[p] += w[d] * kap
                        row[q] -= w[d] * kap
                rows.append(row)
    return np.array(rows)


def interior_mask(nx, ny, nz, r):
    m = np.zeros(si.padded_shape(nx, ny, nz, r), dtype=bool)
    m[r:r + nz, r:r + ny, r:r + nx] = True
    return m.ravel()


def rel_inf(x, ref):
    return np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)), 1e-300)


# ---------------------------------------------------- closed form: eigenmode
@pytest.mark.parametrize("n,m", [((64, 64, 64), (1, 1, 1)), ((13, 9, 7), (2, 3, 1)), ((20, 11, 6), (5, 1, 4))])
def test_sweep_eigenmode_decay(n, m):
    """A zero-halo sine mode is an eigenvector of the 7-point Jacobi sweep with
    eigenvalue (cos tx + cos ty + cos tz)/3, t_a = m_a pi/(n_a+1)."""
    nx, ny, nz = n
    u0 = si.sine_mode(nx, ny, nz, 1, m)
    lam = sum(math.cos(ma * math.pi / (na + 1)) for ma, na in zip(m, n)) / 3.0
    sweeps = 7
    u = oracle.stencil_sweep(u0, L7, 1, sweeps)
    assert rel_inf(interior(u, 1), lam ** sweeps * interior(u0, 1)) < 1e-13
    assert np.all(u[0] == 0) and np.all(u[:, 0] == 0) and np.all(u[:, :, -1] == 0)


def test_residual_norm_closed_form_64cubed():
    """||S u - u|| of lam^n u0 equals |1-lam| lam^n ||u0|| with ||u0||^2 = prod (n_a+1)/2."""
    n = 64
    u0 = si.sine_mode(n, n, n, 1)
    lam = math.cos(math.pi / 65)
    u = oracle.stencil_sweep(u0, L7, 1, 100)
    expect = abs(1 - lam) * lam ** 100 * math.sqrt((65 / 2) ** 3)
    got = oracle.residual_norm(u, L7, 1)
    assert abs(got - expect) / expect < 1e-10
    assert abs(lam ** 100 - 0.8897) < 1e-4  # the figure quoted for 64^3 after 100 sweeps


@pytest.mark.parametrize("c", [(0.1, 0.12, 0.03), (0.0, 0.1, 0.0666)])
def test_radius2_one_sweep_eigenvalue(c):
    """With the halo holding the odd extension of the sine (the sine function
    evaluated on the padded index range), one radius-2 sweep multiplies the
    interior by c0 + sum_d c_d * 2 (cos d tx + cos d ty + cos d tz)."""
    nx, ny, nz, r = 11, 8, 6, 2
    m = (1, 2, 1)
    ii = [np.arange(1 - r, na + r + 1) for na in (nx, ny, nz)]
    fx, fy, fz = (np.sin(ma * np.pi * ia / (na + 1)) for ma, ia, na in zip(m, ii, (nx, ny, nz)))
    u = fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
    th = [ma * math.pi / (na + 1) for ma, na in zip(m, (nx, ny, nz))]
    lam = c[0] + sum(c[d] * 2 * sum(math.cos(d * t) for t in th) for d in (1, 2))
    out = oracle.sweep(u, c, 2)
    assert rel_inf(interior(out, 2), lam * interior(u, 2)) < 1e-13


def test_one_dimensional_reduction():
    """ny = nz = 1 with a zero halo: the y and z neighbours vanish and the sweep is
    the 1D update (u[i-1]+u[i+1])/6, whose eigenvalues are cos(m pi/(n+1))/3."""
    n = 17
    for m in (1, 4, 11):
        u0 = si.sine_mode(n, 1, 1, 1, (m, 1, 1))
        out = oracle.sweep(u0, L7, 1)
        lam = math.cos(m * math.pi / (n + 1)) / 3.0
        assert rel_inf(interior(out, 1), lam * interior(u0, 1)) < 1e-13


# ------------------------------------------------------------- invariants
@pytest.mark.parametrize("r,c", [(1, (0.0, 1 / 6)), (1, (0.4, 0.1)), (2, (0.1, 0.1, 0.05)), (2, (0.0, 0.125, 1 / 24))])
def test_constant_field_is_fixed(r, c):
    assert abs(c[0] + 6 * sum(c[1:]) - 1.0) < 1e-15
    u = np.full(si.padded_shape(9, 7, 5, r), 0.73)
    out = oracle.sweep(u, c, r)
    assert rel_inf(out, u) < 8e-16


@pytest.mark.parametrize("r,c", [(1, (0.0, 1 / 6)), (2, (0.1, 0.1, 0.05))])
def test_linear_field_is_fixed(r, c):
    """A linear field filled including the halo has zero discrete Laplacian."""
    u = si.linear_field(9, 7, 5, r, 0.3, -1.1, 0.7, 2.0)
    out = oracle.sweep(u, c, r)
    assert rel_inf(out, u) < 1e-14


def test_quadratic_field_constant_laplacian():
    """u = i^2 + 2 j^2 - k^2: each neighbour pair at distance d adds 2 d^2 * coefficient
    of that axis' square, so S u - u = sum_d c_d 2 d^2 (1 + 2 - 1) for a normalised stencil."""
    r, c = 2, (0.1, 0.1, 0.05)
    nx, ny, nz = 7, 6, 5
    k, j, i = np.meshgrid(np.arange(1, nz + 2 * r + 1), np.arange(1, ny + 2 * r + 1),
                          np.arange(1, nx + 2 * r + 1), indexing="ij")
    u = (i ** 2 + 2.0 * j ** 2 - k ** 2).astype(np.float64)
    out = oracle.sweep(u, c, r)
    expect = sum(c[d] * 2 * d * d for d in (1, 2)) * (1 + 2 - 1)
    assert np.max(np.abs(interior(out - u, r) - expect)) < 1e-11


# ------------------------------------------------------------ brute force
@pytest.mark.parametrize("n,r,c", [((4, 4, 4), 1, (0.0, 1 / 6)), ((3, 4, 5), 1, (0.3, 0.11)),
                                   ((5, 5, 5), 2, (0.2, 0.09, 0.04)), ((4, 3, 5), 2, (-0.1, 0.2, -0.03))])
def test_sweep_matches_dense_operator(n, r, c):
    nx, ny, nz = n
    u = si.uniform_interior(nx, ny, nz, r, seed=11, lo=-1, hi=1)
    # non-zero halo so that halo reads are checked too
    halo = ~interior_mask(nx, ny, nz, r)
    u.ravel()[halo] = si.rng(12).random(int(halo.sum())) - 0.5
    b = si.normal_interior(nx, ny, nz, r, seed=13)
    S = dense_sweep_operator(nx, ny, nz, r, c)
    expect = S @ u.ravel() + b.ravel()[interior_mask(nx, ny, nz, r)]
    got = oracle.sweep(u, c, r, b)
    assert np.max(np.abs(interior(got, r).ravel() - expect)) < 1e-14
    assert np.array_equal(got.ravel()[halo], u.ravel()[halo])
    # residual norm brute force
    rho = expect - u.ravel()[interior_mask(nx, ny, nz, r)]
    assert abs(oracle.residual_norm(u, c, r, b) - np.linalg.norm(rho)) < 1e-13 * max(1, np.linalg.norm(rho))


def test_sweep_f32_matches_dense_operator():
    nx, ny, nz, r, c = 5, 4, 3, 1, (0.0, 1 / 6)
    u = si.uniform_interior(nx, ny, nz, r, seed=21, dtype=np.float32)
    S = dense_sweep_operator(nx, ny, nz, r, np.array(c, dtype=np.float32).astype(np.float64))
    expect = S @ u.ravel().astype(np.float64)
    got = oracle.sweep(u, c, r)
    assert got.dtype == np.float32
    assert np.max(np.abs(interior(got, r).ravel().astype(np.float64) - expect)) < 4 * 2.0 ** -24
    # and float32 really is float32 arithmetic: not equal to the double result in general
    got64 = oracle.sweep(u.astype(np.float64), c, r)
    assert not np.array_equal(got.astype(np.float64), got64)


def test_stencil_sweep_iters_zero_and_one():
    u = si.uniform_interior(6, 5, 4, 1, seed=31)
    assert np.array_equal(oracle.stencil_sweep(u, L7, 1, 0), u)
    assert np.array_equal(oracle.stencil_sweep(u, L7, 1, 1), oracle.sweep(u, L7, 1))
    two = oracle.sweep(oracle.sweep(u, L7, 1), L7, 1)
    assert np.array_equal(oracle.stencil_sweep(u, L7, 1, 2), two)


# ---------------------------------------------------------------- solves
def test_dense_solve_matches_numpy():
    g = si.rng(41)
    for n in (1, 5, 30):
        A = g.standard_normal((n, n)) + n * np.eye(n)
        b = g.standard_normal(n)
        assert np.allclose(oracle.dense_solve(A, b), np.linalg.solve(A, b), rtol=1e-12, atol=1e-12)
    # pivoting needed: zero leading diagonal
    A = np.array([[0.0, 2.0, 1.0], [1.0, 1.0, 0.0], [3.0, 0.0, 1.0]])
    b = np.array([1.0, 2.0, 3.0])
    assert np.allclose(oracle.dense_solve(A, b), np.linalg.solve(A, b), rtol=1e-14)
    with pytest.raises(np.linalg.LinAlgError):
        oracle.dense_solve(np.zeros((2, 2)), np.ones(2))


def test_jacobi_solve_matches_direct_solve():
    nx, ny, nz, r = 5, 4, 6, 1
    b = si.normal_interior(nx, ny, nz, r, seed=5)
    mask = interior_mask(nx, ny, nz, r)
    S = dense_sweep_operator(nx, ny, nz, r, L7)[:, mask]
    x = oracle.dense_solve(np.eye(mask.sum()) - S, b.ravel()[mask])
    tol = 1e-12
    u, iters, rel, st = oracle.jacobi_solve(b, np.zeros_like(b), L7, r, tol, 10000, 10)
    assert st == 0 and rel <= tol and iters % 10 == 0
    kappa = np.linalg.cond(np.eye(mask.sum()) - S)
    assert np.max(np.abs(u.ravel()[mask] - x)) / np.max(np.abs(x)) < 10 * kappa * tol


def test_jacobi_iteration_count_matches_contraction():
    """b = 0 from an eigenmode: the residual after n sweeps is |1-lam| lam^n ||u0||, so
    the first checked multiple of K with residual <= tol is known in closed form."""
    nx, ny, nz, K, tol = 12, 9, 7, 5, 1e-6
    u0 = si.sine_mode(nx, ny, nz, 1)
    lam = sum(math.cos(math.pi / (na + 1)) for na in (nx, ny, nz)) / 3
    norm0 = math.sqrt((nx + 1) * (ny + 1) * (nz + 1) / 8)
    n = 0
    while True:  # the residual is measured on iterate n = K-1, 2K-1, ...
        n += K
        if abs(1 - lam) * lam ** (n - 1) * norm0 <= tol:
            break
    u, iters, rel, st = oracle.jacobi_solve(None, u0, L7, 1, tol, 100000, K)
    assert st == 0 and iters == n
    assert abs(rel - abs(1 - lam) * lam ** (n - 1) * norm0) < 1e-9 * rel
    _, iters2, rel2, st2 = oracle.jacobi_solve(None, u0, L7, 1, tol, n - K, K)
    assert st2 == 1 and iters2 == n - K and rel2 > tol


# ------------------------------------------------------- variable coefficient
def test_varcoef_apply_matches_dense_and_is_symmetric():
    nx, ny, nz, R, w = 5, 4, 5, 2, si.VARCOEF_W
    a = si.uniform_full(nx, ny, nz, R, seed=3)
    A = dense_varcoef_operator(a, nx, ny, nz, R, w)
    u = si.uniform_interior(nx, ny, nz, R, seed=7, lo=-1, hi=1)
    halo = ~interior_mask(nx, ny, nz, R)
    u.ravel()[halo] = si.rng(8).random(int(halo.sum()))
    got = oracle.varcoef_apply(u, a, w, R)
    assert np.max(np.abs(interior(got, R).ravel() - A @ u.ravel())) < 1e-13
    mask = interior_mask(nx, ny, nz, R)
    Ai = A[:, mask]
    assert np.max(np.abs(Ai - Ai.T)) < 1e-15
    assert np.all(np.linalg.eigvalsh(Ai) > 0)


def test_varcoef_constant_a_reduces_to_star_stencil():
    """a = 1: kappa = 1, so the Jacobi update is the constant star stencil with
    c_d = w_d / (6 sum w) and source f / (6 sum w)."""
    nx, ny, nz, R, w = 7, 5, 6, 2, si.VARCOEF_W
    a = np.ones(si.padded_shape(nx, ny, nz, R))
    f = si.normal_interior(nx, ny, nz, R, seed=9)
    u = si.uniform_interior(nx, ny, nz, R, seed=10)
    den = 6 * (w[1] + w[2])
    got = oracle.varcoef_sweep(u, a, f, w, R)
    ref = oracle.sweep(u, (0.0, w[1] / den, w[2] / den), R, f / den)
    assert rel_inf(interior(got, R), interior(ref, R)) < 1e-14


def test_varcoef_jacobi_and_residual_match_dense():
    nx, ny, nz, R, w = 4, 5, 3, 2, si.VARCOEF_W
    a = si.uniform_full(nx, ny, nz, R, seed=3)
    f = si.normal_interior(nx, ny, nz, R, seed=5)
    mask = interior_mask(nx, ny, nz, R)
    Ai = dense_varcoef_operator(a, nx, ny, nz, R, w)[:, mask]
    x = np.linalg.solve(Ai, f.ravel()[mask])
    tol = 1e-11
    u, iters, rel, st = oracle.varcoef_jacobi_solve(a, f, np.zeros_like(f), w, R, tol, 20000, 4)
    assert st == 0 and rel <= tol
    res = f.ravel()[mask] - Ai @ u.ravel()[mask]
    assert abs(oracle.varcoef_residual_norm(u, a, f, w, R) - np.linalg.norm(res)) < 1e-12 * np.linalg.norm(f)
    assert np.max(np.abs(u.ravel()[mask] - x)) / np.max(np.abs(x)) < 10 * np.linalg.cond(Ai) * tol


def test_varcoef_sweep_f32_close_to_f64():
    nx, ny, nz, R, w = 6, 5, 4, 2, si.VARCOEF_W
    a = si.uniform_full(nx, ny, nz, R, seed=3)
    f = si.normal_interior(nx, ny, nz, R, seed=5)
    u = si.uniform_interior(nx, ny, nz, R, seed=6)
    s64 = oracle.varcoef_sweep(u, a, f, w, R)
    s32 = oracle.varcoef_sweep(u.astype(np.float32), a.astype(np.float32), f.astype(np.float32), w, R)
    assert s32.dtype == np.float32
    assert rel_inf(interior(s32, R).astype(np.float64), interior(s64, R)) < 1e-5


def test_refined_solve_reaches_tolerance():
    """Refinement end state: the double residual it reports is recomputed by the
    dense operator, and the solution matches the direct solve."""
    nx, ny, nz, R, w = 5, 4, 4, 2, si.VARCOEF_W
    a = si.uniform_full(nx, ny, nz, R, seed=3)
    f = si.normal_interior(nx, ny, nz, R, seed=5)
    mask = interior_mask(nx, ny, nz, R)
    Ai = dense_varcoef_operator(a, nx, ny, nz, R, w)[:, mask]
    tol = 1e-12
    u, outer, rel, st = oracle.varcoef_refined_solve(a, f, np.zeros_like(f), w, R, tol, 200, 50)
    assert st == 0 and outer >= 2
    res = np.linalg.norm(f.ravel()[mask] - Ai @ u.ravel()[mask]) / np.linalg.norm(f.ravel()[mask])
    assert res <= tol and abs(res - rel) <= 1e-3 * tol
    x = np.linalg.solve(Ai, f.ravel()[mask])
    assert np.max(np.abs(u.ravel()[mask] - x)) / np.max(np.abs(x)) < 10 * np.linalg.cond(Ai) * tol


def significant_bits(x):
    """Bits between the highest and lowest set bit of a dyadic double."""
    if x == 0:
        return 0
    num = abs(int(x * 2.0 ** 60))
    assert num == abs(x) * 2.0 ** 60  # dyadic with denominator <= 2^60
    while num % 2 == 0:
        num //= 2
    return num.bit_length()


@pytest.mark.parametrize("r,c,inner", [(1, (0.0, 0.125), 1), (1, (0.0, 0.125), 3), (1, (0.0, 0.125), 5),
                                       (2, (0.0625, 0.0625, 0.03125), 1), (2, (0.0625, 0.0625, 0.03125), 2),
                                       (2, (0.0625, 0.0625, 0.03125), 3)])
def test_refinement_step_is_exact_on_dyadic_data(r, c, inner):
    """One outer step of the constant-coefficient refinement, pinned step by
    step in a regime where float arithmetic is exact: dyadic coefficients, a
    right-hand side of small dyadic values with max |b| = 1 (so the scale is 1
    and float(rho / s) = b), and few enough inner sweeps that every float
    value needs at most 24 significant bits.  Then the inner float Jacobi
    iterate is the exact e_m = sum_{j<m} S^j b, which numpy computes here in
    double with the dense operator (any order gives the same exact value), the
    update gives u_1 = e_m bitwise, and the reported relative residual is
    ||S u_1 + b - u_1|| / ||b|| computed from the dense operator."""
    nx, ny, nz = 5, 4, 3
    rng = np.random.default_rng(61 + inner)
    b = np.zeros(si.padded_shape(nx, ny, nz, r))
    b[r:-r, r:-r, r:-r] = rng.integers(-8, 9, size=(nz, ny, nx)) / 8.0
    b[r, r, r] = 1.0  # max |b| = 1
    mask = interior_mask(nx, ny, nz, r)
    S = dense_sweep_operator(nx, ny, nz, r, c)
    bi = b.ravel()[mask]
    e = np.zeros(b.size)
    for _ in range(inner):
        e_new = np.zeros(b.size)
        e_new[mask] = S @ e + bi  # halo of e stays 0
        e = e_new
    # the regime is exact: every iterate value (and so every partial sum on
    # the way, which carries no finer bits) fits a float's 24-bit significand
    assert max(significant_bits(v) for v in e) <= 20
    u, outer, rel, st = oracle.refined_solve(b, np.zeros_like(b), c, r, 0.0, inner, 1)
    assert outer == 1 and st == 1
    assert np.array_equal(u.ravel()[mask], e[mask])  # u_1 = 1 * e_m, bitwise
    assert not u.ravel()[~mask].any()  # the halo is untouched
    rho = S @ u.ravel() + bi - u.ravel()[mask]
    want = np.linalg.norm(rho) / np.linalg.norm(bi)
    assert abs(rel - want) <= 1e-14 * want


@pytest.mark.parametrize("m", [7, 20])
def test_refinement_contracts_an_eigenmode_by_lambda_to_the_inner_sweeps(m):
    """Closed form for the refinement's outer steps.  With u = 0 and residual
    rho, one step adds e_m = sum_{j<m} S^j rho, so the next residual is
    S^m rho exactly (in exact arithmetic).  For a sine eigenmode b (S b = lam
    b) the relative residual after k outer steps is |lam|^(m k) and the
    iterate is b (1 - lam^(m k)) / (1 - lam); the float inner sweeps perturb
    each step by about m (6r+2) 2^-24 relative."""
    nx, ny, nz, r = 7, 5, 6, 1
    b = si.sine_mode(nx, ny, nz, r, m=(1, 2, 1))
    lam = (math.cos(math.pi / (nx + 1)) + math.cos(2 * math.pi / (ny + 1)) + math.cos(math.pi / (nz + 1))) / 3
    inner = interior(b, r)
    for k in (1, 2, 3, 4):
        u, outer, rel, st = oracle.refined_solve(b, np.zeros_like(b), L7, r, 0.0, m, k)
        assert outer == k and st == 1
        want = abs(lam) ** (m * k)
        assert abs(rel / want - 1) <= k * m * 8 * 2.0 ** -24 * 4, (k, rel, want)
        series = (1 - lam ** (m * k)) / (1 - lam)
        assert np.max(np.abs(interior(u, r) - series * inner)) <= m * 8 * 2.0 ** -24 * series * np.max(np.abs(inner))


def dyadic_varcoef(nx, ny, nz, R):
    """A coefficient field on the padded grid whose Jacobi diagonals are all
    powers of two.  Radius 1, w = (0, 1): a = 1, 3 alternating along i, so the
    six face weights kappa = (a(p)+a(q))/2 sum to 8 or 16.  Radius 2,
    w = (0, 1, 1): a = 1 or 3 by the parity of i + j (constant along k), so the
    twelve face weights sum to 16 or 32."""
    k, j, i = np.indices(si.padded_shape(nx, ny, nz, R))
    if R == 1:
        return np.where(i % 2 == 0, 1.0, 3.0), (0.0, 1.0)
    return np.where((i + j) % 2 == 0, 1.0, 3.0), (0.0, 1.0, 1.0)


def jacobi_split(a, nx, ny, nz, R, w):
    """A = D - N on the interior, from the dense operator."""
    mask = interior_mask(nx, ny, nz, R)
    Ai = dense_varcoef_operator(a, nx, ny, nz, R, w)[:, mask]
    D = np.diag(Ai).copy()
    return Ai, D, np.diag(D) - Ai, mask


@pytest.mark.parametrize("R,inner", [(1, 1), (1, 2), (1, 3), (1, 4), (2, 1), (2, 2), (2, 3)])
def test_varcoef_refinement_step_is_exact_on_dyadic_data(R, inner):
    """One outer step of the variable-coefficient refinement, pinned step by
    step where float arithmetic is exact: every Jacobi diagonal a power of
    two, face weights in {1, 2, 3}, f of small dyadic values with max |f| = 1
    (scale 1, float(rho / s) = f).  The inner float iterate is then the exact
    e_m = sum_{j<m} (D^-1 N)^j D^-1 f, the update gives u_1 = e_m bitwise, and
    the new residual f - A u_1 is exactly (N D^-1)^m f (A = D - N gives
    A e_m = f - (N D^-1)^m f)."""
    nx, ny, nz = 5, 4, 3
    a, w = dyadic_varcoef(nx, ny, nz, R)
    Ai, D, N, mask = jacobi_split(a, nx, ny, nz, R, w)
    assert set(np.unique(D)) <= {8.0, 16.0, 32.0}
    rng = np.random.default_rng(71 + inner)
    f = np.zeros(si.padded_shape(nx, ny, nz, R))
    f[R:-R, R:-R, R:-R] = rng.integers(-8, 9, size=(nz, ny, nx)) / 8.0
    f[R, R, R] = -1.0  # max |f| = 1
    fi = f.ravel()[mask]
    e = np.zeros_like(fi)
    for _ in range(inner):
        # the exactness regime: every partial sum of the float sweep is a
        # multiple of the finest bit of e and f, bounded by |f| + sum t |e|
        finest = min(2.0 ** -(significant_bits(v) - 1 - math.floor(math.log2(abs(v)))) if v else 1.0
                     for v in np.concatenate([e, fi]))
        bound = 1.0 + D.max() * np.max(np.abs(e))
        assert bound / finest < 2.0 ** 24, (bound, finest)
        e = (fi + N @ e) / D
    u, outer, rel, st = oracle.varcoef_refined_solve(a, f, np.zeros_like(f), w, R, 0.0, inner, 1)
    assert outer == 1 and st == 1
    assert np.array_equal(u.ravel()[mask], e)  # u_1 = 1 * e_m, bitwise
    assert not u.ravel()[~mask].any()  # the halo is untouched
    rho = fi - Ai @ u.ravel()[mask]
    closed = fi.copy()
    for _ in range(inner):
        closed = N @ (closed / D)
    assert np.array_equal(rho, closed)
    want = np.linalg.norm(closed) / np.linalg.norm(fi)
    assert abs(rel - want) <= 1e-14 * want


@pytest.mark.parametrize("m", [4, 11])
def test_varcoef_refinement_maps_the_residual_by_N_D_inverse_to_the_m(m):
    """Closed form for the variable-coefficient refinement's outer steps on
    random coefficients: with A = D - N, one step of m inner Jacobi sweeps from
    e = 0 takes the residual rho to (N D^-1)^m rho, up to the float rounding
    of the inner sweeps and of a and w.  Each sweep rounds about 12R+2
    operations per value and the sweeps contract (N D^-1 does not expand in
    the 1-norm), so the deviation stays near m (12R+2) 2^-24 of ||rho||_1;
    the test allows four times that.  Each outer step k is checked against
    the oracle's own residual after step k-1, recomputed from the dense
    operator; one inner sweep too many is checked to land at least ten times
    outside the allowance, so an off-by-one count, a lost scale or a wrong
    face weight fails."""
    nx, ny, nz, R, w = 5, 4, 6, 2, si.VARCOEF_W
    a = si.uniform_full(nx, ny, nz, R, seed=13)
    f = si.normal_interior(nx, ny, nz, R, seed=14)
    Ai, D, N, mask = jacobi_split(a, nx, ny, nz, R, w)
    fi = f.ravel()[mask]
    prev = fi
    for k in (1, 2, 3):
        u, outer, rel, st = oracle.varcoef_refined_solve(a, f, np.zeros_like(f), w, R, 0.0, m, k)
        assert outer == k and st == 1
        rho = fi - Ai @ u.ravel()[mask]
        closed = prev.copy()
        for _ in range(m):
            closed = N @ (closed / D)
        err = np.abs(rho - closed).sum() / np.abs(prev).sum()
        allow = 4 * m * (12 * R + 2) * 2.0 ** -24
        assert err <= allow, (k, err)
        # and the mistake the pin is meant to catch is far outside it
        assert np.abs(N @ (closed / D) - closed).sum() / np.abs(prev).sum() > 10 * allow
        assert abs(rel - np.linalg.norm(rho) / np.linalg.norm(fi)) <= 1e-12 * rel
        prev = rho


def test_constant_refined_solve_reaches_tolerance():
    """Constant-coefficient refinement end state: its reported double residual is
    recomputed from the dense operator, and u matches the direct solve of
    (I - S) u = b."""
    nx, ny, nz, r = 5, 4, 6, 1
    b = si.normal_interior(nx, ny, nz, r, seed=5)
    mask = interior_mask(nx, ny, nz, r)
    S = dense_sweep_operator(nx, ny, nz, r, L7)[:, mask]
    M = np.eye(mask.sum()) - S
    tol = 1e-12
    u, outer, rel, st = oracle.refined_solve(b, np.zeros_like(b), L7, r, tol, 300, 40)
    assert st == 0 and outer >= 2
    res = np.linalg.norm(b.ravel()[mask] - M @ u.ravel()[mask]) / np.linalg.norm(b.ravel()[mask])
    assert res <= tol and abs(res - rel) <= 1e-3 * tol
    x = np.linalg.solve(M, b.ravel()[mask])
    assert np.max(np.abs(u.ravel()[mask] - x)) / np.max(np.abs(x)) < 10 * np.linalg.cond(M) * tol
