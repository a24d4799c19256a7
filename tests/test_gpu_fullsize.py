"""Parity at the benchmarks' full sizes, in the launch configurations they time.

The oracle cannot sweep a 512^3 grid a thousand times, but an output point
after s sweeps depends only on the input within s*r of it.  So each check
cuts windows out of the full-size input (with s*r cells of context around
them, or the grid's own halo at a boundary), runs the oracle on the window
alone, and compares the window's inner region -- where the dependence cone
lies inside the window -- bitwise with the GPU's full-size result.  Windows
sit at corners, edges and the middle.  Full-size residual norms are compared
whole: with the oracle's residual field summed pairwise (tight), and with the
oracle's left-to-right sum within that sum's own error bound.
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


def full_norm_checks(norm, got, sweep_once, r, oracle_norm):
    """The GPU's fused norm against (1) the oracle's residual field summed by
    numpy's pairwise summation (error <= log2(n) u sum, so 1e-12 relative is a
    real test) and (2) the oracle's own left-to-right norm within the bound of
    a sequential sum of n terms, n u relative on the norm."""
    rho = sweep_once(got).astype(np.float64) - got.astype(np.float64)
    inner = tuple(slice(r, m - r) for m in got.shape)
    tight = float(np.sqrt(np.sum(np.square(rho[inner]))))
    assert abs(norm - tight) <= 1e-12 * tight
    n = rho[inner].size
    assert abs(norm - oracle_norm) <= n * 2.0 ** -53 * oracle_norm


def windows(shape, w, dep):
    """Starts (padded coordinates, per axis) of windows of w output cells whose
    dependence context `dep` fits in the padded array: first, middle, last."""
    out = []
    for n in shape:
        lo, hi = dep, n - dep - w
        out.append(sorted({lo, (lo + hi) // 2, hi}))
    return out


def check_windows3(full_in, full_out, step, r, sweeps, w=6):
    """step(window) -> the oracle's result on that padded window."""
    dep = r * sweeps
    nz, ny, nx = full_in.shape
    for k0 in windows((nz,), w, dep)[0]:
        for j0 in windows((ny,), w, dep)[0]:
            for i0 in windows((nx,), w, dep)[0]:
                win = np.ascontiguousarray(full_in[k0 - dep:k0 + w + dep, j0 - dep:j0 + w + dep,
                                                   i0 - dep:i0 + w + dep])
                ref = step(win)
                got = full_out[k0:k0 + w, j0:j0 + w, i0:i0 + w]
                exp = ref[dep:dep + w, dep:dep + w, dep:dep + w]
                assert bitwise(np.ascontiguousarray(got), np.ascontiguousarray(exp)), (k0, j0, i0)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_512cubed_sweeps_sampled_windows_and_full_norm(lib, cuda, dtype):
    """The 512^3 workloads (FP64 default kernel, FP32 column kernel) after 3
    sweeps; then the fused residual norm of the result against the oracle's
    full-size norm."""
    n, r, sweeps = 512, 1, 3
    u0 = si.uniform_interior(n, n, n, r, seed=2, dtype=dtype)
    d_in, d_out = to_dev(u0), to_dev(np.zeros_like(u0))
    fn = lib.stencil_sweep_f64 if dtype == np.float64 else lib.stencil_sweep_f32
    fn(d_in, d_out, si.LAPLACE7, r, sweeps)
    got = to_host(d_out)
    # the windows' own halo cells stay at their input values in the oracle, so
    # only output cells whose cone stays inside the window are compared
    check_windows3(u0, got, lambda win: oracle.stencil_sweep(win, si.LAPLACE7, r, sweeps), r, sweeps)
    norm = (lib.residual_norm_f64 if dtype == np.float64 else lib.residual_norm_f32)(d_out, si.LAPLACE7, r)
    full_norm_checks(norm, got, lambda x: oracle.sweep(x, si.LAPLACE7, r), r,
                     oracle.residual_norm(got, si.LAPLACE7, r))


def test_varcoef_768x768x384_float_sweeps_sampled_windows(lib, cuda):
    """The variable-coefficient workload's float sweep (radius 2, a ~ U[0.5,1.5]
    seed 3 on the padded grid, f ~ N(0,1) seed 4) at full size from e = 0,
    2 sweeps, against the oracle on windows (dependence radius 4)."""
    nx, ny, nz, R, sweeps = 768, 768, 384, 2, 2
    W = si.VARCOEF_W
    a = si.uniform_full(nx, ny, nz, R, seed=3)
    f = si.normal_interior(nx, ny, nz, R, seed=4)
    a32, f32 = a.astype(np.float32), f.astype(np.float32)
    e0 = np.zeros_like(f32)
    d_in, d_out = to_dev(e0), to_dev(np.zeros_like(e0))
    lib.varcoef_sweep_f32(d_in, d_out, to_dev(a32), to_dev(f32), W, R, sweeps)
    got = to_host(d_out)
    dep, w = R * sweeps, 6
    for k0 in windows((nz + 2 * R,), w, dep)[0]:
        for j0 in windows((ny + 2 * R,), w, dep)[0]:
            for i0 in windows((nx + 2 * R,), w, dep)[0]:
                sl = (slice(k0 - dep, k0 + w + dep), slice(j0 - dep, j0 + w + dep), slice(i0 - dep, i0 + w + dep))
                ref = np.ascontiguousarray(e0[sl])
                aw, fw = np.ascontiguousarray(a32[sl]), np.ascontiguousarray(f32[sl])
                for _ in range(sweeps):
                    ref = oracle.varcoef_sweep(ref, aw, fw, W, R)
                inner = (slice(k0, k0 + w), slice(j0, j0 + w), slice(i0, i0 + w))
                exp = ref[dep:dep + w, dep:dep + w, dep:dep + w]
                assert bitwise(np.ascontiguousarray(got[inner]), np.ascontiguousarray(exp)), (k0, j0, i0)


def test_jacobi2d_1024_sampled_windows(lib, cuda):
    """The paper's 2-D grid (1024^2, resident path) after 7 sweeps, against the
    2-D oracle on windows (dependence radius 7)."""
    n, r, sweeps, w = 1024, 1, 7, 16
    u0 = si.uniform_interior2d(n, n, r, seed=7)
    d_out = to_dev(np.zeros_like(u0))
    lib.stencil_sweep2d_f64(to_dev(u0), d_out, si.LAPLACE5, r, sweeps)
    got = to_host(d_out)
    dep = r * sweeps
    for j0 in windows((n + 2 * r,), w, dep)[0]:
        for i0 in windows((n + 2 * r,), w, dep)[0]:
            win = np.ascontiguousarray(u0[j0 - dep:j0 + w + dep, i0 - dep:i0 + w + dep])
            ref = oracle.stencil_sweep2d(win, si.LAPLACE5, r, sweeps)
            assert bitwise(np.ascontiguousarray(got[j0:j0 + w, i0:i0 + w]),
                           np.ascontiguousarray(ref[dep:dep + w, dep:dep + w])), (j0, i0)
    full_norm_checks(lib.residual_norm2d_f64(d_out, si.LAPLACE5, r), got,
                     lambda x: oracle.sweep2d(x, si.LAPLACE5, r), r, oracle.residual_norm2d(got, si.LAPLACE5, r))


def _hash_field_device(NX, NY, NZ, comp, device):
    """stencil_inputs.hash_field computed on the device plane by plane (integer
    arithmetic, then an exact scaling: the same bits as the numpy version)."""
    import torch
    a, b, c, d = si.HASH_MULS
    out = torch.empty((NZ, NY, NX), dtype=torch.float64, device=device)
    i = torch.arange(NX, device=device, dtype=torch.int64)
    j = torch.arange(NY, device=device, dtype=torch.int64)
    base = a * i[None, :] + b * j[:, None] + d * comp
    for k in range(NZ):
        out[k] = ((base + c * k) % 65536).to(torch.float64) / 32768.0 - 1.0
    return out


def test_advect_2048x1024x1024_sampled_windows(lib, cuda):
    """The advection stand-in at the paper's pw-advection size (2048 x 1024 x
    1024, u, v, w advecting themselves, FP64): windows of 6^3 cells (plus one
    cell of context) at corners, edges and the middle against the oracle."""
    import torch
    nx, ny, nz = 2048, 1024, 1024
    NX, NY, NZ = nx + 2, ny + 2, nz + 2
    c = (0.25, 0.25, 0.25)
    vel = [_hash_field_device(NX, NY, NZ, m, "cuda") for m in range(3)]
    outs = [torch.empty_like(vel[0]) for _ in range(3)]
    lib.advect_f64(vel[0], vel[1], vel[2], outs, c)
    torch.cuda.synchronize()
    w, dep = 6, 1
    starts = [windows((n,), w, dep)[0] for n in (NZ, NY, NX)]
    for k0 in starts[0]:
        for j0 in starts[1]:
            for i0 in starts[2]:
                fw = [si.hash_field(NX, NY, k0 - dep, k0 + w + dep, m)[:, j0 - dep:j0 + w + dep, i0 - dep:i0 + w + dep]
                      for m in range(3)]
                fw = [np.ascontiguousarray(x) for x in fw]
                for m in range(3):
                    ref = oracle.advect(fw[0], fw[1], fw[2], fw[m], c)[dep:dep + w, dep:dep + w, dep:dep + w]
                    got = outs[m][k0:k0 + w, j0:j0 + w, i0:i0 + w].cpu().numpy()
                    assert bitwise(np.ascontiguousarray(got), np.ascontiguousarray(ref)), (m, k0, j0, i0)
    # the device generator reproduces the host one
    assert bitwise(vel[1][5:7].cpu().numpy(), si.hash_field(NX, NY, 5, 7, 1))
