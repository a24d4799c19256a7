"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke run.

This module holds random numbers and shapes only -- none of the stencil
arithmetic -- so that the CPU oracle and the CUDA library can both be fed from
it without sharing any code with each other.

Layout: every grid is a C-contiguous numpy array of shape (nz+2r, ny+2r, nx+2r),
i.e. the Fortran column-major array u(1:nx+2r, 1:ny+2r, 1:nz+2r) with the first
index fastest (arXiv 2409.18824 Sec. 5.2: 1-based Fortran indices mapped to
0-based offsets).  Random interiors are drawn in that memory order from numpy's
PCG64 generator with a stated seed.

Workloads (the paper's jacobi benchmark, Sec. 4, is a 2D 1024x1024 Laplace
Jacobi; its data are not published, so these seeded grids stand in for it):
  * 64^3  FP64 r=1, interior U[0,1) seed 1, zero halo, c = {0, 1/6}, 100 sweeps + norm
  * 512^3 FP64 r=1, interior U[0,1) seed 2, zero halo, 1000 sweeps
  * 768x768x384 r=2 variable coefficient, a ~ U[0.5,1.5] (seed 3) on the padded
    grid, manufactured (1,1,1) sine-mode solution
  * batches of solves with per-axis sizes log-uniform in [16,128] (seed 4),
    right-hand sides N(0,1) (seed 5)
  * serving arrivals: sizes log-uniform in [32,256] (seed 6), Poisson arrivals
  * the advection stand-in (pw-like): u, v, w on 2048 x 1024 x 1024 from the
    integer hash of hash_field (exact in any precision, so a device-side
    generator can reproduce it bit for bit)
  * the paper's own 2-D jacobi: 1024 x 1024 FP64 r=1, interior U[0,1) seed 7,
    zero halo, c = {0, 1/4}, 100000 sweeps (2-D grids are C-contiguous arrays
    of shape (ny+2r, nx+2r), i fastest)
"""
from __future__ import annotations

import math

import numpy as np

#: 7-point normalised Jacobi weights {c0, c1}: the discrete Laplace update.
LAPLACE7 = (0.0, 1.0 / 6.0)
#: 5-point normalised Jacobi weights {c0, c1} of the 2-D Laplace update.
LAPLACE5 = (0.0, 0.25)
#: radius-2 weights w = {unused, w1, w2} of the variable-coefficient operator.
VARCOEF_W = (0.0, 1.0, 0.25)


def padded_shape(nx: int, ny: int, nz: int, r: int):
    return (nz + 2 * r, ny + 2 * r, nx + 2 * r)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_interior(nx, ny, nz, r, seed, dtype=np.float64, lo=0.0, hi=1.0, halo=0.0):
    """Interior ~ U[lo, hi) in Fortran order, halo filled with `halo`."""
    g = np.full(padded_shape(nx, ny, nz, r), halo, dtype=np.float64)
    vals = rng(seed).random(nx * ny * nz) * (hi - lo) + lo
    g[r:r + nz, r:r + ny, r:r + nx] = vals.reshape(nz, ny, nx)
    return g.astype(dtype)


def normal_interior(nx, ny, nz, r, seed, dtype=np.float64):
    """Interior ~ N(0, 1) in Fortran order, zero halo."""
    g = np.zeros(padded_shape(nx, ny, nz, r), dtype=np.float64)
    g[r:r + nz, r:r + ny, r:r + nx] = rng(seed).standard_normal(nx * ny * nz).reshape(nz, ny, nx)
    return g.astype(dtype)


def uniform_full(nx, ny, nz, r, seed, lo=0.5, hi=1.5, dtype=np.float64):
    """Every padded cell ~ U[lo, hi) (coefficient fields live on the padded grid)."""
    shape = padded_shape(nx, ny, nz, r)
    return (rng(seed).random(int(np.prod(shape))) * (hi - lo) + lo).reshape(shape).astype(dtype)


def sine_mode(nx, ny, nz, r, m=(1, 1, 1), dtype=np.float64):
    """prod_a sin(m_a*pi*i_a/(n_a+1)) on the interior (i_a = 1..n_a), zero halo.

    An exact eigenvector of the constant-coefficient 7-point Jacobi sweep with a
    zero Dirichlet halo; also the manufactured solution of the Poisson solves.
    """
    g = np.zeros(padded_shape(nx, ny, nz, r), dtype=np.float64)
    sx = np.sin(m[0] * np.pi * np.arange(1, nx + 1) / (nx + 1))
    sy = np.sin(m[1] * np.pi * np.arange(1, ny + 1) / (ny + 1))
    sz = np.sin(m[2] * np.pi * np.arange(1, nz + 1) / (nz + 1))
    g[r:r + nz, r:r + ny, r:r + nx] = sz[:, None, None] * sy[None, :, None] * sx[None, None, :]
    return g.astype(dtype)


def linear_field(nx, ny, nz, r, alpha, beta, gamma, delta, dtype=np.float64):
    """alpha*i + beta*j + gamma*k + delta on every padded cell (1-based i, j, k)."""
    k, j, i = np.meshgrid(np.arange(1, nz + 2 * r + 1), np.arange(1, ny + 2 * r + 1),
                          np.arange(1, nx + 2 * r + 1), indexing="ij")
    return (alpha * i + beta * j + gamma * k + delta).astype(dtype)


def log_uniform_sizes(count, lo, hi, seed):
    """(count, 3) int array of per-axis sizes (nx, ny, nz), log-uniform in [lo, hi]."""
    x = rng(seed).random((count, 3))
    s = np.exp(math.log(lo) + x * (math.log(hi) - math.log(lo)))
    return np.clip(np.floor(s + 0.5).astype(np.int64), lo, hi)


def poisson_arrival_times(count, rate_per_s, seed):
    """Arrival times (seconds from 0) of a Poisson process with the given rate."""
    gaps = rng(seed).exponential(1.0 / rate_per_s, size=count)
    return np.cumsum(gaps)


# ------------------------------------------------------------------- 2-D --
def padded_shape2d(nx: int, ny: int, r: int):
    return (ny + 2 * r, nx + 2 * r)


def uniform_interior2d(nx, ny, r, seed, dtype=np.float64, lo=0.0, hi=1.0, halo=0.0):
    """2-D interior ~ U[lo, hi) with i fastest, halo filled with `halo`."""
    g = np.full(padded_shape2d(nx, ny, r), halo, dtype=np.float64)
    g[r:r + ny, r:r + nx] = (rng(seed).random(nx * ny) * (hi - lo) + lo).reshape(ny, nx)
    return g.astype(dtype)


def uniform_full2d(nx, ny, r, seed, lo=0.0, hi=1.0, dtype=np.float64):
    """Every padded 2-D cell (halo included) ~ U[lo, hi)."""
    shape = padded_shape2d(nx, ny, r)
    return (rng(seed).random(int(np.prod(shape))) * (hi - lo) + lo).reshape(shape).astype(dtype)


def sine_mode2d(nx, ny, r, m=(1, 1), dtype=np.float64):
    """sin(m_x*pi*i/(nx+1)) * sin(m_y*pi*j/(ny+1)) on the interior, zero halo."""
    g = np.zeros(padded_shape2d(nx, ny, r), dtype=np.float64)
    sx = np.sin(m[0] * np.pi * np.arange(1, nx + 1) / (nx + 1))
    sy = np.sin(m[1] * np.pi * np.arange(1, ny + 1) / (ny + 1))
    g[r:r + ny, r:r + nx] = sy[:, None] * sx[None, :]
    return g.astype(dtype)


def linear_field2d(nx, ny, r, alpha, beta, delta, dtype=np.float64):
    """alpha*i + beta*j + delta on every padded 2-D cell (1-based i, j)."""
    j, i = np.meshgrid(np.arange(1, ny + 2 * r + 1), np.arange(1, nx + 2 * r + 1), indexing="ij")
    return (alpha * i + beta * j + delta).astype(dtype)


# ----------------------------------------------------------- hashed fields --
HASH_MULS = (73, 179, 283, 419)  # per-axis and per-component multipliers


def hash_field(NX, NY, k0, k1, comp, dtype=np.float64):
    """Padded planes [k0, k1) of an NX x NY-plane field whose cell (i, j, k)
    holds ((73 i + 179 j + 283 k + 419 comp) mod 65536) / 32768 - 1: values in
    [-1, 1) with 16-bit resolution, exact in float and double."""
    k, j, i = np.meshgrid(np.arange(k0, k1, dtype=np.int64), np.arange(NY, dtype=np.int64),
                          np.arange(NX, dtype=np.int64), indexing="ij")
    a, b, c, d = HASH_MULS
    h = (a * i + b * j + c * k + d * comp) % 65536
    return (h.astype(np.float64) / 32768.0 - 1.0).astype(dtype)
