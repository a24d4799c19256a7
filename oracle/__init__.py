"""CPU oracle for the 3D Jacobi stencil path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` legs may import this package.  The
product package ``paper_2409_18824_gb300`` never imports it and it never
imports the product: the two share no code.  Inputs come from the seeded
generators in ``stencil_inputs`` (random numbers and shapes only).

The arithmetic lives in ``oracle.c`` (plain C, double precision, k-j-i loops,
built with ``-O2 -ffp-contract=off`` so that no multiply-add is fused).  This
module compiles it with gcc into ``liboracle.so`` beside the source and wraps
each function for numpy arrays laid out as the library expects: a C-contiguous
array of shape (nz+2r, ny+2r, nx+2r), which is the Fortran column-major array
u(1:nx+2r, 1:ny+2r, 1:nz+2r) (arXiv 2409.18824 Sec. 5.2, Listing 7).

Two-dimensional grids (the paper's own jacobi benchmark) are C-contiguous
arrays of shape (ny+2r, nx+2r), i fastest; their functions carry a ``2d``
suffix and are pinned in tests/test_oracle_2d.py.

Pins (tests/test_oracle.py): closed-form eigenmode decay, constant and linear
invariants, dense brute force, Gaussian elimination, symmetry of the
variable-coefficient operator.  The constant-coefficient refinement
(``refined_solve``) is pinned step by step in an exact dyadic regime (one
outer step equals numpy's dense iteration bitwise) and by its end state.  The
variable-coefficient refinement driver (``varcoef_refined_solve``) is pinned
the same ways: one outer step bitwise where every Jacobi diagonal is a power
of two, each outer step against the closed form rho -> (N D^-1)^m rho
(A = D - N, m inner sweeps), and its end state.  No function is left
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, no FP contraction, OpenMP off)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        sig = {
            "oracle_sweep_f64": (None, [_dp, _dp, _dp, _i64, _i64, _i64, _dp, ctypes.c_int]),
            "oracle_sweep_f32": (None, [_fp, _fp, _fp, _i64, _i64, _i64, _fp, ctypes.c_int]),
            "oracle_stencil_sweep_f64": (ctypes.c_int, [_dp, _dp, _i64, _i64, _i64, _dp, ctypes.c_int, _i64]),
            "oracle_stencil_sweep_f32": (ctypes.c_int, [_fp, _fp, _i64, _i64, _i64, _fp, ctypes.c_int, _i64]),
            "oracle_residual_norm_f64": (ctypes.c_double, [_dp, _dp, _i64, _i64, _i64, _dp, ctypes.c_int]),
            "oracle_residual_norm_f32": (ctypes.c_double, [_fp, _fp, _i64, _i64, _i64, _fp, ctypes.c_int]),
            "oracle_interior_norm_f64": (ctypes.c_double, [_dp, _i64, _i64, _i64, ctypes.c_int]),
            "oracle_jacobi_solve_f64": (ctypes.c_int, [_dp, _dp, _i64, _i64, _i64, _dp, ctypes.c_int,
                                                       ctypes.c_double, _i64, _i64,
                                                       ctypes.POINTER(_i64), _dp]),
            "oracle_varcoef_apply_f64": (None, [_dp, _dp, _dp, _i64, _i64, _i64, _dp, ctypes.c_int]),
            "oracle_varcoef_sweep_f64": (None, [_dp, _dp, _dp, _dp, _i64, _i64, _i64, _dp, ctypes.c_int]),
            "oracle_varcoef_sweep_f32": (None, [_fp, _fp, _fp, _fp, _i64, _i64, _i64, _fp, ctypes.c_int]),
            "oracle_varcoef_residual_norm_f64": (ctypes.c_double, [_dp, _dp, _dp, _i64, _i64, _i64, _dp,
                                                                   ctypes.c_int]),
            "oracle_varcoef_jacobi_solve_f64": (ctypes.c_int, [_dp, _dp, _dp, _i64, _i64, _i64, _dp,
                                                               ctypes.c_int, ctypes.c_double, _i64, _i64,
                                                               ctypes.POINTER(_i64), _dp]),
            "oracle_varcoef_refined_solve": (ctypes.c_int, [_dp, _dp, _dp, _i64, _i64, _i64, _dp,
                                                            ctypes.c_int, ctypes.c_double, _i64, _i64,
                                                            ctypes.POINTER(_i64), _dp]),
            "oracle_dense_solve": (ctypes.c_int, [_dp, _dp, _i64]),
            "oracle_sum_f64": (ctypes.c_double, [_dp, _i64]),
            "oracle_advect_f64": (None, [_dp, _dp, _dp, _dp, _dp, _i64, _i64, _i64, _dp]),
            "oracle_advect_f32": (None, [_fp, _fp, _fp, _fp, _fp, _i64, _i64, _i64, _fp]),
            "oracle_dot_f64": (ctypes.c_double, [_dp, _dp, _i64]),
            "oracle_sweep2d_f64": (None, [_dp, _dp, _dp, _i64, _i64, _dp, ctypes.c_int]),
            "oracle_sweep2d_f32": (None, [_fp, _fp, _fp, _i64, _i64, _fp, ctypes.c_int]),
            "oracle_stencil_sweep2d_f64": (ctypes.c_int, [_dp, _dp, _i64, _i64, _dp, ctypes.c_int, _i64]),
            "oracle_stencil_sweep2d_f32": (ctypes.c_int, [_fp, _fp, _i64, _i64, _fp, ctypes.c_int, _i64]),
            "oracle_residual_norm2d_f64": (ctypes.c_double, [_dp, _dp, _i64, _i64, _dp, ctypes.c_int]),
            "oracle_residual_norm2d_f32": (ctypes.c_double, [_fp, _fp, _i64, _i64, _fp, ctypes.c_int]),
            "oracle_refined_solve_f64": (ctypes.c_int, [_dp, _dp, _i64, _i64, _i64, _dp, ctypes.c_int,
                                                        ctypes.c_double, _i64, _i64, ctypes.POINTER(_i64), _dp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _grid(a: np.ndarray, dtype) -> np.ndarray:
    if a.dtype != dtype or not a.flags["C_CONTIGUOUS"] or a.ndim != 3:
        raise ValueError(f"oracle wants a C-contiguous 3D {np.dtype(dtype).name} array, got "
                         f"{a.dtype} {a.shape}")
    return a


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def interior_shape(u: np.ndarray, r: int):
    nz, ny, nx = (s - 2 * r for s in u.shape)
    if min(nx, ny, nz) < 1:
        raise ValueError("grid smaller than its halo")
    return nx, ny, nz


def sweep(u: np.ndarray, coeffs, r: int, b: np.ndarray | None = None) -> np.ndarray:
    """One sweep; returns a new padded array whose halo is u's halo."""
    lib = _load()
    if u.dtype == np.float64:
        _grid(u, np.float64)
        out = u.copy()
        c = np.ascontiguousarray(coeffs, dtype=np.float64)
        if b is not None:
            _grid(b, np.float64)
        lib.oracle_sweep_f64(_ptr(u, ctypes.c_double), _ptr(b, ctypes.c_double), _ptr(out, ctypes.c_double),
                             *interior_shape(u, r), _ptr(c, ctypes.c_double), r)
    elif u.dtype == np.float32:
        _grid(u, np.float32)
        out = u.copy()
        c = np.asarray(coeffs, dtype=np.float64).astype(np.float32)
        if b is not None:
            _grid(b, np.float32)
        lib.oracle_sweep_f32(_ptr(u, ctypes.c_float), _ptr(b, ctypes.c_float), _ptr(out, ctypes.c_float),
                             *interior_shape(u, r), _ptr(c, ctypes.c_float), r)
    else:
        raise TypeError(u.dtype)
    return out


def stencil_sweep(u: np.ndarray, coeffs, r: int, iters: int) -> np.ndarray:
    """`iters` sweeps (no source term), returns the final padded grid."""
    lib = _load()
    out = np.empty_like(u)
    if u.dtype == np.float64:
        c = np.ascontiguousarray(coeffs, dtype=np.float64)
        rc = lib.oracle_stencil_sweep_f64(_ptr(u, ctypes.c_double), _ptr(out, ctypes.c_double),
                                          *interior_shape(u, r), _ptr(c, ctypes.c_double), r, iters)
    else:
        c = np.asarray(coeffs, dtype=np.float64).astype(np.float32)
        rc = lib.oracle_stencil_sweep_f32(_ptr(_grid(u, np.float32), ctypes.c_float), _ptr(out, ctypes.c_float),
                                          *interior_shape(u, r), _ptr(c, ctypes.c_float), r, iters)
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return out


def residual_norm(u: np.ndarray, coeffs, r: int, b: np.ndarray | None = None) -> float:
    lib = _load()
    if u.dtype == np.float64:
        c = np.ascontiguousarray(coeffs, dtype=np.float64)
        return lib.oracle_residual_norm_f64(_ptr(_grid(u, np.float64), ctypes.c_double), _ptr(b, ctypes.c_double),
                                            *interior_shape(u, r), _ptr(c, ctypes.c_double), r)
    c = np.asarray(coeffs, dtype=np.float64).astype(np.float32)
    return lib.oracle_residual_norm_f32(_ptr(_grid(u, np.float32), ctypes.c_float), _ptr(b, ctypes.c_float),
                                        *interior_shape(u, r), _ptr(c, ctypes.c_float), r)


def interior_norm(x: np.ndarray, r: int) -> float:
    lib = _load()
    return lib.oracle_interior_norm_f64(_ptr(_grid(x, np.float64), ctypes.c_double), *interior_shape(x, r), r)


def jacobi_solve(b: np.ndarray | None, u0: np.ndarray, coeffs, r: int, tol: float, max_iters: int,
                 check_every: int):
    """Returns (u, iters, rel_res, status) with status 0 converged / 1 not."""
    lib = _load()
    u = _grid(u0, np.float64).copy()
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    it = _i64(0)
    rel = ctypes.c_double(0.0)
    st = lib.oracle_jacobi_solve_f64(_ptr(b, ctypes.c_double), _ptr(u, ctypes.c_double), *interior_shape(u, r),
                                     _ptr(c, ctypes.c_double), r, tol, max_iters, check_every,
                                     ctypes.byref(it), ctypes.byref(rel))
    if st < 0:
        raise MemoryError("oracle allocation failed")
    return u, it.value, rel.value, st


# ------------------------------------------------------------- advection --
def advect(u, v, w, q, c) -> np.ndarray:
    """Tendency of q under the velocity (u, v, w) (flux-form centred advection,
    halo 1); the result's halo is zero."""
    lib = _load()
    dt = u.dtype.type
    for a in (u, v, w, q):
        _grid(a, dt)
        if a.shape != u.shape:
            raise ValueError("shape mismatch")
    s = np.zeros_like(u)
    nx, ny, nz = interior_shape(u, 1)
    if dt == np.float64:
        cc = np.ascontiguousarray(c, dtype=np.float64)
        lib.oracle_advect_f64(*(_ptr(a, ctypes.c_double) for a in (u, v, w, q, s)), nx, ny, nz,
                              _ptr(cc, ctypes.c_double))
    else:
        cc = np.asarray(c, dtype=np.float64).astype(np.float32)
        lib.oracle_advect_f32(*(_ptr(a, ctypes.c_float) for a in (u, v, w, q, s)), nx, ny, nz,
                              _ptr(cc, ctypes.c_float))
    return s


# -------------------------------------------------------- sum, dotproduct --
def _vec(a):
    if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("oracle wants a C-contiguous float64 array")
    return a


def sum_(x: np.ndarray) -> float:
    """The sum intrinsic: sequential add-reduction from zero (Sec. 5.3)."""
    return _load().oracle_sum_f64(_ptr(_vec(x), ctypes.c_double), x.size)


def dot(x: np.ndarray, y: np.ndarray) -> float:
    """The dotproduct intrinsic: sequential add-reduction of x_i * y_i from zero."""
    if x.size != y.size:
        raise ValueError("length mismatch")
    return _load().oracle_dot_f64(_ptr(_vec(x), ctypes.c_double), _ptr(_vec(y), ctypes.c_double), x.size)


# ------------------------------------------------------------------- 2-D --
def _grid2(a: np.ndarray, dtype) -> np.ndarray:
    if a.dtype != dtype or not a.flags["C_CONTIGUOUS"] or a.ndim != 2:
        raise ValueError(f"oracle wants a C-contiguous 2D {np.dtype(dtype).name} array, got "
                         f"{a.dtype} {a.shape}")
    return a


def interior_shape2d(u: np.ndarray, r: int):
    ny, nx = (s - 2 * r for s in u.shape)
    if min(nx, ny) < 1:
        raise ValueError("grid smaller than its halo")
    return nx, ny


def _c2(coeffs, dtype):
    c = np.asarray(coeffs, dtype=np.float64)
    return np.ascontiguousarray(c if dtype == np.float64 else c.astype(np.float32))


def sweep2d(u: np.ndarray, coeffs, r: int, b: np.ndarray | None = None) -> np.ndarray:
    """One 2-D sweep of a padded (ny+2r, nx+2r) array; the halo is copied."""
    lib = _load()
    dt = u.dtype.type
    _grid2(u, dt)
    if b is not None:
        _grid2(b, dt)
    out = u.copy()
    c = _c2(coeffs, dt)
    if dt == np.float64:
        lib.oracle_sweep2d_f64(_ptr(u, ctypes.c_double), _ptr(b, ctypes.c_double), _ptr(out, ctypes.c_double),
                               *interior_shape2d(u, r), _ptr(c, ctypes.c_double), r)
    else:
        lib.oracle_sweep2d_f32(_ptr(u, ctypes.c_float), _ptr(b, ctypes.c_float), _ptr(out, ctypes.c_float),
                               *interior_shape2d(u, r), _ptr(c, ctypes.c_float), r)
    return out


def stencil_sweep2d(u: np.ndarray, coeffs, r: int, iters: int) -> np.ndarray:
    """`iters` 2-D sweeps (no source term); returns the final padded grid."""
    lib = _load()
    dt = u.dtype.type
    _grid2(u, dt)
    out = np.empty_like(u)
    c = _c2(coeffs, dt)
    if dt == np.float64:
        rc = lib.oracle_stencil_sweep2d_f64(_ptr(u, ctypes.c_double), _ptr(out, ctypes.c_double),
                                            *interior_shape2d(u, r), _ptr(c, ctypes.c_double), r, iters)
    else:
        rc = lib.oracle_stencil_sweep2d_f32(_ptr(u, ctypes.c_float), _ptr(out, ctypes.c_float),
                                            *interior_shape2d(u, r), _ptr(c, ctypes.c_float), r, iters)
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return out


def residual_norm2d(u: np.ndarray, coeffs, r: int, b: np.ndarray | None = None) -> float:
    lib = _load()
    dt = u.dtype.type
    _grid2(u, dt)
    if b is not None:
        _grid2(b, dt)
    c = _c2(coeffs, dt)
    if dt == np.float64:
        return lib.oracle_residual_norm2d_f64(_ptr(u, ctypes.c_double), _ptr(b, ctypes.c_double),
                                              *interior_shape2d(u, r), _ptr(c, ctypes.c_double), r)
    return lib.oracle_residual_norm2d_f32(_ptr(u, ctypes.c_float), _ptr(b, ctypes.c_float),
                                          *interior_shape2d(u, r), _ptr(c, ctypes.c_float), r)


def _w3(w):
    w = np.asarray(w, dtype=np.float64)
    out = np.zeros(3, dtype=np.float64)
    out[1:1 + len(w) - 1] = w[1:]
    return out


def varcoef_apply(u: np.ndarray, a: np.ndarray, w, R: int) -> np.ndarray:
    """A u on the interior (halo of the result: zero)."""
    lib = _load()
    out = np.zeros_like(_grid(u, np.float64))
    ww = _w3(w)
    lib.oracle_varcoef_apply_f64(_ptr(u, ctypes.c_double), _ptr(_grid(a, np.float64), ctypes.c_double),
                                 _ptr(out, ctypes.c_double), *interior_shape(u, R), _ptr(ww, ctypes.c_double), R)
    return out


def varcoef_sweep(u: np.ndarray, a: np.ndarray, f: np.ndarray, w, R: int) -> np.ndarray:
    lib = _load()
    out = u.copy()
    if u.dtype == np.float64:
        ww = _w3(w)
        lib.oracle_varcoef_sweep_f64(_ptr(u, ctypes.c_double), _ptr(_grid(a, np.float64), ctypes.c_double),
                                     _ptr(_grid(f, np.float64), ctypes.c_double), _ptr(out, ctypes.c_double),
                                     *interior_shape(u, R), _ptr(ww, ctypes.c_double), R)
    else:
        ww = _w3(w).astype(np.float32)
        lib.oracle_varcoef_sweep_f32(_ptr(_grid(u, np.float32), ctypes.c_float),
                                     _ptr(_grid(a, np.float32), ctypes.c_float),
                                     _ptr(_grid(f, np.float32), ctypes.c_float), _ptr(out, ctypes.c_float),
                                     *interior_shape(u, R), _ptr(ww, ctypes.c_float), R)
    return out


def varcoef_residual_norm(u: np.ndarray, a: np.ndarray, f: np.ndarray, w, R: int) -> float:
    lib = _load()
    ww = _w3(w)
    return lib.oracle_varcoef_residual_norm_f64(_ptr(_grid(u, np.float64), ctypes.c_double),
                                                _ptr(_grid(a, np.float64), ctypes.c_double),
                                                _ptr(_grid(f, np.float64), ctypes.c_double),
                                                *interior_shape(u, R), _ptr(ww, ctypes.c_double), R)


def varcoef_jacobi_solve(a, f, u0, w, R, tol, max_iters, check_every):
    lib = _load()
    u = _grid(u0, np.float64).copy()
    ww = _w3(w)
    it = _i64(0)
    rel = ctypes.c_double(0.0)
    st = lib.oracle_varcoef_jacobi_solve_f64(_ptr(_grid(a, np.float64), ctypes.c_double),
                                             _ptr(_grid(f, np.float64), ctypes.c_double),
                                             _ptr(u, ctypes.c_double), *interior_shape(u, R),
                                             _ptr(ww, ctypes.c_double), R, tol, max_iters, check_every,
                                             ctypes.byref(it), ctypes.byref(rel))
    if st < 0:
        raise MemoryError("oracle allocation failed")
    return u, it.value, rel.value, st


def varcoef_refined_solve(a, f, u0, w, R, tol, inner_sweeps, max_outer):
    lib = _load()
    u = _grid(u0, np.float64).copy()
    ww = _w3(w)
    outer = _i64(0)
    rel = ctypes.c_double(0.0)
    st = lib.oracle_varcoef_refined_solve(_ptr(_grid(a, np.float64), ctypes.c_double),
                                          _ptr(_grid(f, np.float64), ctypes.c_double),
                                          _ptr(u, ctypes.c_double), *interior_shape(u, R),
                                          _ptr(ww, ctypes.c_double), R, tol, inner_sweeps, max_outer,
                                          ctypes.byref(outer), ctypes.byref(rel))
    if st < 0:
        raise MemoryError("oracle allocation failed")
    return u, outer.value, rel.value, st


def refined_solve(b, u0, coeffs, r, tol, inner_sweeps, max_outer):
    """Constant-coefficient refinement; returns (u, outer, rel_res, status)."""
    lib = _load()
    u = _grid(u0, np.float64).copy()
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    outer = _i64(0)
    rel = ctypes.c_double(0.0)
    st = lib.oracle_refined_solve_f64(_ptr(b, ctypes.c_double), _ptr(u, ctypes.c_double), *interior_shape(u, r),
                                      _ptr(c, ctypes.c_double), r, tol, inner_sweeps, max_outer,
                                      ctypes.byref(outer), ctypes.byref(rel))
    if st < 0:
        raise MemoryError("oracle allocation failed")
    return u, outer.value, rel.value, st


def dense_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Gaussian elimination with partial pivoting (textbook, in oracle.c)."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.float64).copy()
    x = np.ascontiguousarray(b, dtype=np.float64).copy()
    n = A.shape[0]
    if lib.oracle_dense_solve(_ptr(A, ctypes.c_double), _ptr(x, ctypes.c_double), n) != 0:
        raise np.linalg.LinAlgError("singular")
    return x
