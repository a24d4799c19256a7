"""Thin binding of libstencil_host.so (C ABI in include/stencil_host.h): the
multi-core host path of the Jacobi sweep, the paper's threaded jacobi
(arXiv 2409.18824 Sec. 6.2, Table 4).  A separate library that the GPU path
never calls.  Grids are numpy arrays (or raw host addresses) in the layout
of the GPU calls: C-contiguous (nz+2r, ny+2r, nx+2r) or (ny+2r, nx+2r).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstencil_host.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it first "
                      "(python -c 'import __graft_entry__ as g; g.build()')")

_lib = ctypes.CDLL(LIB_PATH)
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dp = ctypes.POINTER(ctypes.c_double)

#: every entry point of include/stencil_host.h with (restype, argtypes)
SIGNATURES = {
    "stencil_host_last_error": (ctypes.c_char_p, []),
    "stencil_host_threads": (_int, []),
    "stencil_host_sweep_f64": (_int, [_vp, _vp, _i64, _i64, _i64, _dp, _int, _i64, _int]),
    "stencil_host_residual_norm_f64": (_int, [_vp, _vp, _i64, _i64, _i64, _dp, _int, _dp, _int]),
    "stencil_host_sweep2d_f64": (_int, [_vp, _vp, _i64, _i64, _dp, _int, _i64, _int]),
    "stencil_host_residual_norm2d_f64": (_int, [_vp, _vp, _i64, _i64, _dp, _int, _dp, _int]),
    "stencil_host_advect_f64": (_int, [_vp, _vp, _vp, ctypes.POINTER(_vp), _int, ctypes.POINTER(_vp), _i64, _i64,
                                       _i64, _dp, _int]),
}
for _name, (_res, _args) in SIGNATURES.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


class HostStencilError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libstencil_host error {code}: {msg}")
        self.code = code


def lib():
    return _lib


def _check(rc):
    if rc < 0:
        raise HostStencilError(rc, _lib.stencil_host_last_error().decode())
    return rc


def _addr(x, shape=None):
    """Address of a host grid: a C-contiguous float64 array, of `shape` when
    given (every grid of a call has the shape of its first), or a raw address
    the caller vouches for."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not (isinstance(x, np.ndarray) and x.flags.c_contiguous and x.dtype == np.float64):
        raise TypeError("host grids are C-contiguous float64 numpy arrays")
    if shape is not None and x.shape != tuple(shape):
        raise ValueError(f"grid of shape {x.shape}, the call's grids are {tuple(shape)}")
    return x.ctypes.data


def _coeffs(c):
    arr = (ctypes.c_double * len(c))(*[float(v) for v in c])
    return ctypes.cast(arr, _dp), arr


def threads() -> int:
    return _lib.stencil_host_threads()


def stencil_host_sweep_f64(in_, out, coeffs, radius, iters, nthreads=0):
    nz, ny, nx = (d - 2 * radius for d in in_.shape)
    cp, _keep = _coeffs(coeffs)
    return _check(_lib.stencil_host_sweep_f64(_addr(in_), _addr(out, in_.shape), nx, ny, nz, cp, radius, iters, nthreads))


def stencil_host_residual_norm_f64(u, coeffs, radius, b=None, nthreads=0) -> float:
    nz, ny, nx = (d - 2 * radius for d in u.shape)
    cp, _keep = _coeffs(coeffs)
    v = ctypes.c_double(0.0)
    _check(_lib.stencil_host_residual_norm_f64(_addr(u), _addr(b, u.shape), nx, ny, nz, cp, radius, ctypes.byref(v),
                                               nthreads))
    return v.value


def stencil_host_sweep2d_f64(in_, out, coeffs, radius, iters, nthreads=0):
    ny, nx = (d - 2 * radius for d in in_.shape)
    cp, _keep = _coeffs(coeffs)
    return _check(_lib.stencil_host_sweep2d_f64(_addr(in_), _addr(out, in_.shape), nx, ny, cp, radius, iters, nthreads))


def stencil_host_residual_norm2d_f64(u, coeffs, radius, b=None, nthreads=0) -> float:
    ny, nx = (d - 2 * radius for d in u.shape)
    cp, _keep = _coeffs(coeffs)
    v = ctypes.c_double(0.0)
    _check(_lib.stencil_host_residual_norm2d_f64(_addr(u), _addr(b, u.shape), nx, ny, cp, radius, ctypes.byref(v),
                                                 nthreads))
    return v.value


def stencil_host_advect_f64(u, v, w, s, c, q=None, nthreads=0):
    """Tendencies of q (a list of fields; None: u, v, w themselves) into the
    list s; halo-1 grids of shape (nz+2, ny+2, nx+2)."""
    nz, ny, nx = (d - 2 for d in u.shape)
    cp, _keep = _coeffs(c)
    qa = None if q is None else (_vp * len(q))(*[_addr(x, u.shape) for x in q])
    sa = (_vp * len(s))(*[_addr(x, u.shape) for x in s])
    return _check(_lib.stencil_host_advect_f64(_addr(u), _addr(v, u.shape), _addr(w, u.shape), qa, 0 if q is None else len(q), sa,
                                               nx, ny, nz, cp, nthreads))
