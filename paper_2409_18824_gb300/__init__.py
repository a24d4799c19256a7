"""Thin Python binding of libstencil.so (C ABI in include/stencil.h).

The functions below have the C ABI's names and only marshal arguments: every
step of the Jacobi path runs in the library's CUDA kernels.  Grid arguments
may be torch tensors (CUDA or CPU), numpy arrays, or raw integer addresses;
a grid is the Fortran array u(1:nx+2r, 1:ny+2r, 1:nz+2r), i.e. a C-contiguous
array of shape (nz+2r, ny+2r, nx+2r) (arXiv 2409.18824 Sec. 5.2, Listing 7).
For tensor / array arguments the interior extents are taken from the shape
when not given.

There is no CPU fallback: importing this package raises if libstencil.so has
not been built (``python -c "import __graft_entry__ as g; g.build()"``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstencil.so")

STN_OK = 0
STN_NOT_CONVERGED = 1
STN_EINVAL = -1
STN_ENOMEM = -2
STN_ECUDA = -3
STN_ETIMEOUT = -4
STN_EBUSY = -5
STN_PENDING = 2


class StencilError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libstencil error {code}: {msg}")
        self.code = code


class Problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
                ("rhs", ctypes.c_void_p), ("u", ctypes.c_void_p)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("outer", ctypes.c_int64), ("rel_res", ctypes.c_double),
                ("res_norm", ctypes.c_double), ("rhs_norm", ctypes.c_double), ("status", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("radius", ctypes.c_int), ("coeffs", ctypes.c_double * 3),
                ("tol", ctypes.c_double), ("refined", ctypes.c_int), ("max_iters", ctypes.c_int64),
                ("inner_sweeps", ctypes.c_int64), ("inner_tol", ctypes.c_double), ("check_every", ctypes.c_int64),
                ("max_outer", ctypes.c_int64), ("max_inflight", ctypes.c_int), ("queue_capacity", ctypes.c_int),
                ("engine", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
                ("rhs", ctypes.c_void_p), ("u0", ctypes.c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("info", SolveInfo), ("latency_s", ctypes.c_double), ("queue_s", ctypes.c_double),
                ("rc", ctypes.c_int)]

    def as_dict(self):
        d = self.info.as_dict()
        d.update(latency_s=self.latency_s, queue_s=self.queue_s, rc=self.rc)
        return d


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("pending", ctypes.c_int64),
                ("running", ctypes.c_int64), ("bytes_in_use", ctypes.c_size_t), ("status", ctypes.c_int)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("device", ctypes.c_char * 64), ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("nz", ctypes.c_int64), ("esize", ctypes.c_int32), ("radius", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("chunks", ctypes.c_int32), ("depth", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("glups", ctypes.c_double), ("default_glups", ctypes.c_double)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}
        d["device"] = self.device.decode()
        return d


class LaunchPlan(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int32) for f in ("variant", "grid_x", "grid_y", "grid_z", "block_threads", "tile_w",
                                              "tile_h", "kchunk", "stage_elems", "smem_bytes", "row_stride",
                                              "row_pad", "bulk_copy", "reserved")] + [
        ("scratch_bytes", ctypes.c_int64), ("xchg_offset", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                      "(python -c 'import __graft_entry__ as g; g.build()')")

_lib = ctypes.CDLL(LIB_PATH)
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double
_dp = ctypes.POINTER(ctypes.c_double)
_info_p = ctypes.POINTER(SolveInfo)

#: every entry point of include/stencil.h with (restype, argtypes)
SIGNATURES = {
    "stencil_last_error": (ctypes.c_char_p, []),
    "stencil_version": (ctypes.c_char_p, []),
    "stencil_release_workspace": (_int, []),
    "stencil_tune_set": (_int, [ctypes.c_char_p, _i64]),
    "stencil_tune_get": (_int, [ctypes.c_char_p, ctypes.POINTER(_i64)]),
    "stencil_sched_stats": (_int, [ctypes.POINTER(ctypes.c_uint64), _int]),
    "stencil_autotune_sweep": (_int, [_i64, _i64, _i64, _int, _int, _dp, _int, ctypes.POINTER(TuneEntry), _vp]),
    "stencil_tune_cache_put": (_int, [ctypes.POINTER(TuneEntry)]),
    "stencil_tune_cache_get": (_int, [ctypes.c_char_p, _i64, _i64, _i64, _int, _int, ctypes.POINTER(TuneEntry)]),
    "stencil_tune_cache_size": (_i64, []),
    "stencil_tune_cache_clear": (_int, []),
    "stencil_tune_cache_save": (_int, [ctypes.c_char_p]),
    "stencil_tune_cache_load": (_int, [ctypes.c_char_p]),
    "stencil_plan_query": (_int, [ctypes.c_char_p, _i64, _i64, _i64, _int, _int, ctypes.POINTER(LaunchPlan)]),
    "stencil_sweep_f64": (_int, [_vp, _vp, _i64, _i64, _i64, _dp, _int, _i64, _vp]),
    "stencil_sweep_f32": (_int, [_vp, _vp, _i64, _i64, _i64, _dp, _int, _i64, _vp]),
    "stencil_apply_f64": (_int, [_vp, _vp, _vp, _i64, _i64, _i64, _dp, _int, _vp]),
    "stencil_apply_f32": (_int, [_vp, _vp, _vp, _i64, _i64, _i64, _dp, _int, _vp]),
    "residual_norm_f64": (_int, [_vp, _vp, _i64, _i64, _i64, _dp, _int, _dp, _vp]),
    "residual_norm_f32": (_int, [_vp, _vp, _i64, _i64, _i64, _dp, _int, _dp, _vp]),
    "residual_norm_f64_noalloc": (_int, [_vp, _vp, _i64, _i64, _i64, _dp, _int, _dp, _vp]),
    "reduce_sum_f64": (_int, [_vp, _i64, _dp, _vp]),
    "advect_f64": (_int, [_vp, _vp, _vp, ctypes.POINTER(_vp), _int, ctypes.POINTER(_vp), _i64, _i64, _i64, _dp, _vp]),
    "advect_f32": (_int, [_vp, _vp, _vp, ctypes.POINTER(_vp), _int, ctypes.POINTER(_vp), _i64, _i64, _i64, _dp, _vp]),
    "dot_f64": (_int, [_vp, _vp, _i64, _dp, _vp]),
    "stencil_sweep2d_f64": (_int, [_vp, _vp, _i64, _i64, _dp, _int, _i64, _vp]),
    "stencil_sweep2d_f32": (_int, [_vp, _vp, _i64, _i64, _dp, _int, _i64, _vp]),
    "residual_norm2d_f64": (_int, [_vp, _vp, _i64, _i64, _dp, _int, _dp, _vp]),
    "residual_norm2d_f32": (_int, [_vp, _vp, _i64, _i64, _dp, _int, _dp, _vp]),
    "jacobi_solve_f64": (_int, [_vp, _vp, _i64, _i64, _i64, _dp, _int, _dbl, _i64, _i64, _info_p, _vp]),
    "jacobi_solve_refined_f64": (_int, [_vp, _vp, _i64, _i64, _i64, _dp, _int, _dbl, _i64, _dbl, _i64, _i64,
                                        _info_p, _vp]),
    "jacobi_solve_batched_f64": (_int, [ctypes.POINTER(Problem), _i64, _dp, _int, _dbl, _i64, _i64, _info_p,
                                        _vp]),
    "jacobi_solve_batched_refined": (_int, [ctypes.POINTER(Problem), _i64, _dp, _int, _dbl, _i64, _dbl, _i64,
                                            _i64, _info_p, _vp]),
    "stn_server_create": (_vp, [ctypes.POINTER(ServerOpts)]),
    "stn_submit": (_int, [_vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "stn_poll": (_int, [_vp, ctypes.c_uint64, ctypes.POINTER(Result)]),
    "stn_wait": (_int, [_vp, ctypes.c_uint64, _dbl, ctypes.POINTER(Result)]),
    "stn_result_copy": (_int, [_vp, ctypes.c_uint64, _vp]),
    "stn_release": (_int, [_vp, ctypes.c_uint64]),
    "stn_server_stats": (_int, [_vp, ctypes.POINTER(ServerStats)]),
    "stn_server_destroy": (None, [_vp]),
    "varcoef_apply_f64": (_int, [_vp, _vp, _vp, _i64, _i64, _i64, _dp, _int, _vp]),
    "varcoef_sweep_f64": (_int, [_vp, _vp, _vp, _vp, _i64, _i64, _i64, _dp, _int, _i64, _vp]),
    "varcoef_sweep_f32": (_int, [_vp, _vp, _vp, _vp, _i64, _i64, _i64, _dp, _int, _i64, _vp]),
    "varcoef_residual_norm_f64": (_int, [_vp, _vp, _vp, _i64, _i64, _i64, _dp, _int, _dp, _vp]),
    "jacobi_solve_varcoef_f64": (_int, [_vp, _vp, _vp, _i64, _i64, _i64, _dp, _int, _dbl, _i64, _i64,
                                        _info_p, _vp]),
    "jacobi_solve_varcoef_refined": (_int, [_vp, _vp, _vp, _i64, _i64, _i64, _dp, _int, _dbl, _i64, _i64,
                                            _info_p, _vp]),
}
for _name, (_res, _args) in SIGNATURES.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def lib() -> ctypes.CDLL:
    return _lib


def last_error() -> str:
    return _lib.stencil_last_error().decode()


def version() -> str:
    return _lib.stencil_version().decode()


# ------------------------------------------------------------- marshalling --
def _buffer_check(is_float, itemsize, n, esize, count):
    if esize is not None and (not is_float or itemsize != esize):
        raise TypeError(f"grid of {itemsize}-byte {'floats' if is_float else 'non-floats'}: this call takes "
                        f"{esize}-byte floats")
    if count is not None and n < count:
        raise ValueError(f"grid holds {n} elements, the extents need {count}")


def _addr(x, esize=None, count=None):
    """Address of a grid argument (torch tensor, numpy array, int or None).
    Arrays and tensors must be contiguous, hold floats of `esize` bytes and at
    least `count` elements, so that the kernels never run past them; a raw
    address (int) is the caller's to vouch for."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("grid arrays must be C-contiguous (Fortran column-major u(i,j,k))")
        _buffer_check(x.dtype.kind == "f", x.itemsize, x.size, esize, count)
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("grid tensors must be contiguous (Fortran column-major u(i,j,k))")
        _buffer_check(x.is_floating_point(), x.element_size(), x.numel(), esize, count)
        return x.data_ptr()
    raise TypeError(f"unsupported grid argument {type(x)}")


def _n3(nx, ny, nz, r):
    return (nx + 2 * r) * (ny + 2 * r) * (nz + 2 * r)


def _n2(nx, ny, r):
    return (nx + 2 * r) * (ny + 2 * r)


def _stream(stream, *grids):
    """cudaStream_t for the call: explicit, else torch's current stream when a
    grid is a CUDA tensor, else NULL (legacy default stream)."""
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    for g in grids:
        if hasattr(g, "is_cuda") and g.is_cuda:
            import torch
            return torch.cuda.current_stream(g.device).cuda_stream
    return None


def _coeffs(c):
    arr = (ctypes.c_double * len(c))(*[float(v) for v in c])
    return ctypes.cast(arr, _dp), arr


def _extents(grid, r, nx, ny, nz):
    if nx is not None:
        return nx, ny, nz
    shape = tuple(grid.shape)
    if len(shape) != 3:
        raise ValueError("pass nx, ny, nz or a 3D grid")
    return shape[2] - 2 * r, shape[1] - 2 * r, shape[0] - 2 * r


def _extents2d(grid, r, nx, ny):
    if nx is not None:
        return nx, ny
    shape = tuple(grid.shape)
    if len(shape) != 2:
        raise ValueError("pass nx, ny or a 2D grid")
    return shape[1] - 2 * r, shape[0] - 2 * r


def _check(rc):
    if rc < 0:
        raise StencilError(rc, last_error())
    return rc


# ------------------------------------------------------------ entry points --
def stencil_sweep_f64(in_, out, coeffs, radius, iters, nx=None, ny=None, nz=None, stream=None):
    nx, ny, nz = _extents(in_, radius, nx, ny, nz)
    cp, _keep = _coeffs(coeffs)
    return _check(_lib.stencil_sweep_f64(_addr(in_, 8, _n3(nx, ny, nz, radius)), _addr(out, 8, _n3(nx, ny, nz, radius)), nx, ny, nz, cp, radius, iters,
                                         _stream(stream, in_, out)))


def stencil_sweep_f32(in_, out, coeffs, radius, iters, nx=None, ny=None, nz=None, stream=None):
    nx, ny, nz = _extents(in_, radius, nx, ny, nz)
    cp, _keep = _coeffs(coeffs)
    return _check(_lib.stencil_sweep_f32(_addr(in_, 4, _n3(nx, ny, nz, radius)), _addr(out, 4, _n3(nx, ny, nz, radius)), nx, ny, nz, cp, radius, iters,
                                         _stream(stream, in_, out)))


def stencil_apply_f64(u, out, coeffs, radius, b=None, nx=None, ny=None, nz=None, stream=None):
    nx, ny, nz = _extents(u, radius, nx, ny, nz)
    cp, _keep = _coeffs(coeffs)
    return _check(_lib.stencil_apply_f64(_addr(u, 8, _n3(nx, ny, nz, radius)), _addr(b, 8, _n3(nx, ny, nz, radius)), _addr(out, 8, _n3(nx, ny, nz, radius)), nx, ny, nz, cp, radius,
                                         _stream(stream, u, out, b)))


def stencil_apply_f32(u, out, coeffs, radius, b=None, nx=None, ny=None, nz=None, stream=None):
    nx, ny, nz = _extents(u, radius, nx, ny, nz)
    cp, _keep = _coeffs(coeffs)
    return _check(_lib.stencil_apply_f32(_addr(u, 4, _n3(nx, ny, nz, radius)), _addr(b, 4, _n3(nx, ny, nz, radius)), _addr(out, 4, _n3(nx, ny, nz, radius)), nx, ny, nz, cp, radius,
                                         _stream(stream, u, out, b)))


def residual_norm_f64(u, coeffs, radius, b=None, nx=None, ny=None, nz=None, stream=None) -> float:
    nx, ny, nz = _extents(u, radius, nx, ny, nz)
    cp, _keep = _coeffs(coeffs)
    out = ctypes.c_double(0.0)
    _check(_lib.residual_norm_f64(_addr(u, 8, _n3(nx, ny, nz, radius)), _addr(b, 8, _n3(nx, ny, nz, radius)), nx, ny, nz, cp, radius, ctypes.byref(out),
                                  _stream(stream, u, b)))
    return out.value


def residual_norm_f32(u, coeffs, radius, b=None, nx=None, ny=None, nz=None, stream=None) -> float:
    nx, ny, nz = _extents(u, radius, nx, ny, nz)
    cp, _keep = _coeffs(coeffs)
    out = ctypes.c_double(0.0)
    _check(_lib.residual_norm_f32(_addr(u, 4, _n3(nx, ny, nz, radius)), _addr(b, 4, _n3(nx, ny, nz, radius)), nx, ny, nz, cp, radius, ctypes.byref(out),
                                  _stream(stream, u, b)))
    return out.value


def residual_norm_f64_noalloc(u, coeffs, radius, b=None, nx=None, ny=None, nz=None, stream=None) -> float:
    """residual_norm_f64 without any allocation (device grids only; see include/stencil.h)."""
    nx, ny, nz = _extents(u, radius, nx, ny, nz)
    cp, _keep = _coeffs(coeffs)
    out = ctypes.c_double(0.0)
    _check(_lib.residual_norm_f64_noalloc(_addr(u, 8, _n3(nx, ny, nz, radius)), _addr(b, 8, _n3(nx, ny, nz, radius)), nx, ny, nz, cp, radius, ctypes.byref(out),
                                          _stream(stream, u, b)))
    return out.value


def _numel(a, n):
    if n is not None:
        return n
    return int(a.numel()) if hasattr(a, "numel") else int(a.size)


def _advect(fn, esize, u, v, w, s, c, q, nx, ny, nz, stream):
    nx, ny, nz = _extents(u, 1, nx, ny, nz)
    n = _n3(nx, ny, nz, 1)
    cp, _keep = _coeffs(c)
    outs = (_vp * len(s))(*[_addr(x, esize, n) for x in s])
    if q is None:
        qs, nq = None, 3
    else:
        qs = (_vp * len(q))(*[_addr(x, esize, n) for x in q])
        nq = len(q)
    return _check(fn(_addr(u, esize, n), _addr(v, esize, n), _addr(w, esize, n), qs, nq, outs, nx, ny, nz, cp, _stream(stream, u, v, w)))


def advect_f64(u, v, w, s, c, q=None, nx=None, ny=None, nz=None, stream=None):
    """Tendencies s[m] of fields q[m] under the velocity (u, v, w) (flux-form
    centred advection); q=None: the velocity components advect themselves."""
    return _advect(_lib.advect_f64, 8, u, v, w, s, c, q, nx, ny, nz, stream)


def advect_f32(u, v, w, s, c, q=None, nx=None, ny=None, nz=None, stream=None):
    return _advect(_lib.advect_f32, 4, u, v, w, s, c, q, nx, ny, nz, stream)


def reduce_sum_f64(x, n=None, stream=None) -> float:
    """Sum of the n contiguous doubles of x (the sum intrinsic)."""
    out = ctypes.c_double(0.0)
    n = _numel(x, n)
    _check(_lib.reduce_sum_f64(_addr(x, 8, n), n, ctypes.byref(out), _stream(stream, x)))
    return out.value


def dot_f64(x, y, n=None, stream=None) -> float:
    """Dot product of two contiguous double vectors (the dotproduct intrinsic)."""
    out = ctypes.c_double(0.0)
    n = _numel(x, n)
    _check(_lib.dot_f64(_addr(x, 8, n), _addr(y, 8, n), n, ctypes.byref(out), _stream(stream, x, y)))
    return out.value


def stencil_sweep2d_f64(in_, out, coeffs, radius, iters, nx=None, ny=None, stream=None):
    """`iters` 2-D sweeps of a padded (ny+2r, nx+2r) grid (synchronising)."""
    nx, ny = _extents2d(in_, radius, nx, ny)
    cp, _keep = _coeffs(coeffs)
    return _check(_lib.stencil_sweep2d_f64(_addr(in_, 8, _n2(nx, ny, radius)), _addr(out, 8, _n2(nx, ny, radius)), nx, ny, cp, radius, iters,
                                           _stream(stream, in_, out)))


def stencil_sweep2d_f32(in_, out, coeffs, radius, iters, nx=None, ny=None, stream=None):
    nx, ny = _extents2d(in_, radius, nx, ny)
    cp, _keep = _coeffs(coeffs)
    return _check(_lib.stencil_sweep2d_f32(_addr(in_, 4, _n2(nx, ny, radius)), _addr(out, 4, _n2(nx, ny, radius)), nx, ny, cp, radius, iters,
                                           _stream(stream, in_, out)))


def residual_norm2d_f64(u, coeffs, radius, b=None, nx=None, ny=None, stream=None) -> float:
    nx, ny = _extents2d(u, radius, nx, ny)
    cp, _keep = _coeffs(coeffs)
    out = ctypes.c_double(0.0)
    _check(_lib.residual_norm2d_f64(_addr(u, 8, _n2(nx, ny, radius)), _addr(b, 8, _n2(nx, ny, radius)), nx, ny, cp, radius, ctypes.byref(out),
                                    _stream(stream, u, b)))
    return out.value


def residual_norm2d_f32(u, coeffs, radius, b=None, nx=None, ny=None, stream=None) -> float:
    nx, ny = _extents2d(u, radius, nx, ny)
    cp, _keep = _coeffs(coeffs)
    out = ctypes.c_double(0.0)
    _check(_lib.residual_norm2d_f32(_addr(u, 4, _n2(nx, ny, radius)), _addr(b, 4, _n2(nx, ny, radius)), nx, ny, cp, radius, ctypes.byref(out),
                                    _stream(stream, u, b)))
    return out.value


def jacobi_solve_f64(rhs, u, coeffs, radius, tol, max_iters, check_every=50, nx=None, ny=None, nz=None,
                     stream=None):
    """Returns (status, info dict)."""
    nx, ny, nz = _extents(u, radius, nx, ny, nz)
    cp, _keep = _coeffs(coeffs)
    info = SolveInfo()
    rc = _check(_lib.jacobi_solve_f64(_addr(rhs, 8, _n3(nx, ny, nz, radius)), _addr(u, 8, _n3(nx, ny, nz, radius)), nx, ny, nz, cp, radius, tol, max_iters,
                                      check_every, ctypes.byref(info), _stream(stream, u, rhs)))
    return rc, info.as_dict()


def jacobi_solve_refined_f64(rhs, u, coeffs, radius, tol, inner_sweeps, inner_tol=0.0, check_every=50,
                             max_outer=50, nx=None, ny=None, nz=None, stream=None):
    """Returns (status, info dict)."""
    nx, ny, nz = _extents(u, radius, nx, ny, nz)
    cp, _keep = _coeffs(coeffs)
    info = SolveInfo()
    rc = _check(_lib.jacobi_solve_refined_f64(_addr(rhs, 8, _n3(nx, ny, nz, radius)), _addr(u, 8, _n3(nx, ny, nz, radius)), nx, ny, nz, cp, radius, tol, inner_sweeps,
                                              inner_tol, check_every, max_outer, ctypes.byref(info),
                                              _stream(stream, u, rhs)))
    return rc, info.as_dict()


def _problems(us, rhss, radius):
    n = len(us)
    arr = (Problem * max(n, 1))()
    for i, (u, b) in enumerate(zip(us, rhss)):
        nx, ny, nz = _extents(u, radius, None, None, None)
        arr[i].nx, arr[i].ny, arr[i].nz = nx, ny, nz
        arr[i].rhs = _addr(b, 8, _n3(nx, ny, nz, radius))
        arr[i].u = _addr(u, 8, _n3(nx, ny, nz, radius))
    return arr, n


def jacobi_solve_batched_f64(us, rhss, coeffs, radius, tol, max_iters, check_every=50, stream=None):
    """Solves every (u, rhs) pair in one persistent launch; returns (status, [info dicts])."""
    arr, n = _problems(us, rhss, radius)
    cp, _keep = _coeffs(coeffs)
    infos = (SolveInfo * max(n, 1))()
    rc = _check(_lib.jacobi_solve_batched_f64(arr, n, cp, radius, tol, max_iters, check_every, infos,
                                              _stream(stream, *us)))
    return rc, [infos[i].as_dict() for i in range(n)]


def jacobi_solve_batched_refined(us, rhss, coeffs, radius, tol, inner_sweeps, inner_tol=0.0, check_every=50,
                                 max_outer=50, stream=None):
    arr, n = _problems(us, rhss, radius)
    cp, _keep = _coeffs(coeffs)
    infos = (SolveInfo * max(n, 1))()
    rc = _check(_lib.jacobi_solve_batched_refined(arr, n, cp, radius, tol, inner_sweeps, inner_tol,
                                                  check_every, max_outer, infos, _stream(stream, *us)))
    return rc, [infos[i].as_dict() for i in range(n)]


def varcoef_apply_f64(u, a, out, w, radius, nx=None, ny=None, nz=None, stream=None):
    nx, ny, nz = _extents(u, radius, nx, ny, nz)
    wp, _keep = _coeffs(w)
    return _check(_lib.varcoef_apply_f64(_addr(u, 8, _n3(nx, ny, nz, radius)), _addr(a, 8, _n3(nx, ny, nz, radius)), _addr(out, 8, _n3(nx, ny, nz, radius)), nx, ny, nz, wp, radius,
                                         _stream(stream, u, a, out)))


def varcoef_sweep_f64(in_, out, a, f, w, radius, iters, nx=None, ny=None, nz=None, stream=None):
    nx, ny, nz = _extents(in_, radius, nx, ny, nz)
    wp, _keep = _coeffs(w)
    return _check(_lib.varcoef_sweep_f64(_addr(in_, 8, _n3(nx, ny, nz, radius)), _addr(out, 8, _n3(nx, ny, nz, radius)), _addr(a, 8, _n3(nx, ny, nz, radius)), _addr(f, 8, _n3(nx, ny, nz, radius)), nx, ny, nz, wp, radius,
                                         iters, _stream(stream, in_, out, a, f)))


def varcoef_sweep_f32(in_, out, a, f, w, radius, iters, nx=None, ny=None, nz=None, stream=None):
    nx, ny, nz = _extents(in_, radius, nx, ny, nz)
    wp, _keep = _coeffs(w)
    return _check(_lib.varcoef_sweep_f32(_addr(in_, 4, _n3(nx, ny, nz, radius)), _addr(out, 4, _n3(nx, ny, nz, radius)), _addr(a, 4, _n3(nx, ny, nz, radius)), _addr(f, 4, _n3(nx, ny, nz, radius)), nx, ny, nz, wp, radius,
                                         iters, _stream(stream, in_, out, a, f)))


def varcoef_residual_norm_f64(u, a, f, w, radius, nx=None, ny=None, nz=None, stream=None) -> float:
    nx, ny, nz = _extents(u, radius, nx, ny, nz)
    wp, _keep = _coeffs(w)
    out = ctypes.c_double(0.0)
    _check(_lib.varcoef_residual_norm_f64(_addr(u, 8, _n3(nx, ny, nz, radius)), _addr(a, 8, _n3(nx, ny, nz, radius)), _addr(f, 8, _n3(nx, ny, nz, radius)), nx, ny, nz, wp, radius,
                                          ctypes.byref(out), _stream(stream, u, a, f)))
    return out.value


def jacobi_solve_varcoef_f64(a, f, u, w, radius, tol, max_iters, check_every=50, nx=None, ny=None, nz=None,
                             stream=None):
    nx, ny, nz = _extents(u, radius, nx, ny, nz)
    wp, _keep = _coeffs(w)
    info = SolveInfo()
    rc = _check(_lib.jacobi_solve_varcoef_f64(_addr(a, 8, _n3(nx, ny, nz, radius)), _addr(f, 8, _n3(nx, ny, nz, radius)), _addr(u, 8, _n3(nx, ny, nz, radius)), nx, ny, nz, wp, radius, tol,
                                              max_iters, check_every, ctypes.byref(info),
                                              _stream(stream, u, a, f)))
    return rc, info.as_dict()


def jacobi_solve_varcoef_refined(a, f, u, w, radius, tol, inner_sweeps, max_outer, nx=None, ny=None,
                                 nz=None, stream=None):
    nx, ny, nz = _extents(u, radius, nx, ny, nz)
    wp, _keep = _coeffs(w)
    info = SolveInfo()
    rc = _check(_lib.jacobi_solve_varcoef_refined(_addr(a, 8, _n3(nx, ny, nz, radius)), _addr(f, 8, _n3(nx, ny, nz, radius)), _addr(u, 8, _n3(nx, ny, nz, radius)), nx, ny, nz, wp, radius, tol,
                                                  inner_sweeps, max_outer, ctypes.byref(info),
                                                  _stream(stream, u, a, f)))
    return rc, info.as_dict()


def stencil_tune_set(knob: str, value: int):
    return _check(_lib.stencil_tune_set(knob.encode(), value))


def stencil_tune_get(knob: str) -> int:
    v = _i64(0)
    _check(_lib.stencil_tune_get(knob.encode(), ctypes.byref(v)))
    return v.value


def stencil_autotune_sweep(nx, ny, nz, esize, radius, coeffs=None, trial_sweeps=0, stream=None) -> dict:
    """Times the sweep configurations for these extents on the device, stores
    the fastest in the tuning cache and returns it (TuneEntry fields)."""
    e = TuneEntry()
    cp, _keep = _coeffs(coeffs) if coeffs is not None else (None, None)
    _check(_lib.stencil_autotune_sweep(nx, ny, nz, esize, radius, cp, trial_sweeps, ctypes.byref(e),
                                       _stream(stream)))
    return e.as_dict()


def stencil_tune_cache_put(nx, ny, nz, esize, radius, variant, chunks, depth=1, device="", glups=0.0,
                           default_glups=0.0):
    e = TuneEntry(device.encode(), nx, ny, nz, esize, radius, variant, chunks, depth, 0, glups, default_glups)
    return _check(_lib.stencil_tune_cache_put(ctypes.byref(e)))


def stencil_tune_cache_get(nx, ny, nz, esize, radius, device=None):
    """The cache entry for these extents (dict), or None."""
    e = TuneEntry()
    found = _check(_lib.stencil_tune_cache_get(device.encode() if device else None, nx, ny, nz, esize, radius,
                                               ctypes.byref(e)))
    return e.as_dict() if found else None


def stencil_tune_cache_size() -> int:
    return _lib.stencil_tune_cache_size()


def stencil_tune_cache_clear():
    return _check(_lib.stencil_tune_cache_clear())


def stencil_tune_cache_save(path: str):
    return _check(_lib.stencil_tune_cache_save(os.fsencode(path)))


def stencil_tune_cache_load(path: str) -> int:
    return _check(_lib.stencil_tune_cache_load(os.fsencode(path)))


def stencil_plan_query(op: str, nx: int, ny: int, nz: int, esize: int, radius: int) -> dict:
    """The launch one sweep of these extents would make (host-side planning;
    nothing launched): variant, grid, block, tile, k chunk and ring sizes."""
    q = LaunchPlan()
    _check(_lib.stencil_plan_query(op.encode(), nx, ny, nz, esize, radius, ctypes.byref(q)))
    return q.as_dict()


class Server:
    """The serving loop of the C ABI (stn_server_*): submit host right-hand
    sides, get tickets, wait for solutions."""

    def __init__(self, hbm_budget, coeffs=(0.0, 1.0 / 6.0), radius=1, tol=1e-8, refined=True, max_iters=10 ** 7,
                 inner_sweeps=200000, inner_tol=1e-2, check_every=50, max_outer=40, max_inflight=64,
                 queue_capacity=4096, engine=0):
        o = ServerOpts()
        o.hbm_budget = int(hbm_budget)
        o.radius = radius
        for i in range(3):
            o.coeffs[i] = float(coeffs[i]) if i < len(coeffs) else 0.0
        o.tol, o.refined, o.max_iters = tol, int(refined), max_iters
        o.inner_sweeps, o.inner_tol, o.check_every, o.max_outer = inner_sweeps, inner_tol, check_every, max_outer
        o.max_inflight, o.queue_capacity, o.engine = max_inflight, queue_capacity, engine
        h = _lib.stn_server_create(ctypes.byref(o))
        if not h:
            raise StencilError(STN_EINVAL, last_error())
        self._h = h
        self.radius = radius

    def submit(self, rhs: np.ndarray, u0: np.ndarray | None = None) -> int:
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        if rhs.ndim != 3:
            raise ValueError("rhs must be a 3D grid")
        nz, ny, nx = (s - 2 * self.radius for s in rhs.shape)
        # converted copies stay referenced until the call has copied them
        u0c = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64)
        if u0c is not None and u0c.shape != rhs.shape:
            raise ValueError(f"u0 of shape {u0c.shape}, rhs of shape {rhs.shape}")
        req = Request(nx, ny, nz, rhs.ctypes.data, None if u0c is None else u0c.ctypes.data)
        t = ctypes.c_uint64(0)
        _check(_lib.stn_submit(self._h, ctypes.byref(req), ctypes.byref(t)))
        return t.value

    def poll(self, ticket):
        r = Result()
        rc = _check(_lib.stn_poll(self._h, ticket, ctypes.byref(r)))
        return None if rc == STN_PENDING else r.as_dict()

    def wait(self, ticket, timeout_s=-1.0):
        r = Result()
        _check(_lib.stn_wait(self._h, ticket, timeout_s, ctypes.byref(r)))
        return r.as_dict()

    def result(self, ticket, shape):
        out = np.empty(shape, dtype=np.float64)
        _check(_lib.stn_result_copy(self._h, ticket, out.ctypes.data))
        return out

    def release(self, ticket):
        return _check(_lib.stn_release(self._h, ticket))

    def stats(self):
        st = ServerStats()
        _check(_lib.stn_server_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in st._fields_}

    def close(self):
        if self._h:
            _lib.stn_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


SCHED_STATS = ("cyc_claim", "cyc_unit", "cyc_done", "cyc_epilogue", "cyc_idle", "units", "epilogues", "misses",
               "fast_claims", "claim_tries")


def stencil_sched_stats() -> dict:
    buf = (ctypes.c_uint64 * len(SCHED_STATS))()
    n = _check(_lib.stencil_sched_stats(buf, len(SCHED_STATS)))
    return {k: int(buf[i]) for i, k in enumerate(SCHED_STATS[:n])}


def release_workspace():
    return _check(_lib.stencil_release_workspace())
