/*
 * stencil_host.h -- C ABI of libstencil_host.so: the multi-core host path of
 * the Jacobi sweep and of the advection stand-in, the paper's threaded jacobi
 * and pw-advection (arXiv 2409.18824 Sec. 6.2 and Table 4: the benchmarks'
 * loops shared out over OpenMP threads).
 *
 * A library of its own: libstencil.so neither links nor calls it, so it is
 * never a fallback for the GPU path.  Grids are HOST arrays in the layout of
 * include/stencil.h: the Fortran array u(1:nx+2r, 1:ny+2r[, 1:nz+2r]), i.e.
 * C-contiguous (nz+2r, ny+2r, nx+2r) or (ny+2r, nx+2r), i fastest, a
 * Dirichlet halo of r layers that is read and never written.  coeffs is a
 * host array {c0, c1[, c2]}.
 *
 * Every point follows the canonical evaluation order of the GPU kernels
 * (S_d = ((u(i-d)+u(i+d)) + (u(j-d)+u(j+d))) [+ (u(k-d)+u(k+d))], acc = c_r S_r,
 * acc += c_d S_d for d = r-1..1, + c0 u when c0 != 0, + b when given), each
 * operation rounded separately, so sweeps are bitwise those of the GPU path
 * and of the CPU oracle, for any thread count.  Residual norms sum one
 * partial per grid row (left to right) and then the rows in order, so a norm
 * does not depend on the thread count either.
 *
 * nthreads: worker threads (the calling thread is one of them); 0 = the
 * hardware's thread count; at most 1024 and at most one per grid row.
 * Threads split the interior rows into contiguous ranges and meet at a
 * barrier after every sweep.
 *
 * Errors (return value): 0 success; -1 invalid argument (NULL pointer,
 * extent < 1, radius not 1 or 2, iters < 0, nthreads < 0, in and out
 * overlapping);
 * -2 allocation failed.  stencil_host_last_error() gives the message.
 */
#ifndef STENCIL_HOST_H
#define STENCIL_HOST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Message of the last failing call on this thread ("" if none). */
const char* stencil_host_last_error(void);

/* Hardware threads of this machine (what nthreads = 0 uses). */
int stencil_host_threads(void);

/* `iters` 3-D sweeps from `in`; the result is in `out`.  As stencil_sweep_f64:
 * `in` is the ping-pong buffer when iters > 1 (its interior is clobbered),
 * the halo of `in` is copied to `out`, iters == 0 copies `in` to `out`. */
int stencil_host_sweep_f64(double* in, double* out, int64_t nx, int64_t ny, int64_t nz, const double* coeffs,
                           int radius, int64_t iters, int nthreads);

/* ||(S u + b) - u||_2 over the interior of a 3-D grid (b may be NULL). */
int stencil_host_residual_norm_f64(const double* u, const double* b, int64_t nx, int64_t ny, int64_t nz,
                                   const double* coeffs, int radius, double* norm_out, int nthreads);

/* The 2-D forms: grids of (ny+2r) rows of nx+2r values. */
int stencil_host_sweep2d_f64(double* in, double* out, int64_t nx, int64_t ny, const double* coeffs, int radius,
                             int64_t iters, int nthreads);
int stencil_host_residual_norm2d_f64(const double* u, const double* b, int64_t nx, int64_t ny,
                                     const double* coeffs, int radius, double* norm_out, int nthreads);

/* The multi-field advection stand-in on the host cores (the paper's threaded
 * pw-advection, Table 4), the same operation and order as advect_f64 in
 * include/stencil.h: per axis a with velocity V,
 *     F- = (V(p-e)+V(p)) * (q(p-e)+q(p)),  F+ = (V(p)+V(p+e)) * (q(p)+q(p+e)),
 *     T_a = c_a * (F- - F+),               s(p) = (T_x + T_y) + T_z,
 * each operation rounded separately.  Halo-1 grids of (nz+2, ny+2, nx+2).
 * q NULL: u, v, w advect themselves and s[0..2] receive their tendencies;
 * otherwise nq (1..6) fields q[0..nq-1] and s[0..nq-1].  Only the interior of
 * each s is written; the outputs must not overlap the inputs or each other.
 * c: 3 finite doubles {c_x, c_y, c_z}.  Errors: -1 (NULL pointers, nq out of
 * range, non-finite c, bad extents, overlap), -2. */
int stencil_host_advect_f64(const double* u, const double* v, const double* w, const double* const* q, int nq,
                            double* const* s, int64_t nx, int64_t ny, int64_t nz, const double* c, int nthreads);

#ifdef __cplusplus
}
#endif

#endif /* STENCIL_HOST_H */
