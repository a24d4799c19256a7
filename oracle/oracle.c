/*
 * CPU oracle for the 3D Jacobi stencil path: TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * legs load this library.  The product path (paper_2409_18824_gb300) never
 * links, imports or calls anything in oracle/, and this file includes nothing
 * from the product.  Everything here is written to be read against the paper,
 * not to be fast: plain triple loops (k outer, then j, then i), double
 * precision, no fused multiply-add (built with -ffp-contract=off).
 *
 * What the method is (arXiv 2409.18824):
 *   - Sec. 4 describes the "jacobi" benchmark: a Jacobi iteration solving
 *     Laplace's equation on a structured grid (2D 1024x1024 in the paper; the
 *     3D grid used here is the same iteration with one more axis).
 *   - Sec. 2.2 places such loops in the stencil dialect: each interior point is
 *     a weighted sum of its neighbours (stencil.apply / stencil.access).
 *   - Sec. 5.2 and Listing 7: Fortran arrays are 1-based; element (i,j,k)
 *     lives at 0-based offset (i-1) + (j-1)*NX + (k-1)*NX*NY, column-major.
 *   - Sec. 5.3 and Listing 8: a sum reduction starts from 0 and adds every
 *     element (linalg.reduce with an add combiner); the residual norm below is
 *     that reduction over the squared residual.
 *
 * Readings where the paper is silent (the same readings the GPU path follows):
 *   - Grid: interior nx*ny*nz points, a Dirichlet halo of `r` layers on every
 *     face (padded extents NX=nx+2r, NY=ny+2r, NZ=nz+2r); the halo is read,
 *     never written.
 *   - Constant-coefficient star stencil of radius r in {1,2} with weights
 *     c[0..r]: out = c0*u + sum_d c_d * S_d + b, S_d the sum of the six
 *     neighbours at distance d.  Canonical evaluation order (so that a GPU
 *     kernel that follows it is bitwise equal):
 *         S_d = ((u[i-d]+u[i+d]) + (u[j-d]+u[j+d])) + (u[k-d]+u[k+d])
 *         acc = c_r*S_r; then acc = acc + c_d*S_d for d = r-1 .. 1;
 *         acc = acc + c0*u   only if c0 != 0;  acc = acc + b   only if b given.
 *   - Residual of an iterate u: rho = (S u + b) - u per interior point, the
 *     norm sqrt(sum rho^2) accumulated in double in k-j-i order.  For float
 *     grids the stencil value is computed in float and the difference and the
 *     square in double.
 *   - Variable-coefficient operator (radius 2, per-point a on the padded grid):
 *         (A u)(p) = sum_{d=1..R} w_d sum_{q = p +- d e_x, e_y, e_z}
 *                    kappa(p,q) (u(p) - u(q)),    kappa = (a(p)+a(q))/2,
 *     Jacobi update u'(p) = (f(p) + N(p)) / D(p) with D = sum w_d kappa and
 *     N = sum w_d kappa u(q), both accumulated d = 1..R, axis x,y,z, the
 *     minus neighbour before the plus neighbour.  (A u)(p) = D u(p) - N.
 *   - Multi-field advection (a synthetic stand-in for the paper's pw-advection
 *     and tra-adv workloads, Sec. 4: fields carried by a wind; their formulas
 *     are not in the paper): second-order centred flux-form advection of a
 *     field q by the velocity (u, v, w), per axis a with velocity V_a,
 *         F-(p) = (V(p-e)+V(p)) * (q(p-e)+q(p)),
 *         F+(p) = (V(p)+V(p+e)) * (q(p)+q(p+e)),
 *         T_a = c_a * (F- - F+),   s = (T_x + T_y) + T_z,
 *     every operation rounded separately in this order.
 *   - Two-dimensional grids (the paper's own jacobi benchmark is 2-D, Sec. 4):
 *     a padded (ny+2r) x (nx+2r) array, i fastest, the same Dirichlet halo
 *     and the same canonical order without the k term:
 *         S_d = (u[i-d]+u[i+d]) + (u[j-d]+u[j+d]).
 *
 * Functions without an independent pin are marked "parity unpinned" in their
 * comment; every other function is pinned by tests/test_oracle.py (closed
 * forms, invariants, dense brute force, GEPP).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef int64_t i64;

/* 0-based offset of 0-based padded coordinates (i, j, k); Fortran column-major
 * (Sec. 5.2, Listing 7: subtract the lower bound 1, then linearise with the
 * first index fastest). */
static inline i64 off3(i64 i, i64 j, i64 k, i64 NX, i64 NY) { return i + NX * (j + NY * k); }

/* ---------------------------------------------------------------------------
 * One Jacobi sweep of the constant-coefficient star stencil, double.
 * Writes the interior of `out` only.  `b` may be NULL (no source term).
 * Sec. 4 (Jacobi for Laplace), Sec. 2.2 (stencil form).
 * ------------------------------------------------------------------------- */
void oracle_sweep_f64(const double* u, const double* b, double* out, i64 nx, i64 ny, i64 nz,
                      const double* c, int r) {
  const i64 NX = nx + 2 * r, NY = ny + 2 * r;
  for (i64 k = r; k < nz + r; k++)
    for (i64 j = r; j < ny + r; j++)
      for (i64 i = r; i < nx + r; i++) {
        const i64 p = off3(i, j, k, NX, NY);
        double acc = 0.0;
        for (int d = r; d >= 1; d--) {
          double sx = u[off3(i - d, j, k, NX, NY)] + u[off3(i + d, j, k, NX, NY)];
          double sy = u[off3(i, j - d, k, NX, NY)] + u[off3(i, j + d, k, NX, NY)];
          double sz = u[off3(i, j, k - d, NX, NY)] + u[off3(i, j, k + d, NX, NY)];
          double s = (sx + sy) + sz;
          double t = c[d] * s;
          acc = (d == r) ? t : acc + t;
        }
        if (c[0] != 0.0) acc = acc + c[0] * u[p];
        if (b) acc = acc + b[p];
        out[p] = acc;
      }
}

/* Same sweep in float arithmetic: coefficients are the float roundings of the
 * double coefficients (the caller passes them already rounded). */
void oracle_sweep_f32(const float* u, const float* b, float* out, i64 nx, i64 ny, i64 nz,
                      const float* c, int r) {
  const i64 NX = nx + 2 * r, NY = ny + 2 * r;
  for (i64 k = r; k < nz + r; k++)
    for (i64 j = r; j < ny + r; j++)
      for (i64 i = r; i < nx + r; i++) {
        const i64 p = off3(i, j, k, NX, NY);
        float acc = 0.0f;
        for (int d = r; d >= 1; d--) {
          float sx = u[off3(i - d, j, k, NX, NY)] + u[off3(i + d, j, k, NX, NY)];
          float sy = u[off3(i, j - d, k, NX, NY)] + u[off3(i, j + d, k, NX, NY)];
          float sz = u[off3(i, j, k - d, NX, NY)] + u[off3(i, j, k + d, NX, NY)];
          float s = (sx + sy) + sz;
          float t = c[d] * s;
          acc = (d == r) ? t : acc + t;
        }
        if (c[0] != 0.0f) acc = acc + c[0] * u[p];
        if (b) acc = acc + b[p];
        out[p] = acc;
      }
}

/* `iters` sweeps from `in`; the result lands in `out` (halo of `out` = halo of
 * `in`).  `in` is left unchanged here; the library may clobber it.
 * Sec. 4: the benchmark repeats the sweep a fixed number of iterations. */
int oracle_stencil_sweep_f64(const double* in, double* out, i64 nx, i64 ny, i64 nz, const double* c,
                             int r, i64 iters) {
  const i64 n = (nx + 2 * r) * (ny + 2 * r) * (nz + 2 * r);
  double* tmp = (double*)malloc(sizeof(double) * (size_t)n);
  if (!tmp) return -2;
  memcpy(out, in, sizeof(double) * (size_t)n);
  memcpy(tmp, in, sizeof(double) * (size_t)n);
  for (i64 it = 0; it < iters; it++) {
    /* src holds the current iterate, dst receives the next; swap by copying
     * back so the iterate always lives in `out` between sweeps. */
    oracle_sweep_f64(out, NULL, tmp, nx, ny, nz, c, r);
    memcpy(out, tmp, sizeof(double) * (size_t)n);
  }
  free(tmp);
  return 0;
}

int oracle_stencil_sweep_f32(const float* in, float* out, i64 nx, i64 ny, i64 nz, const float* c,
                             int r, i64 iters) {
  const i64 n = (nx + 2 * r) * (ny + 2 * r) * (nz + 2 * r);
  float* tmp = (float*)malloc(sizeof(float) * (size_t)n);
  if (!tmp) return -2;
  memcpy(out, in, sizeof(float) * (size_t)n);
  memcpy(tmp, in, sizeof(float) * (size_t)n);
  for (i64 it = 0; it < iters; it++) {
    oracle_sweep_f32(out, NULL, tmp, nx, ny, nz, c, r);
    memcpy(out, tmp, sizeof(float) * (size_t)n);
  }
  free(tmp);
  return 0;
}

/* ---------------------------------------------------------------------------
 * Residual norm sqrt(sum over interior of ((S u + b) - u)^2).
 * Sec. 5.3 / Listing 8: sum reduction initialised to zero, add-combined.
 * ------------------------------------------------------------------------- */
double oracle_residual_norm_f64(const double* u, const double* b, i64 nx, i64 ny, i64 nz,
                                const double* c, int r) {
  const i64 NX = nx + 2 * r, NY = ny + 2 * r, NZ = nz + 2 * r;
  double* s = (double*)malloc(sizeof(double) * (size_t)(NX * NY * NZ));
  if (!s) return NAN;
  oracle_sweep_f64(u, b, s, nx, ny, nz, c, r);
  double sum = 0.0;
  for (i64 k = r; k < nz + r; k++)
    for (i64 j = r; j < ny + r; j++)
      for (i64 i = r; i < nx + r; i++) {
        const i64 p = off3(i, j, k, NX, NY);
        double rho = s[p] - u[p];
        sum = sum + rho * rho;
      }
  free(s);
  return sqrt(sum);
}

double oracle_residual_norm_f32(const float* u, const float* b, i64 nx, i64 ny, i64 nz,
                                const float* c, int r) {
  const i64 NX = nx + 2 * r, NY = ny + 2 * r, NZ = nz + 2 * r;
  float* s = (float*)malloc(sizeof(float) * (size_t)(NX * NY * NZ));
  if (!s) return NAN;
  oracle_sweep_f32(u, b, s, nx, ny, nz, c, r);
  double sum = 0.0;
  for (i64 k = r; k < nz + r; k++)
    for (i64 j = r; j < ny + r; j++)
      for (i64 i = r; i < nx + r; i++) {
        const i64 p = off3(i, j, k, NX, NY);
        double rho = (double)s[p] - (double)u[p];
        sum = sum + rho * rho;
      }
  free(s);
  return sqrt(sum);
}

/* Plain L2 norm of the interior of a padded grid (the same add-reduction). */
double oracle_interior_norm_f64(const double* x, i64 nx, i64 ny, i64 nz, int r) {
  const i64 NX = nx + 2 * r, NY = ny + 2 * r;
  double sum = 0.0;
  for (i64 k = r; k < nz + r; k++)
    for (i64 j = r; j < ny + r; j++)
      for (i64 i = r; i < nx + r; i++) {
        double v = x[off3(i, j, k, NX, NY)];
        sum = sum + v * v;
      }
  return sqrt(sum);
}

/* ---------------------------------------------------------------------------
 * Jacobi solve of u = S u + b to a relative residual tolerance (Sec. 4).
 * Sweeps run in groups of `check_every`; the last sweep of a group also
 * measures the residual of the iterate it starts from.  The solve stops after
 * the first group whose measured residual satisfies ||rho|| <= tol*||b||
 * (absolute ||rho|| <= tol when ||b|| = 0), or when max_iters sweeps are done.
 * On return u holds the last iterate (one sweep past the measured one),
 * *iters_out the sweeps done, *rel_res_out the measured relative residual.
 * Returns 0 if converged, 1 if not.
 * ------------------------------------------------------------------------- */
int oracle_jacobi_solve_f64(const double* b, double* u, i64 nx, i64 ny, i64 nz, const double* c,
                            int r, double tol, i64 max_iters, i64 check_every, i64* iters_out,
                            double* rel_res_out) {
  const i64 n = (nx + 2 * r) * (ny + 2 * r) * (nz + 2 * r);
  double* nxt = (double*)malloc(sizeof(double) * (size_t)n);
  if (!nxt) return -2;
  memcpy(nxt, u, sizeof(double) * (size_t)n);
  const double bnorm = b ? oracle_interior_norm_f64(b, nx, ny, nz, r) : 0.0;
  const double scale = bnorm > 0.0 ? bnorm : 1.0;
  i64 it = 0;
  double rel = INFINITY;
  int status = 1;
  if (check_every < 1) check_every = 1;
  while (it < max_iters) {
    i64 group = check_every;
    if (group > max_iters - it) group = max_iters - it;
    for (i64 g = 0; g < group; g++) {
      if (g == group - 1) rel = oracle_residual_norm_f64(u, b, nx, ny, nz, c, r) / scale;
      oracle_sweep_f64(u, b, nxt, nx, ny, nz, c, r);
      memcpy(u, nxt, sizeof(double) * (size_t)n);
      it++;
    }
    if (rel <= tol) { status = 0; break; }
  }
  free(nxt);
  *iters_out = it;
  *rel_res_out = rel;
  return status;
}

/* ---------------------------------------------------------------------------
 * Variable-coefficient operator (radius R, weights w[1..R], per-point a on the
 * padded grid).  Reading: symmetric face coefficients kappa = (a(p)+a(q))/2;
 * this makes A an M-matrix so Jacobi converges (the paper gives no operator
 * beyond Laplace's, Sec. 4).
 * ------------------------------------------------------------------------- */
static void varcoef_dn_f64(const double* u, const double* a, i64 p, i64 sx, i64 sy, i64 sz,
                           const double* w, int R, double* D, double* N) {
  const i64 step[3] = {sx, sy, sz};
  double dsum = 0.0, nsum = 0.0;
  for (int d = 1; d <= R; d++)
    for (int ax = 0; ax < 3; ax++)
      for (int sg = -1; sg <= 1; sg += 2) {
        const i64 q = p + sg * d * step[ax];
        double kap = 0.5 * (a[p] + a[q]);
        double t = w[d] * kap;
        dsum = dsum + t;
        nsum = nsum + t * u[q];
      }
  *D = dsum;
  *N = nsum;
}

/* out = A u on the interior. */
void oracle_varcoef_apply_f64(const double* u, const double* a, double* out, i64 nx, i64 ny,
                              i64 nz, const double* w, int R) {
  const i64 NX = nx + 2 * R, NY = ny + 2 * R;
  for (i64 k = R; k < nz + R; k++)
    for (i64 j = R; j < ny + R; j++)
      for (i64 i = R; i < nx + R; i++) {
        const i64 p = off3(i, j, k, NX, NY);
        double D, N;
        varcoef_dn_f64(u, a, p, 1, NX, NX * NY, w, R, &D, &N);
        out[p] = D * u[p] - N;
      }
}

/* One Jacobi sweep for A u = f: out = (f + N) / D. */
void oracle_varcoef_sweep_f64(const double* u, const double* a, const double* f, double* out,
                              i64 nx, i64 ny, i64 nz, const double* w, int R) {
  const i64 NX = nx + 2 * R, NY = ny + 2 * R;
  for (i64 k = R; k < nz + R; k++)
    for (i64 j = R; j < ny + R; j++)
      for (i64 i = R; i < nx + R; i++) {
        const i64 p = off3(i, j, k, NX, NY);
        double D, N;
        varcoef_dn_f64(u, a, p, 1, NX, NX * NY, w, R, &D, &N);
        out[p] = (f[p] + N) / D;
      }
}

/* Float version of the sweep: a, f, u and the weights all float. */
void oracle_varcoef_sweep_f32(const float* u, const float* a, const float* f, float* out, i64 nx,
                              i64 ny, i64 nz, const float* w, int R) {
  const i64 NX = nx + 2 * R, NY = ny + 2 * R;
  const i64 step[3] = {1, NX, NX * NY};
  for (i64 k = R; k < nz + R; k++)
    for (i64 j = R; j < ny + R; j++)
      for (i64 i = R; i < nx + R; i++) {
        const i64 p = off3(i, j, k, NX, NY);
        float dsum = 0.0f, nsum = 0.0f;
        for (int d = 1; d <= R; d++)
          for (int ax = 0; ax < 3; ax++)
            for (int sg = -1; sg <= 1; sg += 2) {
              const i64 q = p + sg * d * step[ax];
              float kap = 0.5f * (a[p] + a[q]);
              float t = w[d] * kap;
              dsum = dsum + t;
              nsum = nsum + t * u[q];
            }
        out[p] = (f[p] + nsum) / dsum;
      }
}

/* ||f - A u||_2 over the interior, double. */
double oracle_varcoef_residual_norm_f64(const double* u, const double* a, const double* f, i64 nx,
                                        i64 ny, i64 nz, const double* w, int R) {
  const i64 NX = nx + 2 * R, NY = ny + 2 * R;
  double sum = 0.0;
  for (i64 k = R; k < nz + R; k++)
    for (i64 j = R; j < ny + R; j++)
      for (i64 i = R; i < nx + R; i++) {
        const i64 p = off3(i, j, k, NX, NY);
        double D, N;
        varcoef_dn_f64(u, a, p, 1, NX, NX * NY, w, R, &D, &N);
        double rho = f[p] - (D * u[p] - N);
        sum = sum + rho * rho;
      }
  return sqrt(sum);
}

/* Plain double Jacobi solve of A u = f (same group/check convention as the
 * constant-coefficient solve above). */
int oracle_varcoef_jacobi_solve_f64(const double* a, const double* f, double* u, i64 nx, i64 ny,
                                    i64 nz, const double* w, int R, double tol, i64 max_iters,
                                    i64 check_every, i64* iters_out, double* rel_res_out) {
  const i64 n = (nx + 2 * R) * (ny + 2 * R) * (nz + 2 * R);
  double* nxt = (double*)malloc(sizeof(double) * (size_t)n);
  if (!nxt) return -2;
  memcpy(nxt, u, sizeof(double) * (size_t)n);
  const double fnorm = oracle_interior_norm_f64(f, nx, ny, nz, R);
  const double scale = fnorm > 0.0 ? fnorm : 1.0;
  i64 it = 0;
  double rel = INFINITY;
  int status = 1;
  if (check_every < 1) check_every = 1;
  while (it < max_iters) {
    i64 group = check_every;
    if (group > max_iters - it) group = max_iters - it;
    for (i64 g = 0; g < group; g++) {
      if (g == group - 1) rel = oracle_varcoef_residual_norm_f64(u, a, f, nx, ny, nz, w, R) / scale;
      oracle_varcoef_sweep_f64(u, a, f, nxt, nx, ny, nz, w, R);
      memcpy(u, nxt, sizeof(double) * (size_t)n);
      it++;
    }
    if (rel <= tol) { status = 0; break; }
  }
  free(nxt);
  *iters_out = it;
  *rel_res_out = rel;
  return status;
}

/* ---------------------------------------------------------------------------
 * Mixed-precision iterative refinement for A u = f (variable coefficient).
 * Not in the paper; steps in order:
 *   outer (double): rho = f - A u; stop if ||rho||/||f|| <= tol;
 *                   s = max|rho|; r32 = float(rho / s)
 *   inner (float) : Jacobi on A e = r32 from e = 0 (a and w rounded to
 *                   float) for `inner_sweeps` sweeps
 *   update(double): u = u + s * double(e)
 * Returns 0 if converged within max_outer steps, 1 if not.  Reports the outer
 * steps taken and the final double relative residual.
 * Pinned by its end state (residual recomputed from the dense operator,
 * solution against a direct solve), by one outer step bitwise on coefficient
 * fields whose Jacobi diagonals are powers of two (float exact there), and by
 * the closed form rho -> (N D^-1)^m rho per outer step (A = D - N).
 * ------------------------------------------------------------------------- */
int oracle_varcoef_refined_solve(const double* a, const double* f, double* u, i64 nx, i64 ny,
                                 i64 nz, const double* w, int R, double tol, i64 inner_sweeps,
                                 i64 max_outer, i64* outer_out, double* rel_res_out) {
  const i64 NX = nx + 2 * R, NY = ny + 2 * R, NZ = nz + 2 * R;
  const i64 n = NX * NY * NZ;
  double* rho = (double*)calloc((size_t)n, sizeof(double));
  float* a32 = (float*)malloc(sizeof(float) * (size_t)n);
  float* r32 = (float*)calloc((size_t)n, sizeof(float));
  float* e = (float*)calloc((size_t)n, sizeof(float));
  float* e2 = (float*)calloc((size_t)n, sizeof(float));
  if (!rho || !a32 || !r32 || !e || !e2) {
    free(rho); free(a32); free(r32); free(e); free(e2);
    return -2;
  }
  float w32[3] = {0.0f, 0.0f, 0.0f};
  for (int d = 1; d <= R; d++) w32[d] = (float)w[d];
  for (i64 p = 0; p < n; p++) a32[p] = (float)a[p];
  const double fnorm = oracle_interior_norm_f64(f, nx, ny, nz, R);
  const double scale = fnorm > 0.0 ? fnorm : 1.0;
  double rel = INFINITY;
  i64 outer = 0;
  int status = 1;
  for (;;) {
    oracle_varcoef_apply_f64(u, a, rho, nx, ny, nz, w, R);
    double ss = 0.0, amax = 0.0;
    for (i64 k = R; k < nz + R; k++)
      for (i64 j = R; j < ny + R; j++)
        for (i64 i = R; i < nx + R; i++) {
          const i64 p = off3(i, j, k, NX, NY);
          double v = f[p] - rho[p];
          rho[p] = v;
          ss = ss + v * v;
          if (fabs(v) > amax) amax = fabs(v);
        }
    rel = sqrt(ss) / scale;
    if (rel <= tol) { status = 0; break; }
    if (outer >= max_outer || amax == 0.0) break;
    for (i64 k = R; k < nz + R; k++)
      for (i64 j = R; j < ny + R; j++)
        for (i64 i = R; i < nx + R; i++) {
          const i64 p = off3(i, j, k, NX, NY);
          r32[p] = (float)(rho[p] / amax);
        }
    memset(e, 0, sizeof(float) * (size_t)n);
    memset(e2, 0, sizeof(float) * (size_t)n);
    for (i64 s = 0; s < inner_sweeps; s++) {
      oracle_varcoef_sweep_f32(e, a32, r32, e2, nx, ny, nz, w32, R);
      float* t = e; e = e2; e2 = t;
    }
    for (i64 k = R; k < nz + R; k++)
      for (i64 j = R; j < ny + R; j++)
        for (i64 i = R; i < nx + R; i++) {
          const i64 p = off3(i, j, k, NX, NY);
          u[p] = u[p] + amax * (double)e[p];
        }
    outer++;
  }
  free(rho); free(a32); free(r32); free(e); free(e2);
  *outer_out = outer;
  *rel_res_out = rel;
  return status;
}

/* ---------------------------------------------------------------------------
 * Mixed-precision iterative refinement for u = S u + b (constant
 * coefficients).  Not in the paper; steps in order:
 *   outer (double): t = S u + b; rho = t - u; stop if ||rho|| <= tol*||b||
 *                   (absolute when b = 0); s = max|rho|; r32 = float(rho / s)
 *   inner (float) : `inner_sweeps` sweeps of e = S e + r32 from e = 0, with
 *                   the coefficients rounded to float
 *   update(double): u = u + s * double(e)
 * Returns 0 if converged within max_outer steps, 1 if not.
 * ------------------------------------------------------------------------- */
int oracle_refined_solve_f64(const double* b, double* u, i64 nx, i64 ny, i64 nz, const double* c,
                             int r, double tol, i64 inner_sweeps, i64 max_outer, i64* outer_out,
                             double* rel_res_out) {
  const i64 NX = nx + 2 * r, NY = ny + 2 * r, NZ = nz + 2 * r;
  const i64 n = NX * NY * NZ;
  double* t = (double*)calloc((size_t)n, sizeof(double));
  float* r32 = (float*)calloc((size_t)n, sizeof(float));
  float* e = (float*)calloc((size_t)n, sizeof(float));
  float* e2 = (float*)calloc((size_t)n, sizeof(float));
  if (!t || !r32 || !e || !e2) {
    free(t); free(r32); free(e); free(e2);
    return -2;
  }
  float c32[3] = {0.0f, 0.0f, 0.0f};
  for (int d = 0; d <= r; d++) c32[d] = (float)c[d];
  const double bnorm = b ? oracle_interior_norm_f64(b, nx, ny, nz, r) : 0.0;
  const double scale = bnorm > 0.0 ? bnorm : 1.0;
  double rel = INFINITY;
  i64 outer = 0;
  int status = 1;
  for (;;) {
    oracle_sweep_f64(u, b, t, nx, ny, nz, c, r);
    double ss = 0.0, amax = 0.0;
    for (i64 k = r; k < nz + r; k++)
      for (i64 j = r; j < ny + r; j++)
        for (i64 i = r; i < nx + r; i++) {
          const i64 p = off3(i, j, k, NX, NY);
          double rho = t[p] - u[p];
          ss = ss + rho * rho;
          if (fabs(rho) > amax) amax = fabs(rho);
        }
    rel = sqrt(ss) / scale;
    if (rel <= tol) { status = 0; break; }
    if (outer >= max_outer || amax == 0.0) break;
    for (i64 k = r; k < nz + r; k++)
      for (i64 j = r; j < ny + r; j++)
        for (i64 i = r; i < nx + r; i++) {
          const i64 p = off3(i, j, k, NX, NY);
          r32[p] = (float)((t[p] - u[p]) / amax);
          e[p] = 0.0f;
        }
    float* cur = e;
    float* nxt = e2;
    for (i64 s = 0; s < inner_sweeps; s++) {
      oracle_sweep_f32(cur, r32, nxt, nx, ny, nz, c32, r);
      float* tmp = cur; cur = nxt; nxt = tmp;
    }
    for (i64 k = r; k < nz + r; k++)
      for (i64 j = r; j < ny + r; j++)
        for (i64 i = r; i < nx + r; i++) {
          const i64 p = off3(i, j, k, NX, NY);
          u[p] = u[p] + amax * (double)cur[p];
        }
    outer++;
  }
  free(t); free(r32); free(e); free(e2);
  *outer_out = outer;
  *rel_res_out = rel;
  return status;
}

/* ---------------------------------------------------------------------------
 * Dense Gaussian elimination with partial pivoting (textbook), A is n x n
 * row-major and overwritten; b is overwritten with the solution.  Used to
 * solve tiny systems exactly as a pin for the iterative solves.
 * Returns 0, or -1 for a singular matrix.
 * ------------------------------------------------------------------------- */
int oracle_dense_solve(double* A, double* b, i64 n) {
  for (i64 col = 0; col < n; col++) {
    i64 piv = col;
    double best = fabs(A[col * n + col]);
    for (i64 row = col + 1; row < n; row++)
      if (fabs(A[row * n + col]) > best) { best = fabs(A[row * n + col]); piv = row; }
    if (best == 0.0) return -1;
    if (piv != col) {
      for (i64 j = 0; j < n; j++) {
        double t = A[col * n + j]; A[col * n + j] = A[piv * n + j]; A[piv * n + j] = t;
      }
      double t = b[col]; b[col] = b[piv]; b[piv] = t;
    }
    for (i64 row = col + 1; row < n; row++) {
      double m = A[row * n + col] / A[col * n + col];
      if (m == 0.0) continue;
      for (i64 j = col; j < n; j++) A[row * n + j] = A[row * n + j] - m * A[col * n + j];
      b[row] = b[row] - m * b[col];
    }
  }
  for (i64 row = n - 1; row >= 0; row--) {
    double s = b[row];
    for (i64 j = row + 1; j < n; j++) s = s - A[row * n + j] * b[j];
    b[row] = s / A[row * n + row];
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * Two-dimensional star stencil: the paper's jacobi benchmark (Sec. 4) is a
 * Jacobi iteration for Laplace's equation on one 2-D grid.  Padded grid of
 * (ny+2r) rows of NX = nx+2r values, i fastest (Sec. 5.2 indexing with two
 * indices).  S_d = (u[i-d]+u[i+d]) + (u[j-d]+u[j+d]); acc = c_r*S_r, then
 * acc + c_d*S_d for d = r-1..1; + c0*u if c0 != 0; + b if b given.
 * ------------------------------------------------------------------------- */
void oracle_sweep2d_f64(const double* u, const double* b, double* out, i64 nx, i64 ny,
                        const double* c, int r) {
  const i64 NX = nx + 2 * r;
  for (i64 j = r; j < ny + r; j++)
    for (i64 i = r; i < nx + r; i++) {
      const i64 p = i + NX * j;
      double acc = 0.0;
      for (int d = r; d >= 1; d--) {
        double sx = u[p - d] + u[p + d];
        double sy = u[p - d * NX] + u[p + d * NX];
        double t = c[d] * (sx + sy);
        acc = (d == r) ? t : acc + t;
      }
      if (c[0] != 0.0) acc = acc + c[0] * u[p];
      if (b) acc = acc + b[p];
      out[p] = acc;
    }
}

void oracle_sweep2d_f32(const float* u, const float* b, float* out, i64 nx, i64 ny,
                        const float* c, int r) {
  const i64 NX = nx + 2 * r;
  for (i64 j = r; j < ny + r; j++)
    for (i64 i = r; i < nx + r; i++) {
      const i64 p = i + NX * j;
      float acc = 0.0f;
      for (int d = r; d >= 1; d--) {
        float sx = u[p - d] + u[p + d];
        float sy = u[p - d * NX] + u[p + d * NX];
        float t = c[d] * (sx + sy);
        acc = (d == r) ? t : acc + t;
      }
      if (c[0] != 0.0f) acc = acc + c[0] * u[p];
      if (b) acc = acc + b[p];
      out[p] = acc;
    }
}

/* `iters` 2-D sweeps from `in` into `out` (halo of `out` = halo of `in`);
 * Sec. 4: a fixed number of Jacobi iterations. */
int oracle_stencil_sweep2d_f64(const double* in, double* out, i64 nx, i64 ny, const double* c,
                               int r, i64 iters) {
  const i64 n = (nx + 2 * r) * (ny + 2 * r);
  double* tmp = (double*)malloc(sizeof(double) * (size_t)n);
  if (!tmp) return -2;
  memcpy(out, in, sizeof(double) * (size_t)n);
  memcpy(tmp, in, sizeof(double) * (size_t)n);
  for (i64 it = 0; it < iters; it++) {
    oracle_sweep2d_f64(out, NULL, tmp, nx, ny, c, r);
    memcpy(out, tmp, sizeof(double) * (size_t)n);
  }
  free(tmp);
  return 0;
}

int oracle_stencil_sweep2d_f32(const float* in, float* out, i64 nx, i64 ny, const float* c, int r,
                               i64 iters) {
  const i64 n = (nx + 2 * r) * (ny + 2 * r);
  float* tmp = (float*)malloc(sizeof(float) * (size_t)n);
  if (!tmp) return -2;
  memcpy(out, in, sizeof(float) * (size_t)n);
  memcpy(tmp, in, sizeof(float) * (size_t)n);
  for (i64 it = 0; it < iters; it++) {
    oracle_sweep2d_f32(out, NULL, tmp, nx, ny, c, r);
    memcpy(out, tmp, sizeof(float) * (size_t)n);
  }
  free(tmp);
  return 0;
}

/* sqrt(sum over the interior of ((S u + b) - u)^2), accumulated in double in
 * j-i order (Sec. 5.3 / Listing 8 add-reduction). */
double oracle_residual_norm2d_f64(const double* u, const double* b, i64 nx, i64 ny,
                                  const double* c, int r) {
  const i64 NX = nx + 2 * r, n = NX * (ny + 2 * r);
  double* t = (double*)malloc(sizeof(double) * (size_t)n);
  if (!t) return -1.0;
  oracle_sweep2d_f64(u, b, t, nx, ny, c, r);
  double sum = 0.0;
  for (i64 j = r; j < ny + r; j++)
    for (i64 i = r; i < nx + r; i++) {
      const double rho = t[i + NX * j] - u[i + NX * j];
      sum = sum + rho * rho;
    }
  free(t);
  return sqrt(sum);
}

double oracle_residual_norm2d_f32(const float* u, const float* b, i64 nx, i64 ny, const float* c,
                                  int r) {
  const i64 NX = nx + 2 * r, n = NX * (ny + 2 * r);
  float* t = (float*)malloc(sizeof(float) * (size_t)n);
  if (!t) return -1.0;
  oracle_sweep2d_f32(u, b, t, nx, ny, c, r);
  double sum = 0.0;
  for (i64 j = r; j < ny + r; j++)
    for (i64 i = r; i < nx + r; i++) {
      const double rho = (double)t[i + NX * j] - (double)u[i + NX * j];
      sum = sum + rho * rho;
    }
  free(t);
  return sqrt(sum);
}

/* ---------------------------------------------------------------------------
 * Array intrinsics of Sec. 5.4 (Table 3): `sum` of a double array and
 * `dotproduct` of two double vectors, each the linalg.reduce of Sec. 5.3 /
 * Listing 8 -- an accumulator initialised to zero and an add combiner applied
 * to the elements in order (for the dot product, to the products).
 * ------------------------------------------------------------------------- */
double oracle_sum_f64(const double* x, i64 n) {
  double acc = 0.0;
  for (i64 i = 0; i < n; i++) acc = acc + x[i];
  return acc;
}

double oracle_dot_f64(const double* x, const double* y, i64 n) {
  double acc = 0.0;
  for (i64 i = 0; i < n; i++) acc = acc + x[i] * y[i];
  return acc;
}

/* ---------------------------------------------------------------------------
 * Multi-field advection stand-in (see the header): the tendency s of one
 * field q under the velocity (u, v, w) on the interior of a halo-1 grid.
 * Writes the interior of s only.
 * ------------------------------------------------------------------------- */
void oracle_advect_f64(const double* u, const double* v, const double* w, const double* q,
                       double* s, i64 nx, i64 ny, i64 nz, const double* c) {
  const i64 NX = nx + 2, NY = ny + 2;
  const double* vel[3] = {u, v, w};
  const i64 step[3] = {1, NX, NX * NY};
  for (i64 k = 1; k <= nz; k++)
    for (i64 j = 1; j <= ny; j++)
      for (i64 i = 1; i <= nx; i++) {
        const i64 p = off3(i, j, k, NX, NY);
        double t[3];
        for (int a = 0; a < 3; a++) {
          const double* V = vel[a];
          const i64 e = step[a];
          const double fm = (V[p - e] + V[p]) * (q[p - e] + q[p]);
          const double fp = (V[p] + V[p + e]) * (q[p] + q[p + e]);
          t[a] = c[a] * (fm - fp);
        }
        s[p] = (t[0] + t[1]) + t[2];
      }
}

void oracle_advect_f32(const float* u, const float* v, const float* w, const float* q, float* s,
                       i64 nx, i64 ny, i64 nz, const float* c) {
  const i64 NX = nx + 2, NY = ny + 2;
  const float* vel[3] = {u, v, w};
  const i64 step[3] = {1, NX, NX * NY};
  for (i64 k = 1; k <= nz; k++)
    for (i64 j = 1; j <= ny; j++)
      for (i64 i = 1; i <= nx; i++) {
        const i64 p = off3(i, j, k, NX, NY);
        float t[3];
        for (int a = 0; a < 3; a++) {
          const float* V = vel[a];
          const i64 e = step[a];
          const float fm = (V[p - e] + V[p]) * (q[p - e] + q[p]);
          const float fp = (V[p] + V[p + e]) * (q[p] + q[p + e]);
          t[a] = c[a] * (fm - fp);
        }
        s[p] = (t[0] + t[1]) + t[2];
      }
}
