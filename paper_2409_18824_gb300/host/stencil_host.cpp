// Multi-core host path of the Jacobi sweep (C ABI in include/stencil_host.h):
// the paper's threaded jacobi, whose loops it shares out over OpenMP threads
// (arXiv 2409.18824 Sec. 6.2, Table 4).  Here persistent std::threads split
// the interior rows into contiguous ranges and meet at a spinning barrier
// after every sweep; the calling thread is worker 0.  The update of a row is
// a plain loop over i in the canonical evaluation order (the compiler
// vectorises it; the library is built with -ffp-contract=off so that no
// multiply and add fuse), so every thread count gives the same bits.
#include "stencil_host.h"

#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <new>
#include <string>
#include <thread>
#include <vector>

namespace {

using i64 = int64_t;

thread_local std::string g_err;

int fail(const char* msg) {
  g_err = std::string("invalid argument: ") + msg;
  return -1;
}

// All workers wait until every one has arrived; generation counting makes it
// reusable.  Waiters spin briefly, then yield (threads never block forever:
// every worker reaches every barrier).
class Barrier {
 public:
  explicit Barrier(int n) : n_(n) {}
  void wait() {
    const unsigned g = gen_.load(std::memory_order_acquire);
    if (arrived_.fetch_add(1, std::memory_order_acq_rel) == n_ - 1) {
      arrived_.store(0, std::memory_order_relaxed);
      gen_.fetch_add(1, std::memory_order_release);
      return;
    }
    for (int spin = 0; gen_.load(std::memory_order_acquire) == g; spin++)
      if (spin > 256) std::this_thread::yield();
  }

 private:
  const int n_;
  std::atomic<int> arrived_{0};
  std::atomic<unsigned> gen_{0};
};

constexpr int kMaxThreads = 1024;

int resolve_threads(int nthreads, i64 rows) {
  int t = nthreads > 0 ? nthreads : (int)std::max(1u, std::thread::hardware_concurrency());
  if (t > kMaxThreads) t = kMaxThreads;
  if ((i64)t > rows) t = (int)std::max<i64>(rows, 1);
  return t;
}

// Runs body(t) on threads 0..T-1 (0 = the caller) and joins them.
template <typename F>
int run_workers(int T, F&& body) {
  std::vector<std::thread> th;
  try {
    th.reserve((size_t)T - 1);
    for (int t = 1; t < T; t++) th.emplace_back(body, t);
  } catch (...) {
    for (auto& x : th) x.join();
    g_err = "cannot start worker threads";
    return -2;
  }
  body(0);
  for (auto& x : th) x.join();
  return 0;
}

// One row of interior points starting at padded offset p0 (n points): the
// star update with radius R, written to out[i] for the row's i-th point
// (`out` points at the row's first point); sy = NX (row stride), sz = NX*NY
// (plane stride, 0 for the 2-D form).
template <int R, bool D3, bool C0, bool HB>
void row_update(const double* __restrict u, const double* __restrict b, double* __restrict out, i64 p0, i64 n,
                i64 sy, i64 sz, const double* c) {
  const double c1 = c[1], cr = c[R], c0 = c[0];
  for (i64 i = 0; i < n; i++) {
    const i64 p = p0 + i;
    double sx = u[p - R] + u[p + R];
    double syv = u[p - R * sy] + u[p + R * sy];
    double s = sx + syv;
    if (D3) s = s + (u[p - R * sz] + u[p + R * sz]);
    double acc = cr * s;
    if (R == 2) {
      double tx = u[p - 1] + u[p + 1];
      double ty = u[p - sy] + u[p + sy];
      double t = tx + ty;
      if (D3) t = t + (u[p - sz] + u[p + sz]);
      acc = acc + c1 * t;
    }
    if (C0) acc = acc + c0 * u[p];
    if (HB) acc = acc + b[p];
    out[i] = acc;
  }
}

using RowFn = void (*)(const double*, const double*, double*, i64, i64, i64, i64, const double*);

template <bool D3>
RowFn pick_row(int r, bool c0, bool hb) {
  if (r == 1) {
    if (c0) return hb ? row_update<1, D3, true, true> : row_update<1, D3, true, false>;
    return hb ? row_update<1, D3, false, true> : row_update<1, D3, false, false>;
  }
  if (c0) return hb ? row_update<2, D3, true, true> : row_update<2, D3, true, false>;
  return hb ? row_update<2, D3, false, true> : row_update<2, D3, false, false>;
}

struct Geom {
  i64 nx, ny, nz;  // nz = 1 for the 2-D form (no z halo)
  int r;
  bool d3;
  i64 NX() const { return nx + 2 * r; }
  i64 NY() const { return ny + 2 * r; }
  i64 NZ() const { return d3 ? nz + 2 * r : 1; }
  i64 count() const { return NX() * NY() * NZ(); }
  i64 rows() const { return ny * nz; }
  // padded offset of interior row q (0 .. rows-1), first interior point
  i64 row_start(i64 q) const {
    const i64 j = q % ny + r, k = d3 ? q / ny + r : 0;
    return r + NX() * (j + NY() * k);
  }
};

int check(i64 nx, i64 ny, i64 nz, int radius, const double* coeffs, int nthreads) {
  if (!coeffs) return fail("NULL coeffs");
  if (radius != 1 && radius != 2) return fail("radius must be 1 or 2");
  if (nx < 1 || ny < 1 || nz < 1) return fail("interior extents must be >= 1");
  const i64 lim = (i64)1 << 28;
  if (nx > lim || ny > lim || nz > lim) return fail("extent too large");
  if ((double)(nx + 2 * radius) * (double)(ny + 2 * radius) * (double)(nz + 2 * radius) > 1e15)
    return fail("grid too large");
  if (nthreads < 0) return fail("nthreads < 0");
  return 0;
}

int sweep(double* in, double* out, const Geom& g, const double* c, i64 iters, int nthreads) {
  if (!in || !out) return fail("NULL grid");
  if (iters < 0) return fail("iters < 0");
  const size_t bytes = (size_t)g.count() * sizeof(double);
  const char *a = (const char*)in, *z = (const char*)out;
  if (a < z + bytes && z < a + bytes) return fail("in and out overlap");
  memcpy(out, in, bytes);  // out's halo (and everything, for iters == 0)
  if (iters == 0) return 0;
  const RowFn fn = g.d3 ? pick_row<true>(g.r, c[0] != 0.0, false) : pick_row<false>(g.r, c[0] != 0.0, false);
  const i64 rows = g.rows();
  const int T = resolve_threads(nthreads, rows);
  Barrier bar(T);
  const i64 sy = g.NX(), sz = g.d3 ? g.NX() * g.NY() : 0;
  // sweep `it` reads in (even it) or out (odd it) and writes the other
  int rc = run_workers(T, [&](int t) {
    const i64 q0 = rows * t / T, q1 = rows * (t + 1) / T;
    for (i64 it = 0; it < iters; it++) {
      const double* src = it % 2 ? out : in;
      double* dst = it % 2 ? in : out;
      for (i64 q = q0; q < q1; q++) {
        const i64 p0 = g.row_start(q);
        fn(src, nullptr, dst + p0, p0, g.nx, sy, sz, c);
      }
      bar.wait();  // every row of this sweep written before any is read again
    }
  });
  if (rc) return rc;
  // after an odd count the last sweep wrote `out`; after an even count, `in`
  if (iters % 2 == 0) memcpy(out, in, bytes);
  return 0;
}

int residual(const double* u, const double* b, const Geom& g, const double* c, double* norm_out, int nthreads) {
  if (!u) return fail("NULL grid");
  if (!norm_out) return fail("NULL norm_out");
  const i64 rows = g.rows();
  std::vector<double> part;
  std::vector<double> tmp;
  try {
    part.assign((size_t)rows, 0.0);
  } catch (const std::bad_alloc&) {
    g_err = "host allocation failed";
    return -2;
  }
  const RowFn fn = g.d3 ? pick_row<true>(g.r, c[0] != 0.0, b != nullptr)
                        : pick_row<false>(g.r, c[0] != 0.0, b != nullptr);
  const int T = resolve_threads(nthreads, rows);
  const i64 sy = g.NX(), sz = g.d3 ? g.NX() * g.NY() : 0;
  try {
    tmp.assign((size_t)T * (size_t)g.nx, 0.0);  // one row buffer per thread
  } catch (const std::bad_alloc&) {
    g_err = "host allocation failed";
    return -2;
  }
  int rc = run_workers(T, [&](int t) {
    const i64 q0 = rows * t / T, q1 = rows * (t + 1) / T;
    double* row = tmp.data() + (size_t)t * (size_t)g.nx;
    for (i64 q = q0; q < q1; q++) {
      const i64 p0 = g.row_start(q);
      fn(u, b, row, p0, g.nx, sy, sz, c);
      double s = 0.0;
      for (i64 i = 0; i < g.nx; i++) {
        const double rho = row[i] - u[p0 + i];
        s = s + rho * rho;
      }
      part[(size_t)q] = s;
    }
  });
  if (rc) return rc;
  double sum = 0.0;
  for (i64 q = 0; q < rows; q++) sum = sum + part[(size_t)q];
  *norm_out = sqrt(sum);
  return 0;
}

// One row of advection tendencies: for each of the nf fields q[m], s[m] at
// the row's interior points (i = 1..nx, padded offset p0 + i - 1), in the
// order of advect_f64.
void advect_row(const double* __restrict u, const double* __restrict v, const double* __restrict w,
                const double* const* q, double* const* s, int nf, i64 p0, i64 nx, i64 NX, i64 NXY,
                const double* c) {
  const double cx = c[0], cy = c[1], cz = c[2];
  for (int m = 0; m < nf; m++) {
    const double* __restrict f = q[m];
    double* __restrict o = s[m];
    for (i64 i = 0; i < nx; i++) {
      const i64 p = p0 + i;
      const double fmx = (u[p - 1] + u[p]) * (f[p - 1] + f[p]);
      const double fpx = (u[p] + u[p + 1]) * (f[p] + f[p + 1]);
      const double tx = cx * (fmx - fpx);
      const double fmy = (v[p - NX] + v[p]) * (f[p - NX] + f[p]);
      const double fpy = (v[p] + v[p + NX]) * (f[p] + f[p + NX]);
      const double ty = cy * (fmy - fpy);
      const double fmz = (w[p - NXY] + w[p]) * (f[p - NXY] + f[p]);
      const double fpz = (w[p] + w[p + NXY]) * (f[p] + f[p + NXY]);
      const double tz = cz * (fmz - fpz);
      o[p] = (tx + ty) + tz;
    }
  }
}

}  // namespace

extern "C" {

const char* stencil_host_last_error(void) { return g_err.c_str(); }

int stencil_host_threads(void) { return (int)std::max(1u, std::thread::hardware_concurrency()); }

int stencil_host_sweep_f64(double* in, double* out, int64_t nx, int64_t ny, int64_t nz, const double* coeffs,
                           int radius, int64_t iters, int nthreads) {
  g_err.clear();
  if (int rc = check(nx, ny, nz, radius, coeffs, nthreads)) return rc;
  return sweep(in, out, Geom{nx, ny, nz, radius, true}, coeffs, iters, nthreads);
}

int stencil_host_residual_norm_f64(const double* u, const double* b, int64_t nx, int64_t ny, int64_t nz,
                                   const double* coeffs, int radius, double* norm_out, int nthreads) {
  g_err.clear();
  if (int rc = check(nx, ny, nz, radius, coeffs, nthreads)) return rc;
  return residual(u, b, Geom{nx, ny, nz, radius, true}, coeffs, norm_out, nthreads);
}

int stencil_host_sweep2d_f64(double* in, double* out, int64_t nx, int64_t ny, const double* coeffs, int radius,
                             int64_t iters, int nthreads) {
  g_err.clear();
  if (int rc = check(nx, ny, 1, radius, coeffs, nthreads)) return rc;
  return sweep(in, out, Geom{nx, ny, 1, radius, false}, coeffs, iters, nthreads);
}

int stencil_host_advect_f64(const double* u, const double* v, const double* w, const double* const* q, int nq,
                            double* const* s, int64_t nx, int64_t ny, int64_t nz, const double* c, int nthreads) {
  g_err.clear();
  if (!u || !v || !w || !s || !c) return fail("NULL pointer");
  if (q && (nq < 1 || nq > 6)) return fail("nq must be in [1, 6]");
  if (int rc = check(nx, ny, nz, 1, c, nthreads)) return rc;
  for (int a = 0; a < 3; a++)
    if (!std::isfinite(c[a])) return fail("non-finite coefficient");
  const int nf = q ? nq : 3;
  const double* fields[6];
  double* outs[6];
  for (int m = 0; m < nf; m++) {
    fields[m] = q ? q[m] : (m == 0 ? u : (m == 1 ? v : w));
    outs[m] = s[m];
    if (!fields[m] || !outs[m]) return fail("NULL field or output");
  }
  const Geom g{nx, ny, nz, 1, true};
  const size_t bytes = (size_t)g.count() * sizeof(double);
  auto overlaps = [&](const void* x, const void* y) {
    const char *a = (const char*)x, *b = (const char*)y;
    return a < b + bytes && b < a + bytes;
  };
  for (int m = 0; m < nf; m++) {
    for (const double* in : {u, v, w})
      if (overlaps(outs[m], in)) return fail("an output overlaps an input");
    for (int k = 0; k < nf; k++)
      if (overlaps(outs[m], fields[k]) || (k != m && overlaps(outs[m], outs[k])))
        return fail("an output overlaps an input or another output");
  }
  const i64 rows = g.rows();
  const int T = resolve_threads(nthreads, rows);
  const i64 NX = g.NX(), NXY = g.NX() * g.NY();
  return run_workers(T, [&](int t) {
    const i64 q0 = rows * t / T, q1 = rows * (t + 1) / T;
    for (i64 r = q0; r < q1; r++) advect_row(u, v, w, fields, outs, nf, g.row_start(r), nx, NX, NXY, c);
  });
}

int stencil_host_residual_norm2d_f64(const double* u, const double* b, int64_t nx, int64_t ny,
                                     const double* coeffs, int radius, double* norm_out, int nthreads) {
  g_err.clear();
  if (int rc = check(nx, ny, 1, radius, coeffs, nthreads)) return rc;
  return residual(u, b, Geom{nx, ny, 1, radius, false}, coeffs, norm_out, nthreads);
}

}  // extern "C"
