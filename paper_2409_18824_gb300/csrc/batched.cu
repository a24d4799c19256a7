// Batched Jacobi solves in one persistent launch (thread-block clusters).
//
// Many independent problems u = S u + b of different extents (the solve of
// arXiv 2409.18824 Sec. 4, many times over) run in ONE kernel launch: every
// cluster of CS CTAs takes the next problem from a device-side queue (ordered
// largest-work first), sweeps it to convergence and takes the next one.
//   * the sweeps of one problem are split into work units (32 x 8 column
//     tiles x k chunks) dealt round-robin to the cluster's CTAs; each unit is
//     swept by star_tile, the same code (and so the same bits) as the
//     single-problem path;
//   * consecutive sweeps are separated by the cluster's hardware barrier
//     (barrier.cluster arrive/wait, release/acquire): no software spin-wait;
//   * convergence checks reduce per-CTA partial sums through distributed
//     shared memory in rank order, so every CTA takes the same decision and a
//     result depends only on its own problem, never on the other problems of
//     the launch.
// The refined variant keeps double only for the residual and the update and
// runs the sweeps of the correction equation e = S e + rho/s in float.
#include <cooperative_groups.h>

#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "work_sched.h"
#include "star.cuh"

namespace cg = cooperative_groups;

namespace stn {

namespace {

constexpr int BT = TX * TY;  // threads per CTA (256)
constexpr int BATCH_CS = 8;  // CTAs per cluster

struct BatchProblem {
  int nx, ny, nz;
  int pad;
  double* u;        // caller's iterate (in/out)
  const double* b;  // caller's source term (may be null)
  double* t;        // scratch double grid
  float* e;         // refined: correction iterate
  float* e2;        // refined: correction ping-pong
  float* r32;       // refined: scaled residual (float)
};

struct BatchResult {
  long long iters;
  long long outer;
  double rel_res;
  double res_norm;
  double rhs_norm;
  int status;
  int pad;
};

struct BatchArgs {
  const BatchProblem* probs;
  const int* order;
  int count;
  int* head;
  BatchResult* results;
  double tol;
  long long max_iters;    // plain: sweeps; refined: inner sweeps per outer step
  long long check_every;  // plain: sweeps per check; refined: inner sweeps per inner check
  double inner_tol;       // refined: inner stop at ||rho_e|| <= inner_tol * ||r32|| (0 = never)
  long long max_outer;    // refined
};

// Work units of one problem: 32 x 8 column tiles of the plane x chunks of k.
struct Units {
  int tiles_x, tiles_y, kc, klen, n;
};

__device__ __forceinline__ Units make_units(int nx, int ny, int nz, int cs) {
  Units w;
  w.tiles_x = (nx + TX - 1) / TX;
  w.tiles_y = (ny + TY - 1) / TY;
  const int tiles = w.tiles_x * w.tiles_y;
  int kc = (4 * cs + tiles - 1) / tiles;
  if (kc > nz) kc = nz;
  if (kc < 1) kc = 1;
  w.klen = (nz + kc - 1) / kc;
  w.kc = (nz + w.klen - 1) / w.klen;
  w.n = tiles * w.kc;
  return w;
}

__device__ __forceinline__ int flat_tid() { return threadIdx.x + blockDim.x * threadIdx.y; }

__device__ __forceinline__ double block_max(double v, double* red) {
  const int lane = flat_tid() & 31, warp = flat_tid() >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < BT / 32 ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
  }
  __syncthreads();
  return t;
}

// Sum (or max) of one value per CTA (valid in thread 0) over the cluster, in
// rank order; returned to every thread of every CTA.  `part` is a per-CTA
// shared array of at least CS doubles; rank 0's copy collects the values.
__device__ __forceinline__ double cluster_reduce(cg::cluster_group& cl, double v, double* part,
                                                 double* bcast, bool is_max) {
  const unsigned rank = cl.block_rank(), cs = cl.num_blocks();
  if (flat_tid() == 0) *cl.map_shared_rank(&part[rank], 0) = v;
  cl.sync();
  if (flat_tid() == 0) {
    const double* p0 = cl.map_shared_rank(part, 0);
    double s = 0.0;
    for (unsigned r = 0; r < cs; r++) s = is_max ? fmax(s, p0[r]) : s + p0[r];
    *bcast = s;
  }
  __syncthreads();
  const double s = *bcast;
  cl.sync();  // rank 0's part[] is reused only after every CTA has read it
  return s;
}

// Interior points handed to this CTA: whole rows, CTA `rank` takes rows
// rank, rank+cs, ...; threads stride along the row.  Fixed order per thread.
template <typename F>
__device__ __forceinline__ void for_interior_rows(int nx, int ny, int nz, int r, unsigned rank,
                                                  unsigned cs, F&& f) {
  const i64 NX = nx + 2 * r, NY = ny + 2 * r;
  const i64 rows = (i64)ny * nz;
  for (i64 row = rank; row < rows; row += cs) {
    const i64 j = row % ny + r, k = row / ny + r;
    const i64 base = r + NX * (j + NY * k);
    for (int i = flat_tid(); i < nx; i += BT) f(base + i);
  }
}

// Every cell of the padded grid (halo included), rows dealt to the CTAs.
template <typename F>
__device__ __forceinline__ void for_all_rows(int nx, int ny, int nz, int r, unsigned rank, unsigned cs,
                                             F&& f) {
  const i64 NX = nx + 2 * r;
  const i64 rows = (i64)(ny + 2 * r) * (nz + 2 * r);
  for (i64 row = rank; row < rows; row += cs)
    for (int i = flat_tid(); i < NX; i += BT) f(row * NX + i);
}

// Copies the halo cells of src into dst.
template <typename T>
__device__ __forceinline__ void cluster_copy_halo(const T* src, T* dst, int nx, int ny, int nz,
                                                  int r, unsigned rank, unsigned cs) {
  const int NX = nx + 2 * r, NY = ny + 2 * r;
  const i64 rows = (i64)NY * (nz + 2 * r);
  for (i64 row = rank; row < rows; row += cs) {
    const int j = (int)(row % NY), k = (int)(row / NY);
    const i64 base = row * NX;
    if (k < r || k >= nz + r || j < r || j >= ny + r) {
      for (int i = flat_tid(); i < NX; i += BT) dst[base + i] = src[base + i];
    } else if (flat_tid() < 2 * r) {
      const int i = flat_tid() < r ? flat_tid() : nx + flat_tid();
      dst[base + i] = src[base + i];
    }
  }
}

template <typename T, int R, bool HAS_B, bool HAS_C0, int MODE>
__device__ __forceinline__ double cluster_sweep(const T* cur, const T* b, T* nxt, int nx, int ny,
                                                int nz, const Units& w, unsigned rank, unsigned cs,
                                                const StarCoeffs<T, R>& cf, T (*tile)[TX + 2 * R]) {
  const int NX = nx + 2 * R, NY = ny + 2 * R;
  const int tiles = w.tiles_x * w.tiles_y;
  double rsum = 0.0;
  for (int q = rank; q < w.n; q += cs) {
    const int kci = q / tiles, tq = q - kci * tiles;
    const int ty = tq / w.tiles_x, tx = tq - ty * w.tiles_x;
    const int k0 = R + kci * w.klen;
    const int k1 = min(k0 + w.klen, nz + R);
    star_tile<T, R, HAS_B, HAS_C0, MODE>(cur, b, nxt, nx, ny, NX, NY, tx, ty, k0, k1, cf, TX, TY, &tile[0][0],
                                         &rsum);
  }
  return rsum;
}

// Takes the next problem index for the whole cluster (-1 when none is left).
__device__ __forceinline__ int cluster_next(cg::cluster_group& cl, const BatchArgs& a, int* s_idx) {
  if (cl.block_rank() == 0 && flat_tid() == 0) *s_idx = atomicAdd(a.head, 1);
  cl.sync();
  const int idx = *cl.map_shared_rank(s_idx, 0);
  cl.sync();  // rank 0 overwrites s_idx only after everyone has read it
  return idx < a.count ? idx : -1;
}

__device__ __forceinline__ double rhs_norm(cg::cluster_group& cl, const BatchProblem& P, int R,
                                           double* red, double* part, double* bcast) {
  double bs = 0.0;
  if (P.b) for_interior_rows(P.nx, P.ny, P.nz, R, cl.block_rank(), cl.num_blocks(), [&](i64 p) {
      const double v = P.b[p];
      bs = __fma_rn(v, v, bs);
    });
  return sqrt(cluster_reduce(cl, block_sum_fixed<BT>(bs, red), part, bcast, false));
}

template <int R, bool HAS_C0>
__global__ void __launch_bounds__(BT) batch_jacobi_kernel(BatchArgs a, StarCoeffs<double, R> cf) {
  __shared__ double tile[TY + 2 * R][TX + 2 * R];
  __shared__ double red[BT / 32];
  __shared__ double part[16];
  __shared__ double bcast;
  __shared__ int s_idx;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank(), cs = cl.num_blocks();
  for (;;) {
    const int idx = cluster_next(cl, a, &s_idx);
    if (idx < 0) break;
    const int pi = a.order[idx];
    const BatchProblem P = a.probs[pi];
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const Units w = make_units(nx, ny, nz, cs);
    const double bnorm = rhs_norm(cl, P, R, red, part, &bcast);
    const double scale = bnorm > 0.0 ? bnorm : 1.0;
    cluster_copy_halo(P.u, P.t, nx, ny, nz, R, rank, cs);
    cl.sync();
    double* cur = P.u;
    double* nxt = P.t;
    long long it = 0;
    double rel = INFINITY, res = INFINITY;
    int status = STN_NOT_CONVERGED;
    while (it < a.max_iters) {
      const long long group = min(a.check_every, a.max_iters - it);
      double rs = 0.0;
      for (long long g = 0; g < group; g++) {
        const bool last = g == group - 1;
        if (P.b) {
          if (last) rs = cluster_sweep<double, R, true, HAS_C0, kSweepResidual>(cur, P.b, nxt, nx, ny, nz, w, rank, cs, cf, tile);
          else cluster_sweep<double, R, true, HAS_C0, kSweep>(cur, P.b, nxt, nx, ny, nz, w, rank, cs, cf, tile);
        } else {
          if (last) rs = cluster_sweep<double, R, false, HAS_C0, kSweepResidual>(cur, nullptr, nxt, nx, ny, nz, w, rank, cs, cf, tile);
          else cluster_sweep<double, R, false, HAS_C0, kSweep>(cur, nullptr, nxt, nx, ny, nz, w, rank, cs, cf, tile);
        }
        cl.sync();
        double* t = cur;
        cur = nxt;
        nxt = t;
      }
      it += group;
      res = sqrt(cluster_reduce(cl, block_sum_fixed<BT>(rs, red), part, &bcast, false));
      rel = res / scale;
      if (rel <= a.tol) {
        status = STN_OK;
        break;
      }
    }
    if (cur != P.u) {
      for_interior_rows(nx, ny, nz, R, rank, cs, [&](i64 p) { P.u[p] = cur[p]; });
      cl.sync();
    }
    if (rank == 0 && flat_tid() == 0) {
      BatchResult r;
      r.iters = it;
      r.outer = 0;
      r.rel_res = rel;
      r.res_norm = res;
      r.rhs_norm = bnorm;
      r.status = status;
      r.pad = 0;
      a.results[pi] = r;
    }
  }
}

template <int R, bool HAS_C0>
__global__ void __launch_bounds__(BT)
    batch_refined_kernel(BatchArgs a, StarCoeffs<double, R> cf, StarCoeffs<float, R> cf32) {
  __shared__ double tile[TY + 2 * R][TX + 2 * R];
  __shared__ float tile32[TY + 2 * R][TX + 2 * R];
  __shared__ double red[BT / 32];
  __shared__ double part[16];
  __shared__ double bcast;
  __shared__ int s_idx;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank(), cs = cl.num_blocks();
  for (;;) {
    const int idx = cluster_next(cl, a, &s_idx);
    if (idx < 0) break;
    const int pi = a.order[idx];
    const BatchProblem P = a.probs[pi];
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const Units w = make_units(nx, ny, nz, cs);
    const double bnorm = rhs_norm(cl, P, R, red, part, &bcast);
    const double scale = bnorm > 0.0 ? bnorm : 1.0;
    // the correction grids start at zero, halo included (homogeneous Dirichlet)
    for_all_rows(nx, ny, nz, R, rank, cs, [&](i64 p) {
      P.e[p] = 0.0f;
      P.e2[p] = 0.0f;
      P.r32[p] = 0.0f;
    });
    cl.sync();
    long long outer = 0, sweeps = 0;
    double rel = INFINITY, res = INFINITY;
    int status = STN_NOT_CONVERGED;
    for (;;) {
      // double residual: t = S u + b, rho = t - u
      double rs;
      if (P.b) rs = cluster_sweep<double, R, true, HAS_C0, kSweepResidual>(P.u, P.b, P.t, nx, ny, nz, w, rank, cs, cf, tile);
      else rs = cluster_sweep<double, R, false, HAS_C0, kSweepResidual>(P.u, nullptr, P.t, nx, ny, nz, w, rank, cs, cf, tile);
      cl.sync();
      res = sqrt(cluster_reduce(cl, block_sum_fixed<BT>(rs, red), part, &bcast, false));
      rel = res / scale;
      if (rel <= a.tol) {
        status = STN_OK;
        break;
      }
      if (outer >= a.max_outer) break;
      double mx = 0.0;
      for_interior_rows(nx, ny, nz, R, rank, cs,
                        [&](i64 p) { mx = fmax(mx, fabs(__dsub_rn(P.t[p], P.u[p]))); });
      const double smax = cluster_reduce(cl, block_max(mx, red), part, &bcast, true);
      if (!(smax > 0.0)) break;
      double rn = 0.0;
      for_interior_rows(nx, ny, nz, R, rank, cs, [&](i64 p) {
        const float v = __double2float_rn(__ddiv_rn(__dsub_rn(P.t[p], P.u[p]), smax));
        P.r32[p] = v;
        P.e[p] = 0.0f;
        rn = __fma_rn((double)v, (double)v, rn);
      });
      const double r32norm = sqrt(cluster_reduce(cl, block_sum_fixed<BT>(rn, red), part, &bcast, false));
      // float sweeps of the correction equation e = S e + r32 from e = 0
      float* cur = P.e;
      float* nxt = P.e2;
      long long k = 0;
      while (k < a.max_iters) {
        const long long group = min(a.check_every, a.max_iters - k);
        double rse = 0.0;
        for (long long g = 0; g < group; g++) {
          if (a.inner_tol > 0.0 && g == group - 1)
            rse = cluster_sweep<float, R, true, HAS_C0, kSweepResidual>(cur, P.r32, nxt, nx, ny, nz, w, rank, cs, cf32, tile32);
          else
            cluster_sweep<float, R, true, HAS_C0, kSweep>(cur, P.r32, nxt, nx, ny, nz, w, rank, cs, cf32, tile32);
          cl.sync();
          float* t = cur;
          cur = nxt;
          nxt = t;
        }
        k += group;
        if (a.inner_tol > 0.0) {
          const double rin = sqrt(cluster_reduce(cl, block_sum_fixed<BT>(rse, red), part, &bcast, false));
          if (rin <= a.inner_tol * r32norm) break;
        }
      }
      sweeps += k;
      for_interior_rows(nx, ny, nz, R, rank, cs,
                        [&](i64 p) { P.u[p] = __dadd_rn(P.u[p], __dmul_rn(smax, (double)cur[p])); });
      cl.sync();
      outer++;
    }
    if (rank == 0 && flat_tid() == 0) {
      BatchResult r;
      r.iters = sweeps;
      r.outer = outer;
      r.rel_res = rel;
      r.res_norm = res;
      r.rhs_norm = bnorm;
      r.status = status;
      r.pad = 0;
      a.results[pi] = r;
    }
  }
}

}  // namespace

// Estimated work of a problem: points x sweeps to reduce the slowest mode by
// a fixed factor, 1/(1 - rho) with 1 - rho ~ (pi^2/6) sum_a 1/(n_a+1)^2.
static double est_work(i64 nx, i64 ny, i64 nz) {
  const double g = 1.0 / ((nx + 1.0) * (nx + 1.0)) + 1.0 / ((ny + 1.0) * (ny + 1.0)) +
                   1.0 / ((nz + 1.0) * (nz + 1.0));
  return (double)nx * ny * nz / g;
}

static int batched_clusters(const stn_problem* probs, i64 count, const double* coeffs, int radius,
                            double tol, i64 iters, i64 check_every, double inner_tol, i64 max_outer,
                            bool refined, stn_solve_info* infos, cudaStream_t s) {
  std::vector<BatchProblem> hp((size_t)count);
  std::vector<int> order((size_t)count);
  size_t pool64 = 0, pool32 = 0;
  for (i64 i = 0; i < count; i++) {
    const stn_problem& p = probs[i];
    const size_t n = (size_t)((p.nx + 2 * radius) * (p.ny + 2 * radius) * (p.nz + 2 * radius));
    pool64 += (n + 31) / 32 * 32;
    if (refined) pool32 += 3 * ((n + 63) / 64 * 64);
  }
  // scratch pool, descriptors, order, results, queue head: one allocation
  const size_t off_desc = 0;
  const size_t off_order = off_desc + sizeof(BatchProblem) * (size_t)count;
  const size_t off_res = (off_order + sizeof(int) * (size_t)count + 255) / 256 * 256;
  const size_t off_head = off_res + sizeof(BatchResult) * (size_t)count;
  const size_t off_64 = (off_head + 256 + 255) / 256 * 256;
  const size_t off_32 = off_64 + pool64 * sizeof(double);
  const size_t total = off_32 + pool32 * sizeof(float) + 256;
  char* base = nullptr;
  keep_pool_memory();
  cudaError_t e = cudaMallocAsync((void**)&base, total, s);
  if (e == cudaErrorMemoryAllocation) {
    (void)cudaGetLastError();
    set_error("batched solver: device allocation of scratch failed");
    return STN_ENOMEM;
  }
  STN_CUDA_TRY(e);
  double* p64 = (double*)(base + off_64);
  float* p32 = (float*)(base + off_32);
  std::vector<double> work((size_t)count);
  for (i64 i = 0; i < count; i++) {
    const stn_problem& p = probs[i];
    const size_t n = (size_t)((p.nx + 2 * radius) * (p.ny + 2 * radius) * (p.nz + 2 * radius));
    BatchProblem& b = hp[(size_t)i];
    b.nx = (int)p.nx;
    b.ny = (int)p.ny;
    b.nz = (int)p.nz;
    b.pad = 0;
    b.u = p.u;
    b.b = p.rhs;
    b.t = p64;
    p64 += (n + 31) / 32 * 32;
    b.e = b.e2 = b.r32 = nullptr;
    if (refined) {
      const size_t n32 = (n + 63) / 64 * 64;
      b.e = p32;
      b.e2 = p32 + n32;
      b.r32 = p32 + 2 * n32;
      p32 += 3 * n32;
    }
    order[(size_t)i] = (int)i;
    work[(size_t)i] = est_work(p.nx, p.ny, p.nz);
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
  int rc = STN_OK;
  std::vector<BatchResult> hres((size_t)count);
  do {
    if ((e = cudaMemcpyAsync(base + off_desc, hp.data(), sizeof(BatchProblem) * count, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(base + off_order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(base + off_head, 0, 256, s)) != cudaSuccess) break;
    BatchArgs a;
    a.probs = (const BatchProblem*)(base + off_desc);
    a.order = (const int*)(base + off_order);
    a.count = (int)count;
    a.head = (int*)(base + off_head);
    a.results = (BatchResult*)(base + off_res);
    a.tol = tol;
    a.max_iters = iters;
    a.check_every = check_every;
    a.inner_tol = inner_tol;
    a.max_outer = max_outer;
    const bool hc0 = coeffs[0] != 0.0;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = BATCH_CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(TX, TY, 1);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(BATCH_CS, 1, 1);
#define STN_BATCH_LAUNCH(KERN, ...)                                                      \
  {                                                                                      \
    int ncl = 0;                                                                         \
    if ((e = cudaOccupancyMaxActiveClusters(&ncl, KERN, &cfg)) != cudaSuccess) break;    \
    if (ncl < 1) {                                                                       \
      set_error("batched solver: no cluster fits on an SM group");                       \
      rc = STN_ECUDA;                                                                    \
      break;                                                                             \
    }                                                                                    \
    if (ncl > count) ncl = (int)count;                                                   \
    cfg.gridDim = dim3(BATCH_CS * ncl, 1, 1);                                            \
    if ((e = cudaLaunchKernelEx(&cfg, KERN, __VA_ARGS__)) != cudaSuccess) break;         \
  }
    if (radius == 1) {
      StarCoeffs<double, 1> c64;
      StarCoeffs<float, 1> c32;
      for (int d = 0; d <= 1; d++) {
        c64.c[d] = coeffs[d];
        c32.c[d] = (float)coeffs[d];
      }
      if (refined) {
        if (hc0) STN_BATCH_LAUNCH((batch_refined_kernel<1, true>), a, c64, c32)
        else STN_BATCH_LAUNCH((batch_refined_kernel<1, false>), a, c64, c32)
      } else {
        if (hc0) STN_BATCH_LAUNCH((batch_jacobi_kernel<1, true>), a, c64)
        else STN_BATCH_LAUNCH((batch_jacobi_kernel<1, false>), a, c64)
      }
    } else {
      StarCoeffs<double, 2> c64;
      StarCoeffs<float, 2> c32;
      for (int d = 0; d <= 2; d++) {
        c64.c[d] = coeffs[d];
        c32.c[d] = (float)coeffs[d];
      }
      if (refined) {
        if (hc0) STN_BATCH_LAUNCH((batch_refined_kernel<2, true>), a, c64, c32)
        else STN_BATCH_LAUNCH((batch_refined_kernel<2, false>), a, c64, c32)
      } else {
        if (hc0) STN_BATCH_LAUNCH((batch_jacobi_kernel<2, true>), a, c64)
        else STN_BATCH_LAUNCH((batch_jacobi_kernel<2, false>), a, c64)
      }
    }
#undef STN_BATCH_LAUNCH
    if ((e = cudaMemcpyAsync(hres.data(), base + off_res, sizeof(BatchResult) * count, cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
  } while (false);
  cudaFreeAsync(base, s);
  if (rc != STN_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "batched solver");
  int worst = STN_OK;
  for (i64 i = 0; i < count; i++) {
    const BatchResult& r = hres[(size_t)i];
    if (infos) {
      infos[i].iters = r.iters;
      infos[i].outer = r.outer;
      infos[i].rel_res = r.rel_res;
      infos[i].res_norm = r.res_norm;
      infos[i].rhs_norm = r.rhs_norm;
      infos[i].status = r.status;
    }
    if (r.status != STN_OK) worst = STN_NOT_CONVERGED;
  }
  return worst;
}

// Scheduler engine: one persistent launch of the dynamic unit scheduler
// (sched.cu) over all problems, queued largest estimated work first.
// The persistent launch of a batch as a one-node CUDA graph: captured on a
// private stream, instantiated and launched on the caller's stream (which
// may be the legacy default stream, which cannot be captured).  Any failure
// to capture or instantiate falls back to a plain launch (knob batch_graph:
// 1 default, 0 plain).
static int g_batch_graph = 1;
int tune_set_batch_graph(int v) {
  if (v < 0 || v > 1) return STN_EINVAL;
  g_batch_graph = v;
  return STN_OK;
}
int tune_get_batch_graph() { return g_batch_graph; }

static int launch_sched_graph(const SchedArgs& a, int radius, bool hc0, int ctas, cudaStream_t s) {
  if (!g_batch_graph) return sched_launch(a, radius, hc0, ctas, s);
  if (int rc = sched_prepare()) return rc;
  cudaStream_t cs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool launched = false;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess &&
      cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
    const int rc = sched_launch(a, radius, hc0, ctas, cs);
    const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
    if (rc == STN_OK && ec == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess &&
        cudaGraphLaunch(exec, s) == cudaSuccess)
      launched = true;
  }
  // an executable graph that is still running is freed when it completes
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (cs) cudaStreamDestroy(cs);
  if (launched) {
    sched_set_stats_stream(s);
    return STN_OK;
  }
  (void)cudaGetLastError();
  clear_error();
  return sched_launch(a, radius, hc0, ctas, s);
}

static int batched_sched(const stn_problem* probs, i64 count, const double* coeffs, int radius,
                         double tol, i64 iters, i64 check_every, double inner_tol, i64 max_outer,
                         bool refined, stn_solve_info* infos, cudaStream_t s) {
  const bool hc0 = coeffs[0] != 0.0;
  const int ctas = sched_ctas(radius, hc0, refined);
  if (ctas < 1) {
    set_error("scheduler kernel does not fit on an SM");
    return STN_ECUDA;
  }
  const int nslots = (int)std::min<i64>(count, 96);
  // layout of one device allocation
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = (off + bytes + 255) / 256 * 256;
    return o;
  };
  const size_t o_probs = take(sizeof(SchedProblem) * count);
  const size_t o_slots = take(sizeof(SchedSlot) * nslots);
  const size_t o_words = take(sizeof(unsigned long long) * nslots);
  const size_t o_queue = take(sizeof(int) * count);
  const size_t o_ctr = take(sizeof(int) * 8);
  const size_t o_res = take(sizeof(SchedResult) * count);
  const size_t o_flags = take(sizeof(int) * count);
  std::vector<size_t> o_t((size_t)count), o_part((size_t)count), o_e((size_t)count);
  std::vector<size_t> npts((size_t)count);
  std::vector<int> nunits((size_t)count);
  for (i64 i = 0; i < count; i++) {
    const stn_problem& p = probs[i];
    npts[i] = (size_t)((p.nx + 2 * radius) * (p.ny + 2 * radius) * (p.nz + 2 * radius));
    nunits[i] = (int)sched_units(p.nx, p.ny, p.nz);
    o_t[i] = take(sizeof(double) * npts[i]);
    o_part[i] = take(sizeof(double) * nunits[i]);
  }
  const size_t o_f32 = off;
  for (i64 i = 0; i < count && refined; i++) o_e[i] = take(3 * sizeof(float) * ((npts[i] + 63) / 64 * 64));
  const size_t total = off + 256;
  char* base = nullptr;
  keep_pool_memory();
  cudaError_t e = cudaMallocAsync((void**)&base, total, s);
  if (e == cudaErrorMemoryAllocation) {
    (void)cudaGetLastError();
    set_error("batched solver: device allocation of scratch failed");
    return STN_ENOMEM;
  }
  STN_CUDA_TRY(e);
  std::vector<SchedProblem> hp((size_t)count);
  std::vector<double> work((size_t)count);
  std::vector<int> order((size_t)count);
  for (i64 i = 0; i < count; i++) {
    const stn_problem& p = probs[i];
    SchedProblem& q = hp[i];
    q.nx = (int)p.nx;
    q.ny = (int)p.ny;
    q.nz = (int)p.nz;
    q.nunits = nunits[i];
    q.u = p.u;
    q.b = p.rhs;
    q.t = (double*)(base + o_t[i]);
    q.partials = (double*)(base + o_part[i]);
    q.e = q.e2 = q.r32 = nullptr;
    if (refined) {
      const size_t n32 = (npts[i] + 63) / 64 * 64;
      q.e = (float*)(base + o_e[i]);
      q.e2 = q.e + n32;
      q.r32 = q.e2 + n32;
    }
    order[i] = (int)i;
    work[i] = est_work(p.nx, p.ny, p.nz);
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
  std::vector<SchedSlot> hs((size_t)nslots);
  for (auto& sl : hs) {
    memset(&sl, 0, sizeof(sl));
    sl.claim_free = 1;
  }
  std::vector<SchedResult> hres((size_t)count);
  int herr = 0;
  int rc = STN_OK;
  do {
    if ((e = cudaMemcpyAsync(base + o_probs, hp.data(), sizeof(SchedProblem) * count, cudaMemcpyHostToDevice, s))) break;
    if ((e = cudaMemcpyAsync(base + o_slots, hs.data(), sizeof(SchedSlot) * nslots, cudaMemcpyHostToDevice, s))) break;
    if ((e = cudaMemsetAsync(base + o_words, 0, sizeof(unsigned long long) * nslots, s))) break;
    if ((e = cudaMemcpyAsync(base + o_queue, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s))) break;
    if ((e = cudaMemsetAsync(base + o_ctr, 0, sizeof(int) * 8, s))) break;
    if ((e = cudaMemsetAsync(base + o_flags, 0, sizeof(int) * count, s))) break;
    const int free0 = nslots;
    if ((e = cudaMemcpyAsync(base + o_ctr + 3 * sizeof(int), &free0, sizeof(int), cudaMemcpyHostToDevice, s))) break;
    if (refined && (e = cudaMemsetAsync(base + o_f32, 0, off - o_f32, s))) break;
    bool bad = false;
    for (i64 i = 0; i < count; i++)
      if ((e = cudaMemcpyAsync(hp[i].t, hp[i].u, sizeof(double) * npts[i], cudaMemcpyDeviceToDevice, s))) {
        bad = true;
        break;
      }
    if (bad) break;
    SchedArgs a;
    memset(&a, 0, sizeof(a));
    a.probs = (SchedProblem*)(base + o_probs);
    a.slots = (SchedSlot*)(base + o_slots);
    a.words = (unsigned long long*)(base + o_words);
    a.nslots = nslots;
    a.count = (int)count;
    a.qlen = sched_faults().withhold_last ? (int)count - 1 : (int)count;
    a.queue = (const int*)(base + o_queue);
    a.qcap = (int)count;
    int* ctr = (int*)(base + o_ctr);
    a.qhead = ctr + 0;
    a.finished = ctr + 1;
    a.error = ctr + 2;
    a.free_slots = ctr + 3;
    a.qtail = nullptr;
    a.serving = 0;
    a.results = (SchedResult*)(base + o_res);
    a.done_flags = (int*)(base + o_flags);
    for (int d = 0; d < 3; d++) a.coeffs[d] = d <= radius ? coeffs[d] : 0.0;
    a.tol = tol;
    a.max_iters = iters;
    a.check_every = check_every;
    a.inner_tol = inner_tol;
    a.max_outer = max_outer;
    a.refined = refined ? 1 : 0;
    // idle limit without any claimable unit (2 s by default), in SM clock cycles
    a.idle_cycles = sched_faults().idle_ms * 2070000ll;
    if ((rc = launch_sched_graph(a, radius, hc0, ctas, s)) != STN_OK) break;
    if ((e = cudaMemcpyAsync(hres.data(), base + o_res, sizeof(SchedResult) * count, cudaMemcpyDeviceToHost, s))) break;
    if ((e = cudaMemcpyAsync(&herr, ctr + 2, sizeof(int), cudaMemcpyDeviceToHost, s))) break;
    if ((e = cudaStreamSynchronize(s))) break;
  } while (false);
  cudaFreeAsync(base, s);
  if (rc != STN_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "batched scheduler");
  if (herr != 0) {
    set_error(herr == STN_ETIMEOUT ? "batched scheduler: CTAs found no work within the idle limit (stalled)"
                                   : "batched scheduler: device error");
    return herr;
  }
  int worst = STN_OK;
  for (i64 i = 0; i < count; i++) {
    const SchedResult& r = hres[i];
    if (infos) {
      infos[i].iters = r.iters;
      infos[i].outer = r.outer;
      infos[i].rel_res = r.rel_res;
      infos[i].res_norm = r.res_norm;
      infos[i].rhs_norm = r.rhs_norm;
      infos[i].status = r.status;
    }
    if (r.status != STN_OK) worst = STN_NOT_CONVERGED;
  }
  return worst;
}

static int g_batch_engine = 0;
int tune_set_batch_engine(int v) {
  if (v < 0 || v > 2) return STN_EINVAL;
  g_batch_engine = v;
  return STN_OK;
}
int tune_get_batch_engine() { return g_batch_engine; }

int batched_solve(const stn_problem* probs, i64 count, const double* coeffs, int radius, double tol,
                  i64 iters, i64 check_every, double inner_tol, i64 max_outer, bool refined,
                  stn_solve_info* infos, cudaStream_t s) {
  if (g_batch_engine == 1)
    return batched_clusters(probs, count, coeffs, radius, tol, iters, check_every, inner_tol, max_outer,
                            refined, infos, s);
  if (g_batch_engine == 2)
    return batched_pool(probs, count, coeffs, radius, tol, iters, check_every, inner_tol, max_outer, refined,
                        infos, s);
  return batched_sched(probs, count, coeffs, radius, tol, iters, check_every, inner_tol, max_outer,
                       refined, infos, s);
}

}  // namespace stn
