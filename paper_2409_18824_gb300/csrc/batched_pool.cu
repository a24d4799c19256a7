// Batched solves on a pool of worker streams (batch engine 2).
//
// The persistent scheduler (sched.cu) splits every problem's passes into
// small work units that any CTA claims; that packs many small problems well
// but runs the large ones, which hold most of a batch's work, on its unit
// tile code.  This engine instead hands the problems, largest estimated work
// first, to a fixed pool of host worker threads, each with its own stream:
// a worker solves one problem at a time with the one-problem cores
// (solve_refined_core / solve_jacobi_core: the full-grid kernels, or the
// resident launch for small grids), so the kernels of different problems
// overlap on the device and every problem gets the fastest single-problem
// path.  A problem's result depends only on the problem: it is the same
// bits as jacobi_solve_refined_f64 / jacobi_solve_f64 on it alone.
//
// The worker streams are created once per device and kept, so their
// per-stream workspaces are reused from call to call; each worker keeps one
// set of scratch grids, grown to the largest problem it has met.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

namespace stn {

namespace {

constexpr int kPoolWorkers = 8;
constexpr int kMaxDevices = 64;

struct Worker {
  cudaStream_t stream = nullptr;
  void* scratch = nullptr;  // one double grid and three float grids of the largest problem so far
  size_t bytes = 0;
  bool ready = false;
};

std::mutex g_pool_mu;                   // one batch at a time per process uses the pool
Worker g_workers[kMaxDevices][kPoolWorkers];

int prepare(Worker& w, size_t need) {
  if (!w.stream) {
    STN_CUDA_TRY(cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking));
    // reduction slots sized once: growing them later would synchronise the
    // device under the other workers
    Workspace* ws;
    if (int rc = get_workspace(w.stream, (i64)1 << 17, 0, &ws)) return rc;
  }
  if (w.bytes < need) {
    if (w.scratch) STN_CUDA_TRY(cudaFreeAsync(w.scratch, w.stream));
    w.scratch = nullptr;
    w.bytes = 0;
    keep_pool_memory();
    cudaError_t e = cudaMallocAsync(&w.scratch, need, w.stream);
    if (e == cudaErrorMemoryAllocation) {
      (void)cudaGetLastError();
      set_error("device allocation of batch scratch failed");
      return STN_ENOMEM;
    }
    STN_CUDA_TRY(e);
    w.bytes = need;
  }
  return STN_OK;
}

}  // namespace

int batched_pool(const stn_problem* probs, i64 count, const double* coeffs, int radius, double tol, i64 iters,
                 i64 check_every, double inner_tol, i64 max_outer, bool refined, stn_solve_info* infos,
                 cudaStream_t s) {
  int dev = 0;
  STN_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal out of range for the batch pool");
    return STN_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_pool_mu);
  // largest estimated work first: points x sweeps, the sweeps of a Jacobi
  // solve growing as 1 / (1/nx^2 + 1/ny^2 + 1/nz^2)
  std::vector<i64> order((size_t)count);
  std::vector<double> work((size_t)count);
  size_t need = 0;
  for (i64 i = 0; i < count; i++) {
    const stn_problem& p = probs[i];
    const double inv = 1.0 / ((double)p.nx * p.nx) + 1.0 / ((double)p.ny * p.ny) + 1.0 / ((double)p.nz * p.nz);
    work[(size_t)i] = (double)p.nx * p.ny * p.nz / inv;
    order[(size_t)i] = i;
    const size_t n = (size_t)Grid{p.nx, p.ny, p.nz, radius}.count();
    const size_t b = (n * 8 + 255) / 256 * 256 + (refined ? 3 * ((n * 4 + 255) / 256 * 256) : 0);
    need = std::max(need, b);
  }
  std::stable_sort(order.begin(), order.end(),
                   [&](i64 a, i64 b) { return work[(size_t)a] > work[(size_t)b]; });
  const int nw = (int)std::min<i64>(kPoolWorkers, count);
  // the batch starts after the caller's earlier work on s
  cudaEvent_t start;
  STN_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  STN_CUDA_TRY(cudaEventRecord(start, s));
  std::atomic<i64> next{0};
  std::atomic<int> failed{STN_OK};
  std::vector<int> worst((size_t)nw, STN_OK);
  std::vector<std::string> err((size_t)nw);
  auto run = [&](int w) {
    cudaSetDevice(dev);
    Worker& wk = g_workers[dev][w];
    int rc = prepare(wk, need);
    if (rc == STN_OK && cudaStreamWaitEvent(wk.stream, start, 0) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "wait");
    if (rc != STN_OK) {
      failed.store(rc);
      err[(size_t)w] = stencil_last_error();
      return;
    }
    for (;;) {
      if (failed.load() != STN_OK) return;
      const i64 k = next.fetch_add(1);
      if (k >= count) return;
      const i64 i = order[(size_t)k];
      const stn_problem& p = probs[i];
      const Grid g{p.nx, p.ny, p.nz, radius};
      const size_t n = (size_t)g.count();
      double* t = (double*)wk.scratch;
      float* f32 = (float*)((char*)wk.scratch + (n * 8 + 255) / 256 * 256);
      stn_solve_info info{};
      const int st = refined ? solve_refined_core(p.rhs, p.u, t, f32, g, coeffs, tol, iters, inner_tol, check_every,
                                                  max_outer, &info, wk.stream)
                             : solve_jacobi_core(p.rhs, p.u, t, g, coeffs, tol, iters, check_every, &info, wk.stream);
      if (st < 0) {
        failed.store(st);
        err[(size_t)w] = stencil_last_error();
        return;
      }
      if (infos) infos[i] = info;
      if (st != STN_OK) worst[(size_t)w] = STN_NOT_CONVERGED;
    }
  };
  std::vector<std::thread> th;
  for (int w = 1; w < nw; w++) th.emplace_back(run, w);
  run(0);
  for (auto& x : th) x.join();
  cudaEventDestroy(start);
  // the caller's stream orders after the batch: each worker's solve ended
  // with a synchronisation of its stream, so the work is complete here
  if (const int f = failed.load(); f != STN_OK) {
    for (const auto& m : err)
      if (!m.empty()) {
        set_error(m);
        break;
      }
    return f;
  }
  for (int w : worst)
    if (w != STN_OK) return STN_NOT_CONVERGED;
  return STN_OK;
}

}  // namespace stn
