// C ABI of libstencil.so (declared in include/stencil.h): argument checks,
// host-buffer staging, per-(device, stream) workspace and the drivers that
// string the kernels of sweep.cu / varcoef.cu / reduce.cu / refine.cu into
// the calls of the Jacobi path (arXiv 2409.18824 Sec. 4, Sec. 5.3).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <utility>

#include <cmath>
#include <vector>

#include "internal.h"
#include "work_sched.h"

namespace stn {

// ------------------------------------------------------------------ errors --
static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
void clear_error() { g_err.clear(); }
int cuda_fail(cudaError_t e, const char* what) {
  char buf[512];
  snprintf(buf, sizeof buf, "CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
  set_error(buf);
  return STN_ECUDA;
}
static int einval(const char* msg) {
  set_error(std::string("invalid argument: ") + msg);
  return STN_EINVAL;
}

// --------------------------------------------------------------- workspace --
namespace {
std::mutex g_ws_mu;
std::map<std::pair<int, cudaStream_t>, Workspace*> g_ws;
constexpr int kScalars = 64;
}  // namespace

static int grow(void** p, size_t* cap, size_t want) {
  if (*cap >= want) return STN_OK;
  if (*p) {
    STN_CUDA_TRY(cudaDeviceSynchronize());
    STN_CUDA_TRY(cudaFree(*p));
    *p = nullptr;
    *cap = 0;
  }
  cudaError_t e = cudaMalloc(p, want);
  if (e == cudaErrorMemoryAllocation) {
    (void)cudaGetLastError();
    set_error("device allocation of workspace failed");
    return STN_ENOMEM;
  }
  STN_CUDA_TRY(e);
  *cap = want;
  return STN_OK;
}

void keep_pool_memory() {
  static std::atomic<bool> done[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    (void)cudaGetLastError();
    return;
  }
  if (done[dev].exchange(true)) return;
  cudaMemPool_t pool;
  unsigned long long keep = kPoolKeepBytes;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess ||
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess)
    (void)cudaGetLastError();  // an optimisation only: allocations work without it
}

int get_workspace(cudaStream_t stream, i64 partials, size_t grid_bytes, Workspace** out) {
  int dev = 0;
  STN_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_ws_mu);
  Workspace*& ws = g_ws[{dev, stream}];
  if (!ws) ws = new Workspace();
  if (!ws->scalars) {
    STN_CUDA_TRY(cudaMalloc(&ws->scalars, kScalars * sizeof(double)));
    STN_CUDA_TRY(cudaMemset(ws->scalars, 0, kScalars * sizeof(double)));
    STN_CUDA_TRY(cudaMallocHost(&ws->host_scalars, kScalars * sizeof(double)));
  }
  if (partials < 1024) partials = 1024;
  size_t cap = (size_t)ws->partials_cap * sizeof(double);
  int rc = grow((void**)&ws->partials, &cap, (size_t)partials * sizeof(double) * 2);
  if (rc) return rc;
  ws->partials_cap = (i64)(cap / sizeof(double));
  if (grid_bytes) {
    rc = grow(&ws->grid, &ws->grid_bytes, grid_bytes);
    if (rc) return rc;
  }
  *out = ws;
  return STN_OK;
}
int ensure_grid2(Workspace* ws, size_t bytes) { return grow(&ws->grid2, &ws->grid2_bytes, bytes); }
int ensure_grid3(Workspace* ws, size_t bytes) { return grow(&ws->grid3, &ws->grid3_bytes, bytes); }

static int release_all() {
  int dev = 0;
  STN_CUDA_TRY(cudaGetDevice(&dev));
  STN_CUDA_TRY(cudaDeviceSynchronize());
  std::lock_guard<std::mutex> lk(g_ws_mu);
  for (auto it = g_ws.begin(); it != g_ws.end();) {
    if (it->first.first != dev) {
      ++it;
      continue;
    }
    Workspace* ws = it->second;
    cudaFree(ws->partials);
    cudaFree(ws->scalars);
    cudaFree(ws->grid);
    cudaFree(ws->grid2);
    cudaFree(ws->grid3);
    cudaFreeHost(ws->host_scalars);
    delete ws;
    it = g_ws.erase(it);
  }
  return STN_OK;
}

// ------------------------------------------------------------- validation --
static int check_grid(i64 nx, i64 ny, i64 nz, int r) {
  if (r != 1 && r != 2) return einval("radius must be 1 or 2");
  if (nx < 1 || ny < 1 || nz < 1) return einval("interior extents must be >= 1");
  const i64 lim = (i64)1 << 28;
  if (nx > lim || ny > lim || nz > lim) return einval("extent too large");
  const double cells = (double)(nx + 2 * r) * (double)(ny + 2 * r) * (double)(nz + 2 * r);
  if (cells > 9.0e15) return einval("grid too large");
  return STN_OK;
}

static bool overlap(const void* a, const void* b, size_t bytes) {
  const char* x = (const char*)a;
  const char* y = (const char*)b;
  return x < y + bytes && y < x + bytes;
}

// ---------------------------------------------------------------- staging --
// A grid argument: the caller's pointer and, when it is host memory, a device
// copy for the duration of the call.
struct Arg {
  void* user = nullptr;
  void* dev = nullptr;
  size_t bytes = 0;
  bool host = false;
  bool copy_in = false, copy_out = false;
};

static int classify(const void* p, bool* host) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) return cuda_fail(e, "cudaPointerGetAttributes");
  *host = !(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
  return STN_OK;
}

class Stager {
 public:
  explicit Stager(cudaStream_t s) : s_(s) {}
  ~Stager() {
    for (int i = 0; i < n_; i++)
      if (a_[i].host && a_[i].dev) cudaFreeAsync(a_[i].dev, s_);
  }
  // Registers a grid argument; returns its device pointer in *dev.
  int add(const void* p, size_t bytes, bool in, bool out, void** dev) {
    if (!p) {
      *dev = nullptr;
      return STN_OK;
    }
    Arg& a = a_[n_++];
    a.user = const_cast<void*>(p);
    a.bytes = bytes;
    a.copy_in = in;
    a.copy_out = out;
    int rc = classify(p, &a.host);
    if (rc) return rc;
    if (!a.host) {
      a.dev = a.user;
    } else {
      any_host_ = true;
      keep_pool_memory();
      cudaError_t e = cudaMallocAsync(&a.dev, bytes, s_);
      if (e == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();
        a.dev = nullptr;
        set_error("device allocation for a host grid failed");
        return STN_ENOMEM;
      }
      STN_CUDA_TRY(e);
      if (in) STN_CUDA_TRY(cudaMemcpyAsync(a.dev, a.user, bytes, cudaMemcpyHostToDevice, s_));
    }
    *dev = a.dev;
    return STN_OK;
  }
  // Copies host outputs back and, if any argument was host memory, waits.
  int finish() {
    for (int i = 0; i < n_; i++)
      if (a_[i].host && a_[i].copy_out)
        STN_CUDA_TRY(cudaMemcpyAsync(a_[i].user, a_[i].dev, a_[i].bytes, cudaMemcpyDeviceToHost, s_));
    if (any_host_) STN_CUDA_TRY(cudaStreamSynchronize(s_));
    return STN_OK;
  }
  bool any_host() const { return any_host_; }

 private:
  cudaStream_t s_;
  Arg a_[8];
  int n_ = 0;
  bool any_host_ = false;
};

// ----------------------------------------------------- repeated sweeps --
// Sweep loops over small grids are bound by launch cost, not by the kernels
// (a 64^3 sweep computes in ~3 us but a stream launch costs about as much
// again).  graph_repeat captures `body` -- an even number of ping-pong sweeps,
// so the iterate is back in its first buffer -- once into the body of a CUDA
// graph while node and lets the device repeat it `reps` times, counting in
// a workspace scalar.  The same kernels run in the same order, so the results
// are bitwise those of the host loop.
static int g_repeat_graph = 1;
constexpr i64 kRepeatMaxPoints = (i64)1 << 22;  // above this, launches are hidden by the kernels
constexpr i64 kRepeatBody = 16;                 // sweeps per repetition

static bool use_repeat_graph(const Grid& g, i64 iters) {
  return g_repeat_graph && iters >= kRepeatBody && g.interior() <= kRepeatMaxPoints;
}

template <typename Body>
static int graph_repeat(Workspace* ws, i64 reps, cudaStream_t s, Body&& body) {
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(ws->scalars + 12);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaSuccess;
  int rc = STN_OK;
  do {
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking))) break;
    if ((e = cudaGraphCreate(&graph, 0))) break;
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault))) break;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wn;
    if ((e = cudaGraphAddNode(&wn, graph, nullptr, nullptr, 0, &cp))) break;
    if ((e = cudaStreamBeginCaptureToGraph(cs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeRelaxed)))
      break;
    rc = body(cs);
    if (rc == STN_OK) rc = launch_count(ctr, reps, h, cs);
    cudaGraph_t captured = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &captured);
    if (rc != STN_OK) break;
    if ((e = e2)) break;
    if ((e = cudaGraphInstantiate(&exec, graph, 0))) break;
    if ((e = cudaMemsetAsync(ctr, 0, sizeof(*ctr), s))) break;
    if ((e = cudaGraphLaunch(exec, s))) break;
  } while (false);
  // an executable graph that is still running is freed when it completes
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (cs) cudaStreamDestroy(cs);
  if (rc != STN_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "graph-repeated sweeps");
  return STN_OK;
}

int tune_set_repeat_graph(int v) {
  if (v < 0 || v > 1) return STN_EINVAL;
  g_repeat_graph = v;
  return STN_OK;
}
int tune_get_repeat_graph() { return g_repeat_graph; }

// --------------------------------------------------------------- drivers --
// Resident launches on a stream keep their barrier words in workspace scalar
// 44 and their status word in scalar 6 (low 32 bits), so the synchronising
// calls that read scalars 0..6 see a timeout of an earlier resident sweep on
// the same stream and report it once.
static unsigned* resident_bar(Workspace* ws) { return reinterpret_cast<unsigned*>(ws->scalars + 44); }
static int* resident_status(Workspace* ws) { return reinterpret_cast<int*>(ws->scalars + 6); }
static int take_resident_status(Workspace* ws, cudaStream_t s) {
  int v = 0;
  memcpy(&v, ws->host_scalars + 6, sizeof(int));
  if (v == 0) return STN_OK;
  STN_CUDA_TRY(cudaMemsetAsync(ws->scalars + 6, 0, sizeof(double), s));
  STN_CUDA_TRY(cudaStreamSynchronize(s));
  ws->host_scalars[6] = 0.0;
  set_error("a resident sweep gave up waiting at a grid barrier");
  return STN_ETIMEOUT;
}

// The resident path runs only where nothing asks for a particular per-sweep
// kernel: no forced variant or chunk count (knob or autotuner trial) and no
// tuning-cache entry for the grid.
static bool resident_allowed(const Grid& g, size_t esize) {
  if (!resident3d_applicable(g, esize)) return false;
  if (star_force().variant >= 0 || star_force().chunks > 0 || tune_get_star_variant() >= 0 ||
      tune_get_star_chunks() > 0)
    return false;
  StarChoice tc;
  return !tune_cache_lookup(g, esize, &tc);
}

template <typename T>
static int sweep_impl(T* in, T* out, i64 nx, i64 ny, i64 nz, const double* coeffs, int radius,
                      i64 iters, void* stream) {
  clear_error();
  if (!in || !out) return einval("NULL grid");
  if (!coeffs) return einval("NULL coeffs");
  if (int rc = check_grid(nx, ny, nz, radius)) return rc;
  if (iters < 0) return einval("iters < 0");
  const Grid g{nx, ny, nz, radius};
  const size_t bytes = (size_t)g.count() * sizeof(T);
  if (overlap(in, out, bytes)) return einval("in and out overlap");
  cudaStream_t s = (cudaStream_t)stream;
  Stager st(s);
  T *din, *dout;
  if (int rc = st.add(in, bytes, true, iters > 1, (void**)&din)) return rc;
  if (int rc = st.add(out, bytes, false, true, (void**)&dout)) return rc;
  if (iters == 0) {
    STN_CUDA_TRY(cudaMemcpyAsync(dout, din, bytes, cudaMemcpyDeviceToDevice, s));
    return st.finish();
  }
  if (int rc = launch_copy_halo<T>(din, dout, g, s)) return rc;
  T* cur = din;
  T* nxt = dout;
  // temporal blocking: `depth` sweeps per pass while at least that many remain
  // precedence: the autotuner's trial, the knob, the tuning cache, single
  // sweeps (the built-in choice: measured faster on GB300 so far)
  int depth = star_force().depth > 0 ? star_force().depth : tune_get_temporal_depth();
  StarChoice tc;
  if (depth == 0 && tune_cache_lookup(g, sizeof(T), &tc) && tc.depth > 0) depth = tc.depth;
  if (depth == 0) depth = 1;
  depth = temporal_depth_supported(depth, sizeof(T), radius);
  star_last().depth = depth;
  i64 it = 0;
  if (depth > 1) {
    for (; it + depth <= iters; it += depth) {
      if (int rc = launch_temporal<T>(cur, nxt, g, coeffs, depth, s)) return rc;
      std::swap(cur, nxt);
    }
  }
  if constexpr (sizeof(T) == 8) {
    if (tune_get_double_word() && dw_applicable(g, coeffs, nullptr)) {
      // opt-in: every sweep in double-word float arithmetic (not bitwise)
      for (; it < iters; it++) {
        if (int rc = launch_star_dw(cur, nxt, g, coeffs, s)) return rc;
        std::swap(cur, nxt);
      }
    }
  }
  if (depth <= 1 && it < iters && iters >= 2 && resident_allowed(g, sizeof(T))) {
    // small grids: every sweep in one cooperative launch
    Workspace* ws;
    if (int rc = get_workspace(s, 0, 0, &ws)) return rc;
    if (int rc = launch_star_resident<T>(cur, nxt, nullptr, g, coeffs, iters, false, nullptr, nullptr,
                                         resident_bar(ws), resident_status(ws), s))
      return rc;
    if (iters % 2) std::swap(cur, nxt);
    it = iters;
  }
  if (depth <= 1 && it < iters && use_repeat_graph(g, iters)) {
    Workspace* ws;
    if (int rc = get_workspace(s, 0, 0, &ws)) return rc;
    const i64 reps = iters / kRepeatBody;
    int rc = graph_repeat(ws, reps, s, [&](cudaStream_t cs) -> int {
      for (i64 k = 0; k < kRepeatBody; k++)
        if (int r = launch_star<T>(k % 2 ? nxt : cur, nullptr, k % 2 ? cur : nxt, g, coeffs, kSweep, nullptr, cs))
          return r;
      return STN_OK;
    });
    if (rc) return rc;
    it = reps * kRepeatBody;
  }
  for (; it < iters; it++) {
    if (int rc = launch_star<T>(cur, nullptr, nxt, g, coeffs, kSweep, nullptr, s)) return rc;
    std::swap(cur, nxt);
  }
  if (cur != dout) STN_CUDA_TRY(cudaMemcpyAsync(dout, cur, bytes, cudaMemcpyDeviceToDevice, s));
  return st.finish();
}

template <typename T>
static int apply_impl(const T* u, const T* b, T* out, i64 nx, i64 ny, i64 nz, const double* coeffs,
                      int radius, void* stream) {
  clear_error();
  if (!u || !out) return einval("NULL grid");
  if (!coeffs) return einval("NULL coeffs");
  if (int rc = check_grid(nx, ny, nz, radius)) return rc;
  const Grid g{nx, ny, nz, radius};
  const size_t bytes = (size_t)g.count() * sizeof(T);
  if (overlap(u, out, bytes) || (b && overlap(b, out, bytes))) return einval("out overlaps an input");
  bool hu = false, ho = false, hb = false;
  if (int rc = classify(u, &hu)) return rc;
  if (int rc = classify(out, &ho)) return rc;
  if (b)
    if (int rc = classify(b, &hb)) return rc;
  if (hu || ho || hb) return einval("stencil_apply takes device grids only");
  return launch_star<T>(u, b, out, g, coeffs, kSweep, nullptr, (cudaStream_t)stream);
}

// Reads `n` device scalars of the workspace into its pinned mirror; waits.
static int read_scalars(Workspace* ws, int first, int n, cudaStream_t s) {
  STN_CUDA_TRY(cudaMemcpyAsync(ws->host_scalars + first, ws->scalars + first, n * sizeof(double),
                               cudaMemcpyDeviceToHost, s));
  STN_CUDA_TRY(cudaStreamSynchronize(s));
  return STN_OK;
}



template <typename T>
static int residual_impl(const T* u, const T* b, i64 nx, i64 ny, i64 nz, const double* coeffs,
                         int radius, double* norm_out, void* stream) {
  clear_error();
  if (!u) return einval("NULL grid");
  if (!coeffs || !norm_out) return einval("NULL coeffs or norm_out");
  if (int rc = check_grid(nx, ny, nz, radius)) return rc;
  const Grid g{nx, ny, nz, radius};
  const size_t bytes = (size_t)g.count() * sizeof(T);
  cudaStream_t s = (cudaStream_t)stream;
  Stager st(s);
  T *du, *db;
  if (int rc = st.add(u, bytes, true, false, (void**)&du)) return rc;
  if (int rc = st.add(b, bytes, true, false, (void**)&db)) return rc;
  const i64 nb = star_blocks(g, sizeof(T), du, db, nullptr);
  Workspace* ws;
  if (int rc = get_workspace(s, nb, 0, &ws)) return rc;
  i64 nl = 0;  // the launch's own partial count (its plan, checked against the workspace)
  if (int rc = launch_star<T>(du, db, nullptr, g, coeffs, kResidualOnly, ws->partials, s, ws->partials_cap, &nl))
    return rc;
  if (int rc = launch_finalize(ws->partials, nl, ws->scalars, nullptr, 0.0, s)) return rc;
  if (int rc = read_scalars(ws, 0, 7, s)) return rc;
  if (int rc = take_resident_status(ws, s)) return rc;
  *norm_out = ws->host_scalars[1];
  return st.finish();
}

// ------------------------------------------------------------------- 2-D --
static int check_grid2d(i64 nx, i64 ny, int r) {
  if (r != 1 && r != 2) return einval("radius must be 1 or 2");
  if (nx < 1 || ny < 1) return einval("interior extents must be >= 1");
  const i64 lim = (i64)1 << 28;
  if (nx > lim || ny > lim) return einval("extent too large");
  if ((double)(nx + 2 * r) * (double)(ny + 2 * r) > 9.0e15) return einval("grid too large");
  return STN_OK;
}

template <typename T>
static int sweep2d_impl(T* in, T* out, i64 nx, i64 ny, const double* coeffs, int radius, i64 iters,
                        void* stream) {
  clear_error();
  if (!in || !out) return einval("NULL grid");
  if (!coeffs) return einval("NULL coeffs");
  if (int rc = check_grid2d(nx, ny, radius)) return rc;
  if (iters < 0) return einval("iters < 0");
  const Grid2 g{nx, ny, radius};
  const size_t bytes = (size_t)g.count() * sizeof(T);
  if (overlap(in, out, bytes)) return einval("in and out overlap");
  cudaStream_t s = (cudaStream_t)stream;
  Stager st(s);
  T *din, *dout;
  const Plan2d p = plan_resident2d(g, sizeof(T));
  const bool resident = use_resident2d(p);
  if (int rc = st.add(in, bytes, true, iters > 1 && !resident, (void**)&din)) return rc;
  if (int rc = st.add(out, bytes, false, true, (void**)&dout)) return rc;
  if (iters == 0) {
    STN_CUDA_TRY(cudaMemcpyAsync(dout, din, bytes, cudaMemcpyDeviceToDevice, s));
  } else {
    Workspace* ws;
    if (int rc = get_workspace(s, 0, resident ? p.scratch : 0, &ws)) return rc;
    if (int rc = sweep2d_run<T>(din, dout, g, coeffs, iters, (unsigned char*)ws->grid, p, resident, din, s))
      return rc;
  }
  if (int rc = st.finish()) return rc;
  STN_CUDA_TRY(cudaStreamSynchronize(s));
  return STN_OK;
}

template <typename T>
static int residual2d_impl(const T* u, const T* b, i64 nx, i64 ny, const double* coeffs, int radius,
                           double* norm_out, void* stream) {
  clear_error();
  if (!u) return einval("NULL grid");
  if (!coeffs || !norm_out) return einval("NULL coeffs or norm_out");
  if (int rc = check_grid2d(nx, ny, radius)) return rc;
  const Grid2 g{nx, ny, radius};
  const size_t bytes = (size_t)g.count() * sizeof(T);
  cudaStream_t s = (cudaStream_t)stream;
  Stager st(s);
  T *du, *db;
  if (int rc = st.add(u, bytes, true, false, (void**)&du)) return rc;
  if (int rc = st.add(b, bytes, true, false, (void**)&db)) return rc;
  const i64 nb = star2d_blocks(g);
  Workspace* ws;
  if (int rc = get_workspace(s, nb, 0, &ws)) return rc;
  if (int rc = launch_star2d<T>(du, db, nullptr, g, coeffs, kResidualOnly, ws->partials, s)) return rc;
  if (int rc = launch_finalize(ws->partials, nb, ws->scalars, nullptr, 0.0, s)) return rc;
  if (int rc = read_scalars(ws, 0, 2, s)) return rc;
  *norm_out = ws->host_scalars[1];
  return st.finish();
}

// ------------------------------------------------------ sum, dotproduct --
static int vec_reduce_impl(const double* x, const double* y, i64 n, double* out, void* stream) {
  clear_error();
  if (!out) return einval("NULL out");
  if (n < 0) return einval("n < 0");
  if (n > ((i64)1 << 40)) return einval("n too large");
  if (n > 0 && !x) return einval("NULL array");
  if (((uintptr_t)x & 7) || ((uintptr_t)y & 7)) return einval("arrays must be 8-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  Stager st(s);
  const double *dx = nullptr, *dy = nullptr;
  if (n > 0) {
    if (int rc = st.add(x, (size_t)n * 8, true, false, (void**)&dx)) return rc;
    if (y)
      if (int rc = st.add(y, (size_t)n * 8, true, false, (void**)&dy)) return rc;
  }
  const i64 nb = vec_reduce_blocks(n);
  Workspace* ws;
  if (int rc = get_workspace(s, nb, 0, &ws)) return rc;
  if (int rc = launch_vec_reduce(dx, y ? dy : nullptr, n, ws->partials, s)) return rc;
  if (int rc = launch_finalize(ws->partials, nb, ws->scalars, nullptr, 0.0, s)) return rc;
  if (int rc = read_scalars(ws, 0, 1, s)) return rc;
  *out = ws->host_scalars[0];
  return st.finish();
}

// ------------------------------------------------------------- advection --
template <typename T>
static int advect_impl(const T* u, const T* v, const T* w, const T* const* q, int nq, T* const* s,
                       i64 nx, i64 ny, i64 nz, const double* c, void* stream) {
  clear_error();
  if (!u || !v || !w || !s) return einval("NULL velocity or output list");
  if (!c) return einval("NULL coefficients");
  for (int a = 0; a < 3; a++)
    if (!std::isfinite(c[a])) return einval("coefficients must be finite");
  if (int rc = check_grid(nx, ny, nz, 1)) return rc;
  const int nout = q ? nq : 3;
  if (q && (nq < 1 || nq > 6)) return einval("nq must be in 1..6");
  const Grid g{nx, ny, nz, 1};
  const size_t bytes = (size_t)g.count() * sizeof(T);
  std::vector<const void*> ins = {u, v, w};
  for (int m = 0; q && m < nq; m++) {
    if (!q[m]) return einval("NULL field");
    ins.push_back(q[m]);
  }
  for (int m = 0; m < nout; m++) {
    if (!s[m]) return einval("NULL output");
    for (const void* x : ins)
      if (overlap(s[m], x, bytes)) return einval("an output overlaps an input");
    for (int o = 0; o < m; o++)
      if (overlap(s[m], s[o], bytes)) return einval("outputs overlap");
  }
  std::vector<const void*> all = ins;
  for (int m = 0; m < nout; m++) all.push_back(s[m]);
  for (const void* x : all) {
    bool host = false;
    if (int rc = classify(x, &host)) return rc;
    if (host) return einval("advect takes device grids only");
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (!q) return launch_advect<T>(u, v, w, nullptr, 3, s, g, c, st);
  for (int g0 = 0; g0 < nq; g0 += 3) {
    const int n = std::min(3, nq - g0);
    if (int rc = launch_advect<T>(u, v, w, q + g0, n, s + g0, g, c, st)) return rc;
  }
  return STN_OK;
}

// Scalars layout used by the solvers: [0] sum, [1] norm, [2] rel, [3] flag,
// [4] max|rho|, [8] rhs sum of squares, [9] rhs norm.
template <typename Step>
static int solve_loop(Workspace* ws, i64 max_iters, i64 check_every, i64 nparts, double tol,
                      cudaStream_t s, Step&& step, i64* iters_out, double* rel_out, double* res_out,
                      int* status) {
  i64 it = 0;
  double rel = INFINITY, res = INFINITY;
  *status = STN_NOT_CONVERGED;
  while (it < max_iters) {
    i64 group = check_every < max_iters - it ? check_every : max_iters - it;
    for (i64 gi = 0; gi < group; gi++)
      if (int rc = step(it + gi, gi == group - 1)) return rc;
    it += group;
    if (int rc = launch_finalize(ws->partials, nparts, ws->scalars, ws->scalars + 9, tol, s)) return rc;
    if (int rc = read_scalars(ws, 0, 4, s)) return rc;
    res = ws->host_scalars[1];
    rel = ws->host_scalars[2];
    if (ws->host_scalars[3] != 0.0) {
      *status = STN_OK;
      break;
    }
  }
  *iters_out = it;
  *rel_out = rel;
  *res_out = res;
  return STN_OK;
}

template <typename T>
static int rhs_norm(Workspace* ws, const T* f, const Grid& g, cudaStream_t s, double* out) {
  i64 np = 0;
  if (f) {
    if (int rc = launch_interior_sumsq<T>(f, g, ws->partials, &np, s)) return rc;
    if (int rc = launch_finalize(ws->partials, np, ws->scalars + 8, nullptr, 0.0, s)) return rc;
  } else {
    STN_CUDA_TRY(cudaMemsetAsync(ws->scalars + 8, 0, 2 * sizeof(double), s));
  }
  if (int rc = read_scalars(ws, 8, 2, s)) return rc;
  *out = ws->host_scalars[9];
  return STN_OK;
}

static int g_solve_graph = 1;
int tune_set_solve_graph(int v) {
  if (v < 0 || v > 1) return STN_EINVAL;
  g_solve_graph = v;
  return STN_OK;
}
int tune_get_solve_graph() { return g_solve_graph; }

// Runs full groups of `group` sweeps inside one CUDA graph: a while node whose
// body is the group's sweeps (the last one fused with the residual), the
// device-side decision kernel and, for an odd group, a copy that brings the
// iterate back to `a`.  Stops on convergence or when the next group would
// pass max_full.  On return *it_out sweeps are done (a multiple of group) and
// the iterate is in `a`.  The decision kernel writes its scalars at `dst`
// (dst[9] holds the scale of the relative residual); `dst` lies in the
// workspace's scalars.
template <typename T>
static int graph_groups(T* a, T* bgrid, const T* db, const Grid& g, const double* coeffs, Workspace* ws,
                        double* dst, double tol, i64 group, i64 max_full, cudaStream_t s, i64* it_out,
                        bool* conv_out) {
  const size_t bytes = (size_t)g.count() * sizeof(T);
  cudaGraph_t graph = nullptr, body = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs = nullptr;
  cudaError_t e;
  int rc = STN_OK;
  const int first = (int)(dst - ws->scalars);
  do {
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking))) break;
    if ((e = cudaGraphCreate(&graph, 0))) break;
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault))) break;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wn;
    if ((e = cudaGraphAddNode(&wn, graph, nullptr, nullptr, 0, &cp))) break;
    body = cp.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed))) break;
    T* cur = a;
    T* nxt = bgrid;
    i64 nl = 0;  // partials the group's last (residual) sweep writes
    if (resident_allowed(g, sizeof(T)) && resident3d_blocks(g) <= ws->partials_cap) {
      // small grids: the group's sweeps in one cooperative launch
      rc = launch_star_resident<T>(cur, nxt, db, g, coeffs, group, true, ws->partials, &nl, resident_bar(ws),
                                   resident_status(ws), cs);
      if (group % 2) std::swap(cur, nxt);
    } else {
      for (i64 k = 0; k < group && rc == STN_OK; k++) {
        rc = launch_star<T>(cur, db, nxt, g, coeffs, k == group - 1 ? kSweepResidual : kSweep, ws->partials, cs,
                            ws->partials_cap, &nl);
        std::swap(cur, nxt);
      }
    }
    if (rc == STN_OK) rc = launch_decide(ws->partials, nl, dst, tol, group, max_full, h, cs);
    if (rc == STN_OK && cur != a) e = cudaMemcpyAsync(a, cur, bytes, cudaMemcpyDeviceToDevice, cs);
    cudaGraph_t captured = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &captured);
    if (rc != STN_OK) break;
    if (e != cudaSuccess) break;
    if ((e = e2)) break;
    if ((e = cudaGraphInstantiate(&exec, graph, 0))) break;
    if ((e = cudaMemsetAsync(dst + 5, 0, sizeof(double), s))) break;
    if ((e = cudaGraphLaunch(exec, s))) break;
    if ((rc = read_scalars(ws, first, 6, s))) break;
    if ((rc = read_scalars(ws, 6, 1, s))) break;
    if ((rc = take_resident_status(ws, s))) break;
    *it_out = (i64)ws->host_scalars[first + 5];
    *conv_out = ws->host_scalars[first + 3] != 0.0;
  } while (false);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (cs) cudaStreamDestroy(cs);
  if (rc != STN_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "graph-driven solve");
  return STN_OK;
}

// The double Jacobi solve of one device problem (tmp: a scratch grid of the
// problem's size); synchronises `s`.  Shared by jacobi_solve_f64 and the
// stream-pool server.
int solve_jacobi_core(const double* db, double* du, double* tmp, const Grid& g, const double* coeffs, double tol,
                      i64 max_iters, i64 check_every, stn_solve_info* info, cudaStream_t s) {
  const size_t bytes = (size_t)g.count() * sizeof(double);
  Workspace* ws;
  if (int rc = get_workspace(s, plan_star(g, kStarScalar, 8).blocks() + plan_star(g, kStarColumn, 8).blocks() + plan_star(g, kStarPlane2, 8).blocks() + plan_star(g, kStarStaged, 8).blocks(), 0, &ws))
    return rc;
  const i64 nb_sweep = star_blocks(g, sizeof(double), du, db, tmp);
  if (int rc = launch_copy_halo<double>(du, tmp, g, s)) return rc;
  double bn = 0.0;
  if (int rc = rhs_norm<double>(ws, db, g, s, &bn)) return rc;
  i64 done = 0;
  bool conv = false;
  double rel = 0, res = 0;
  int status = STN_NOT_CONVERGED;
  const i64 max_full = (max_iters / check_every) * check_every;
  if (g_solve_graph && max_full >= check_every) {
    if (int rc = graph_groups<double>(du, tmp, db, g, coeffs, ws, ws->scalars, tol, check_every, max_full, s, &done,
                                      &conv))
      return rc;
    res = ws->host_scalars[1];
    rel = ws->host_scalars[2];
    if (conv) status = STN_OK;
  }
  double* cur = du;
  double* nxt = tmp;
  if (!conv && done < max_iters) {
    auto step = [&](i64, bool last) -> int {
      int rc = launch_star<double>(cur, db, nxt, g, coeffs, last ? kSweepResidual : kSweep, ws->partials, s,
                                   ws->partials_cap);
      std::swap(cur, nxt);
      return rc;
    };
    i64 more = 0;
    if (int rc = solve_loop(ws, max_iters - done, check_every, nb_sweep, tol, s, step, &more, &rel, &res, &status))
      return rc;
    done += more;
  }
  if (max_iters == 0) {
    // no sweep: measure the residual of the initial guess only
    i64 nl = 0;
    if (int rc = launch_star<double>(du, db, nullptr, g, coeffs, kResidualOnly, ws->partials, s, ws->partials_cap, &nl))
      return rc;
    if (int rc = launch_finalize(ws->partials, nl, ws->scalars, ws->scalars + 9, tol, s)) return rc;
    if (int rc = read_scalars(ws, 0, 4, s)) return rc;
    res = ws->host_scalars[1];
    rel = ws->host_scalars[2];
    status = ws->host_scalars[3] != 0.0 ? STN_OK : STN_NOT_CONVERGED;
  }
  if (cur != du) STN_CUDA_TRY(cudaMemcpyAsync(du, cur, bytes, cudaMemcpyDeviceToDevice, s));
  STN_CUDA_TRY(cudaStreamSynchronize(s));
  if (info) {
    info->iters = done;
    info->outer = 0;
    info->rel_res = rel;
    info->res_norm = res;
    info->rhs_norm = bn;
    info->status = status;
  }
  return status;
}

static int jacobi_impl(const double* rhs, double* u, i64 nx, i64 ny, i64 nz, const double* coeffs,
                       int radius, double tol, i64 max_iters, i64 check_every, stn_solve_info* info,
                       void* stream) {
  clear_error();
  if (!u) return einval("NULL grid");
  if (!coeffs) return einval("NULL coeffs");
  if (int rc = check_grid(nx, ny, nz, radius)) return rc;
  if (!(tol >= 0.0)) return einval("tol must be >= 0");
  if (max_iters < 0) return einval("max_iters < 0");
  if (check_every < 1) return einval("check_every < 1");
  const Grid g{nx, ny, nz, radius};
  const size_t bytes = (size_t)g.count() * sizeof(double);
  if (rhs && overlap(rhs, u, bytes)) return einval("rhs and u overlap");
  cudaStream_t s = (cudaStream_t)stream;
  Stager st(s);
  double *du, *db;
  if (int rc = st.add(u, bytes, true, true, (void**)&du)) return rc;
  if (int rc = st.add(rhs, bytes, true, false, (void**)&db)) return rc;
  Workspace* ws;
  if (int rc = get_workspace(s, 0, bytes, &ws)) return rc;
  stn_solve_info loc{};
  const int status = solve_jacobi_core(db, du, (double*)ws->grid, g, coeffs, tol, max_iters, check_every, &loc, s);
  if (status < 0) return status;
  if (int rc = st.finish()) return rc;
  if (info) *info = loc;
  return status;
}

// ------------------------------------------ direct refinement (one problem) --
// The constant-coefficient refinement of jacobi_solve_refined_f64 computed
// with the full-grid kernels of the single-problem sweeps, step for step the
// oracle's refinement:
//   t = S u + b (double sweep with the fused sum of (t - u)^2), stop when
//   ||t - u|| <= tol * ||b||;  s = max |t - u|;  r32 = float((t - u) / s);
//   float sweeps e <- S e + r32 from e = 0 (coefficients rounded to float):
//   inner_sweeps of them, or, with inner_tol > 0, groups of check_every until
//   a group's last sweep changed e by <= inner_tol * ||r32||;  u += s * e.
// Small grids run their inner loops as device-repeated CUDA graphs (the
// decision on the device, one host wait per outer step).  Workspace scalars:
// [0..3] outer norm, [4] s, [8..9] ||b||, [12] graph counter, [16..25] inner
// decisions with [25] = ||r32||.
static int g_refined_engine = 1;  // 1: direct full-grid kernels; 0: the scheduler, one problem
int tune_set_refined_engine(int v) {
  if (v < 0 || v > 1) return STN_EINVAL;
  g_refined_engine = v;
  return STN_OK;
}
int tune_get_refined_engine() { return g_refined_engine; }

int solve_refined_core(const double* db, double* du, double* t, float* f32, const Grid& g, const double* coeffs,
                       double tol, i64 inner_sweeps, double inner_tol, i64 check_every, i64 max_outer,
                       stn_solve_info* info, cudaStream_t s) {
  const i64 n = g.count();
  const size_t b32 = (size_t)n * sizeof(float);
  i64 cap = 2 * 152 * 16;  // interior reductions: one partial per block of at most 152 * 16
  for (int v = 0; v < 4; v++) cap += plan_star(g, v, 8).blocks() + plan_star(g, v, 4).blocks();
  Workspace* ws;
  if (int rc = get_workspace(s, cap, 0, &ws)) return rc;
  float* r32 = f32;
  float* e = r32 + n;
  float* e2 = e + n;
  // the correction's halo is zero (homogeneous Dirichlet): zero both buffers once
  STN_CUDA_TRY(cudaMemsetAsync(e, 0, 2 * b32, s));
  double bn = 0.0;
  if (int rc = rhs_norm<double>(ws, db, g, s, &bn)) return rc;
  i64 outer = 0, sweeps = 0;
  double rel = INFINITY, res = INFINITY;
  int status = STN_NOT_CONVERGED;
  for (;;) {
    i64 nl = 0, nm = 0;
    if (int rc = launch_star<double>(du, db, t, g, coeffs, kSweepResidual, ws->partials, s, ws->partials_cap, &nl))
      return rc;
    if (int rc = launch_finalize(ws->partials, nl, ws->scalars, ws->scalars + 9, tol, s)) return rc;
    if (int rc = launch_diff_max(t, du, g, ws->partials, &nm, s)) return rc;
    if (int rc = launch_max_finalize(ws->partials, nm, ws->scalars + 4, s)) return rc;
    if (int rc = read_scalars(ws, 0, 7, s)) return rc;
    if (int rc = take_resident_status(ws, s)) return rc;  // the previous step's resident sweeps ran whole
    res = ws->host_scalars[1];
    rel = ws->host_scalars[2];
    if (ws->host_scalars[3] != 0.0) {
      status = STN_OK;
      break;
    }
    if (outer >= max_outer || ws->host_scalars[4] == 0.0) break;
    if (int rc = launch_refine_scale_diff(t, du, r32, g, ws->scalars + 4, s)) return rc;
    STN_CUDA_TRY(cudaMemsetAsync(e, 0, b32, s));  // e = 0 (e2's interior is overwritten first)
    float* cur = e;
    float* nxt = e2;
    i64 done = 0;
    if (inner_tol > 0.0) {
      // groups of check_every sweeps, the last fused with ||e' - e||, until it
      // is <= inner_tol * ||r32|| or inner_sweeps are done
      i64 np = 0;
      if (int rc = launch_interior_sumsq<float>(r32, g, ws->partials, &np, s)) return rc;
      if (int rc = launch_finalize(ws->partials, np, ws->scalars + 24, nullptr, 0.0, s)) return rc;
      const i64 max_full = (inner_sweeps / check_every) * check_every;
      bool conv = false;
      if (g_solve_graph && max_full >= check_every) {
        if (int rc = graph_groups<float>(cur, nxt, r32, g, coeffs, ws, ws->scalars + 16, inner_tol, check_every,
                                         max_full, s, &done, &conv))
          return rc;
      }
      // host-driven groups: without graphs, or a last partial group
      while (!conv && done < inner_sweeps) {
        const i64 grp = std::min(check_every, inner_sweeps - done);
        i64 gl = 0;
        for (i64 k = 0; k < grp; k++) {
          if (int rc = launch_star<float>(cur, r32, nxt, g, coeffs, k == grp - 1 ? kSweepResidual : kSweep,
                                          ws->partials, s, ws->partials_cap, &gl))
            return rc;
          std::swap(cur, nxt);
        }
        done += grp;
        if (int rc = launch_finalize(ws->partials, gl, ws->scalars + 16, ws->scalars + 25, inner_tol, s)) return rc;
        if (int rc = read_scalars(ws, 16, 4, s)) return rc;
        conv = ws->host_scalars[19] != 0.0;
      }
    } else {
      if (inner_sweeps >= 2 && resident_allowed(g, sizeof(float))) {
        if (int rc = launch_star_resident<float>(cur, nxt, r32, g, coeffs, inner_sweeps, false, nullptr, nullptr,
                                                 resident_bar(ws), resident_status(ws), s))
          return rc;
        if (inner_sweeps % 2) std::swap(cur, nxt);
        done = inner_sweeps;
      } else if (use_repeat_graph(g, inner_sweeps)) {
        const i64 reps = inner_sweeps / kRepeatBody;
        int rc = graph_repeat(ws, reps, s, [&](cudaStream_t cs) -> int {
          for (i64 k = 0; k < kRepeatBody; k++)
            if (int r = launch_star<float>(k % 2 ? nxt : cur, r32, k % 2 ? cur : nxt, g, coeffs, kSweep, nullptr,
                                           cs))
              return r;
          return STN_OK;
        });
        if (rc) return rc;
        done = reps * kRepeatBody;
      }
      for (; done < inner_sweeps; done++) {
        if (int rc = launch_star<float>(cur, r32, nxt, g, coeffs, kSweep, nullptr, s)) return rc;
        std::swap(cur, nxt);
      }
    }
    sweeps += done;
    if (int rc = launch_refine_update(du, cur, g, ws->scalars + 4, s)) return rc;
    outer++;
  }
  STN_CUDA_TRY(cudaStreamSynchronize(s));
  if (info) {
    info->iters = sweeps;
    info->outer = outer;
    info->rel_res = rel;
    info->res_norm = res;
    info->rhs_norm = bn;
    info->status = status;
  }
  return status;
}

static int refined_direct_impl(const double* rhs, double* u, i64 nx, i64 ny, i64 nz, const double* coeffs,
                               int radius, double tol, i64 inner_sweeps, double inner_tol, i64 check_every,
                               i64 max_outer, stn_solve_info* info, void* stream) {
  clear_error();
  if (!u) return einval("NULL grid");
  if (!coeffs) return einval("NULL coeffs");
  if (int rc = check_grid(nx, ny, nz, radius)) return rc;
  if (!(tol >= 0.0)) return einval("tol must be >= 0");
  if (inner_sweeps < 0 || max_outer < 0) return einval("inner_sweeps or max_outer < 0");
  if (check_every < 1) return einval("check_every < 1");
  if (!(inner_tol >= 0.0)) return einval("inner_tol must be >= 0");
  const Grid g{nx, ny, nz, radius};
  const size_t bytes = (size_t)g.count() * sizeof(double);
  if (rhs && overlap(rhs, u, bytes)) return einval("rhs and u overlap");
  cudaStream_t s = (cudaStream_t)stream;
  Stager st(s);
  double *du, *db;
  if (int rc = st.add(u, bytes, true, true, (void**)&du)) return rc;
  if (int rc = st.add(rhs, bytes, true, false, (void**)&db)) return rc;
  const i64 n = g.count();
  Workspace* ws;
  if (int rc = get_workspace(s, 0, (size_t)n * sizeof(double), &ws)) return rc;
  if (int rc = ensure_grid2(ws, 3 * (size_t)n * sizeof(float))) return rc;
  stn_solve_info loc{};
  const int status = solve_refined_core(db, du, (double*)ws->grid, (float*)ws->grid2, g, coeffs, tol, inner_sweeps,
                                        inner_tol, check_every, max_outer, &loc, s);
  if (status < 0) return status;
  if (int rc = st.finish()) return rc;
  if (info) *info = loc;
  return status;
}

// ----------------------------------------------------- variable coefficient --
template <typename T>
static int var_sweep_impl(T* in, T* out, const T* a, const T* f, i64 nx, i64 ny, i64 nz,
                          const double* w, int radius, i64 iters, void* stream) {
  clear_error();
  if (!in || !out || !a || !f) return einval("NULL grid");
  if (!w) return einval("NULL weights");
  if (int rc = check_grid(nx, ny, nz, radius)) return rc;
  if (iters < 0) return einval("iters < 0");
  const Grid g{nx, ny, nz, radius};
  const size_t bytes = (size_t)g.count() * sizeof(T);
  if (overlap(in, out, bytes)) return einval("in and out overlap");
  if (overlap(a, out, bytes) || overlap(f, out, bytes) || overlap(a, in, bytes) || overlap(f, in, bytes))
    return einval("coefficient or source grid overlaps an iterate");
  cudaStream_t s = (cudaStream_t)stream;
  Stager st(s);
  T *din, *dout, *da, *df;
  if (int rc = st.add(in, bytes, true, iters > 1, (void**)&din)) return rc;
  if (int rc = st.add(out, bytes, false, true, (void**)&dout)) return rc;
  if (int rc = st.add(a, bytes, true, false, (void**)&da)) return rc;
  if (int rc = st.add(f, bytes, true, false, (void**)&df)) return rc;
  if (iters == 0) {
    STN_CUDA_TRY(cudaMemcpyAsync(dout, din, bytes, cudaMemcpyDeviceToDevice, s));
    return st.finish();
  }
  if (int rc = launch_copy_halo<T>(din, dout, g, s)) return rc;
  T* cur = din;
  T* nxt = dout;
  i64 it = 0;
  if (use_repeat_graph(g, iters)) {
    Workspace* ws;
    if (int rc = get_workspace(s, 0, 0, &ws)) return rc;
    const i64 reps = iters / kRepeatBody;
    int rc = graph_repeat(ws, reps, s, [&](cudaStream_t cs) -> int {
      for (i64 k = 0; k < kRepeatBody; k++)
        if (int r = launch_var<T>(k % 2 ? nxt : cur, da, df, k % 2 ? cur : nxt, g, w, kVarSweep, nullptr,
                                  nullptr, cs))
          return r;
      return STN_OK;
    });
    if (rc) return rc;
    it = reps * kRepeatBody;
  }
  for (; it < iters; it++) {
    if (int rc = launch_var<T>(cur, da, df, nxt, g, w, kVarSweep, nullptr, nullptr, s)) return rc;
    std::swap(cur, nxt);
  }
  if (cur != dout) STN_CUDA_TRY(cudaMemcpyAsync(dout, cur, bytes, cudaMemcpyDeviceToDevice, s));
  return st.finish();
}

static int var_apply_impl(const double* u, const double* a, double* out, i64 nx, i64 ny, i64 nz,
                          const double* w, int radius, void* stream) {
  clear_error();
  if (!u || !a || !out) return einval("NULL grid");
  if (!w) return einval("NULL weights");
  if (int rc = check_grid(nx, ny, nz, radius)) return rc;
  const Grid g{nx, ny, nz, radius};
  const size_t bytes = (size_t)g.count() * sizeof(double);
  if (overlap(u, out, bytes) || overlap(a, out, bytes)) return einval("out overlaps an input");
  cudaStream_t s = (cudaStream_t)stream;
  Stager st(s);
  double *du, *da, *dout;
  if (int rc = st.add(u, bytes, true, false, (void**)&du)) return rc;
  if (int rc = st.add(a, bytes, true, false, (void**)&da)) return rc;
  if (int rc = st.add(out, bytes, true, true, (void**)&dout)) return rc;
  if (int rc = launch_var<double>(du, da, nullptr, dout, g, w, kVarApply, nullptr, nullptr, s)) return rc;
  return st.finish();
}

// A bounded wait of the TMA-staged float sweep that ran out (never expected:
// the copies it waits for are its own) leaves a status word set; the
// synchronising variable-coefficient calls report it once, as STN_ETIMEOUT.
static int check_var_tma() {
  int st = 0;
  if (int rc = var_tma_status(true, &st)) return rc;
  if (st != 0) {
    set_error("a TMA-staged variable-coefficient sweep gave up waiting for its tile copies");
    return STN_ETIMEOUT;
  }
  return STN_OK;
}

static int var_residual_impl(const double* u, const double* a, const double* f, i64 nx, i64 ny,
                             i64 nz, const double* w, int radius, double* norm_out, void* stream) {
  clear_error();
  if (!u || !a || !f) return einval("NULL grid");
  if (!w || !norm_out) return einval("NULL weights or norm_out");
  if (int rc = check_grid(nx, ny, nz, radius)) return rc;
  const Grid g{nx, ny, nz, radius};
  const size_t bytes = (size_t)g.count() * sizeof(double);
  cudaStream_t s = (cudaStream_t)stream;
  Stager st(s);
  double *du, *da, *df;
  if (int rc = st.add(u, bytes, true, false, (void**)&du)) return rc;
  if (int rc = st.add(a, bytes, true, false, (void**)&da)) return rc;
  if (int rc = st.add(f, bytes, true, false, (void**)&df)) return rc;
  const ZPlan p = plan_var(g, 8);
  Workspace* ws;
  if (int rc = get_workspace(s, p.blocks(), 0, &ws)) return rc;
  if (int rc = launch_var<double>(du, da, df, nullptr, g, w, kVarResidual, ws->partials, nullptr, s)) return rc;
  if (int rc = launch_finalize(ws->partials, p.blocks(), ws->scalars, nullptr, 0.0, s)) return rc;
  if (int rc = read_scalars(ws, 0, 2, s)) return rc;
  *norm_out = ws->host_scalars[1];
  if (int rc = check_var_tma()) return rc;
  return st.finish();
}

static int var_jacobi_impl(const double* a, const double* f, double* u, i64 nx, i64 ny, i64 nz,
                           const double* w, int radius, double tol, i64 max_iters, i64 check_every,
                           stn_solve_info* info, void* stream) {
  clear_error();
  if (!u || !a || !f) return einval("NULL grid");
  if (!w) return einval("NULL weights");
  if (int rc = check_grid(nx, ny, nz, radius)) return rc;
  if (!(tol >= 0.0)) return einval("tol must be >= 0");
  if (max_iters < 0) return einval("max_iters < 0");
  if (check_every < 1) return einval("check_every < 1");
  const Grid g{nx, ny, nz, radius};
  const size_t bytes = (size_t)g.count() * sizeof(double);
  if (overlap(a, u, bytes) || overlap(f, u, bytes)) return einval("u overlaps a or f");
  cudaStream_t s = (cudaStream_t)stream;
  Stager st(s);
  double *du, *da, *df;
  if (int rc = st.add(u, bytes, true, true, (void**)&du)) return rc;
  if (int rc = st.add(a, bytes, true, false, (void**)&da)) return rc;
  if (int rc = st.add(f, bytes, true, false, (void**)&df)) return rc;
  const ZPlan p = plan_var(g, 8);
  Workspace* ws;
  if (int rc = get_workspace(s, p.blocks(), bytes, &ws)) return rc;
  double* tmp = (double*)ws->grid;
  if (int rc = launch_copy_halo<double>(du, tmp, g, s)) return rc;
  double fn = 0.0;
  if (int rc = rhs_norm<double>(ws, df, g, s, &fn)) return rc;
  double* cur = du;
  double* nxt = tmp;
  auto step = [&](i64, bool last) -> int {
    if (last) {
      int rc = launch_var<double>(cur, da, df, nullptr, g, w, kVarResidual, ws->partials, nullptr, s);
      if (rc) return rc;
    }
    int rc = launch_var<double>(cur, da, df, nxt, g, w, kVarSweep, nullptr, nullptr, s);
    std::swap(cur, nxt);
    return rc;
  };
  i64 iters = 0;
  double rel = 0, res = 0;
  int status = STN_NOT_CONVERGED;
  if (int rc = solve_loop(ws, max_iters, check_every, p.blocks(), tol, s, step, &iters, &rel, &res, &status))
    return rc;
  if (cur != du) STN_CUDA_TRY(cudaMemcpyAsync(du, cur, bytes, cudaMemcpyDeviceToDevice, s));
  if (int rc = st.finish()) return rc;
  STN_CUDA_TRY(cudaStreamSynchronize(s));
  if (info) {
    info->iters = iters;
    info->outer = 0;
    info->rel_res = rel;
    info->res_norm = res;
    info->rhs_norm = fn;
    info->status = status;
  }
  return status;
}

static int refined_impl(const double* a, const double* f, double* u, i64 nx, i64 ny, i64 nz,
                        const double* w, int radius, double tol, i64 inner_sweeps, i64 max_outer,
                        stn_solve_info* info, void* stream) {
  clear_error();
  if (!u || !a || !f) return einval("NULL grid");
  if (!w) return einval("NULL weights");
  if (int rc = check_grid(nx, ny, nz, radius)) return rc;
  if (!(tol >= 0.0)) return einval("tol must be >= 0");
  if (inner_sweeps < 0 || max_outer < 0) return einval("inner_sweeps or max_outer < 0");
  const Grid g{nx, ny, nz, radius};
  const i64 n = g.count();
  const size_t bytes = (size_t)n * sizeof(double);
  if (overlap(a, u, bytes) || overlap(f, u, bytes)) return einval("u overlaps a or f");
  cudaStream_t s = (cudaStream_t)stream;
  Stager st(s);
  double *du, *da, *df;
  if (int rc = st.add(u, bytes, true, true, (void**)&du)) return rc;
  if (int rc = st.add(a, bytes, true, false, (void**)&da)) return rc;
  if (int rc = st.add(f, bytes, true, false, (void**)&df)) return rc;
  const ZPlan p = plan_var(g, 8);
  Workspace* ws;
  // partials: sums in [0, nb), maxima in [nb, 2nb)
  if (int rc = get_workspace(s, 2 * p.blocks(), bytes, &ws)) return rc;
  const size_t b32 = (size_t)n * sizeof(float);
  if (int rc = ensure_grid2(ws, 4 * b32)) return rc;
  double* rho = (double*)ws->grid;
  float* a32 = (float*)ws->grid2;
  float* r32 = a32 + n;
  float* e = r32 + n;
  float* e2 = e + n;
  if (int rc = launch_convert<double, float>(da, a32, n, s)) return rc;
  STN_CUDA_TRY(cudaMemsetAsync(r32, 0, 3 * b32, s));
  double fn = 0.0;
  if (int rc = rhs_norm<double>(ws, df, g, s, &fn)) return rc;
  double* pmax = ws->partials + p.blocks();
  i64 outer = 0, sweeps = 0;
  double rel = INFINITY, res = INFINITY;
  int status = STN_NOT_CONVERGED;
  for (;;) {
    if (int rc = launch_var<double>(du, da, df, rho, g, w, kVarRefine, ws->partials, pmax, s)) return rc;
    if (int rc = launch_finalize(ws->partials, p.blocks(), ws->scalars, ws->scalars + 9, tol, s)) return rc;
    if (int rc = launch_max_finalize(pmax, p.blocks(), ws->scalars + 4, s)) return rc;
    if (int rc = read_scalars(ws, 0, 5, s)) return rc;
    if (int rc = check_var_tma()) return rc;  // the float sweeps of the last step ran whole
    res = ws->host_scalars[1];
    rel = ws->host_scalars[2];
    if (ws->host_scalars[3] != 0.0) {
      status = STN_OK;
      break;
    }
    if (outer >= max_outer || ws->host_scalars[4] == 0.0) break;
    if (int rc = launch_refine_scale(rho, r32, g, ws->scalars + 4, s)) return rc;
    STN_CUDA_TRY(cudaMemsetAsync(e, 0, 2 * b32, s));
    float* cur = e;
    float* nxt = e2;
    i64 it = 0;
    if (use_repeat_graph(g, inner_sweeps)) {
      const i64 reps = inner_sweeps / kRepeatBody;
      int rc = graph_repeat(ws, reps, s, [&](cudaStream_t cs) -> int {
        for (i64 k = 0; k < kRepeatBody; k++)
          if (int r = launch_var<float>(k % 2 ? nxt : cur, a32, r32, k % 2 ? cur : nxt, g, w, kVarSweep,
                                        nullptr, nullptr, cs))
            return r;
        return STN_OK;
      });
      if (rc) return rc;
      it = reps * kRepeatBody;
    }
    for (; it < inner_sweeps; it++) {
      if (int rc = launch_var<float>(cur, a32, r32, nxt, g, w, kVarSweep, nullptr, nullptr, s)) return rc;
      std::swap(cur, nxt);
    }
    sweeps += inner_sweeps;
    if (int rc = launch_refine_update(du, cur, g, ws->scalars + 4, s)) return rc;
    outer++;
  }
  if (int rc = st.finish()) return rc;
  STN_CUDA_TRY(cudaStreamSynchronize(s));
  if (info) {
    info->iters = sweeps;
    info->outer = outer;
    info->rel_res = rel;
    info->res_norm = res;
    info->rhs_norm = fn;
    info->status = status;
  }
  return status;
}

static int batch_impl(const stn_problem* probs, i64 count, const double* coeffs, int radius,
                      double tol, i64 iters, i64 check_every, double inner_tol, i64 max_outer,
                      bool refined, stn_solve_info* infos, void* stream) {
  clear_error();
  if (count < 0) return einval("count < 0");
  if (count > 0 && !probs) return einval("NULL problem array");
  if (!coeffs) return einval("NULL coeffs");
  if (!(tol >= 0.0)) return einval("tol must be >= 0");
  if (iters < 0) return einval("iteration limit < 0");
  if (check_every < 1) return einval("check_every < 1");
  if (!(inner_tol >= 0.0)) return einval("inner_tol must be >= 0");
  if (max_outer < 0) return einval("max_outer < 0");
  if (count > (1 << 30)) return einval("too many problems");
  // the solvers' scratch (a double grid per problem, three float grids when
  // refined, one partial per work unit), bounded before any size arithmetic
  double scratch = 0.0;
  for (i64 i = 0; i < count; i++) {
    const stn_problem& p = probs[i];
    if (int rc = check_grid(p.nx, p.ny, p.nz, radius)) return rc;
    if (p.nx > (1 << 20) || p.ny > (1 << 20) || p.nz > (1 << 20))
      return einval("batched problem extent too large");
    if (!p.u) return einval("NULL problem grid");
    const i64 units = sched_units(p.nx, p.ny, p.nz);
    if (units > kMaxPassUnits) return einval("batched problem needs more than 2^22 work units per pass");
    const size_t bytes = (size_t)Grid{p.nx, p.ny, p.nz, radius}.count() * sizeof(double);
    if (p.rhs && overlap(p.rhs, p.u, bytes)) return einval("problem rhs overlaps its u");
    scratch += (double)Grid{p.nx, p.ny, p.nz, radius}.count() * (refined ? 20.0 : 8.0) + 8.0 * (double)units;
  }
  if (scratch > 1.0e15) {
    set_error("batched problems need more scratch than any device holds");
    return STN_ENOMEM;
  }
  if (count == 0) return STN_OK;
  for (i64 i = 0; i < count; i++) {
    bool h = false;
    if (int rc = classify(probs[i].u, &h)) return rc;
    if (!h && probs[i].rhs)
      if (int rc = classify(probs[i].rhs, &h)) return rc;
    if (h) return einval("batched problems take device grids only");
  }
  return batched_solve(probs, count, coeffs, radius, tol, iters, check_every, inner_tol, max_outer,
                       refined, infos, (cudaStream_t)stream);
}

}  // namespace stn

// ===================================================================== ABI ==
using namespace stn;

extern "C" {

const char* stencil_last_error(void) { return g_err.c_str(); }

const char* stencil_version(void) { return "libstencil 0.1 (sm_103a)"; }

int stencil_tune_set(const char* knob, int64_t value) {
  clear_error();
  if (!knob) return einval("NULL knob");
  if (strcmp(knob, "star_variant") == 0) {
    if (tune_set_star_variant((int)value) != STN_OK) return einval("star_variant must be -1, 0, 1, 2 or 3");
    return STN_OK;
  }
  if (strcmp(knob, "temporal_depth") == 0) {
    if (tune_set_temporal_depth((int)value) != STN_OK) return einval("temporal_depth must be 0..4");
    return STN_OK;
  }
  if (strcmp(knob, "star_chunks") == 0) {
    if (tune_set_star_chunks((int)value) != STN_OK) return einval("star_chunks must be in [0, 65535]");
    return STN_OK;
  }
  if (strcmp(knob, "sweep2d_resident") == 0) {
    if (tune_set_resident2d((int)value) != STN_OK) return einval("sweep2d_resident must be -1, 0 or 1");
    return STN_OK;
  }
  if (strcmp(knob, "sweep2d_chunk") == 0) {
    if (tune_set_chunk2d(value) != STN_OK) return einval("sweep2d_chunk must be in [1, 2^30]");
    return STN_OK;
  }
  if (strcmp(knob, "repeat_graph") == 0) {
    if (tune_set_repeat_graph((int)value) != STN_OK) return einval("repeat_graph must be 0 or 1");
    return STN_OK;
  }
  if (strcmp(knob, "var_variant") == 0) {
    if (tune_set_var_variant((int)value) != STN_OK) return einval("var_variant must be -1, 0, 1 or 2");
    return STN_OK;
  }
  if (strcmp(knob, "sweep2d_ctas_per_sm") == 0) {
    if (tune_set_ctas2d((int)value) != STN_OK) return einval("sweep2d_ctas_per_sm must be in [1, 4]");
    return STN_OK;
  }
  if (strcmp(knob, "sweep2d_tma") == 0) {
    if (tune_set_tma2d((int)value) != STN_OK) return einval("sweep2d_tma must be 0 or 1");
    return STN_OK;
  }
  if (strcmp(knob, "fault_withhold_2d") == 0) {
    if (tune_set_withhold2d((int)value) != STN_OK) return einval("fault_withhold_2d must be 0 or 1");
    return STN_OK;
  }
  if (strcmp(knob, "batch_engine") == 0) {
    if (tune_set_batch_engine((int)value) != STN_OK) return einval("batch_engine must be 0, 1 or 2");
    return STN_OK;
  }
  if (strcmp(knob, "batch_graph") == 0) {
    if (tune_set_batch_graph((int)value) != STN_OK) return einval("batch_graph must be 0 or 1");
    return STN_OK;
  }
  if (strcmp(knob, "solve_graph") == 0) {
    if (tune_set_solve_graph((int)value) != STN_OK) return einval("solve_graph must be 0 or 1");
    return STN_OK;
  }
  if (strcmp(knob, "refined_engine") == 0) {
    if (tune_set_refined_engine((int)value) != STN_OK) return einval("refined_engine must be 0 or 1");
    return STN_OK;
  }
  if (strcmp(knob, "var_chunks") == 0) {
    if (tune_set_var_chunks((int)value) != STN_OK) return einval("var_chunks must be in [0, 65535]");
    return STN_OK;
  }
  if (strcmp(knob, "resident3d") == 0) {
    if (tune_set_resident3d((int)value) != STN_OK) return einval("resident3d must be 0 or 1");
    return STN_OK;
  }
  if (strcmp(knob, "fp64_double_word") == 0) {
    if (tune_set_double_word((int)value) != STN_OK) return einval("fp64_double_word must be 0 or 1");
    return STN_OK;
  }
  if (strcmp(knob, "fault_withhold_3d") == 0) {
    if (tune_set_withhold3d((int)value) != STN_OK) return einval("fault_withhold_3d must be 0 or 1");
    return STN_OK;
  }
  SchedFaults& f = sched_faults();
  if (strcmp(knob, "fault_withhold_last") == 0) {
    if (value < 0 || value > 1) return einval("fault_withhold_last must be 0 or 1");
    f.withhold_last = (int)value;
    return STN_OK;
  }
  if (strcmp(knob, "sched_idle_ms") == 0) {
    if (value < 1 || value > 600000) return einval("sched_idle_ms must be in [1, 600000]");
    f.idle_ms = value;
    return STN_OK;
  }
  if (strcmp(knob, "fault_admit_fail") == 0) {
    if (value < 0) return einval("fault_admit_fail must be >= 0");
    f.admit_fail = (int)value;
    return STN_OK;
  }
  return einval("unknown knob");
}

int stencil_tune_get(const char* knob, int64_t* value) {
  clear_error();
  if (!knob || !value) return einval("NULL knob or value");
  if (strcmp(knob, "star_variant") == 0) {
    *value = tune_get_star_variant();
    return STN_OK;
  }
  if (strcmp(knob, "temporal_depth") == 0) {
    *value = tune_get_temporal_depth();
    return STN_OK;
  }
  if (strcmp(knob, "star_chunks") == 0) {
    *value = tune_get_star_chunks();
    return STN_OK;
  }
  if (strcmp(knob, "sweep2d_resident") == 0) {
    *value = tune_get_resident2d();
    return STN_OK;
  }
  if (strcmp(knob, "sweep2d_chunk") == 0) {
    *value = tune_get_chunk2d();
    return STN_OK;
  }
  if (strcmp(knob, "repeat_graph") == 0) {
    *value = tune_get_repeat_graph();
    return STN_OK;
  }
  if (strcmp(knob, "var_variant") == 0) {
    *value = tune_get_var_variant();
    return STN_OK;
  }
  if (strcmp(knob, "sweep2d_ctas_per_sm") == 0) {
    *value = tune_get_ctas2d();
    return STN_OK;
  }
  if (strcmp(knob, "sweep2d_tma") == 0) {
    *value = tune_get_tma2d();
    return STN_OK;
  }
  if (strcmp(knob, "fault_withhold_2d") == 0) {
    *value = tune_get_withhold2d();
    return STN_OK;
  }
  if (strcmp(knob, "batch_engine") == 0) {
    *value = tune_get_batch_engine();
    return STN_OK;
  }
  if (strcmp(knob, "batch_graph") == 0) {
    *value = tune_get_batch_graph();
    return STN_OK;
  }
  if (strcmp(knob, "solve_graph") == 0) {
    *value = tune_get_solve_graph();
    return STN_OK;
  }
  if (strcmp(knob, "refined_engine") == 0) {
    *value = tune_get_refined_engine();
    return STN_OK;
  }
  if (strcmp(knob, "var_chunks") == 0) {
    *value = tune_get_var_chunks();
    return STN_OK;
  }
  if (strcmp(knob, "resident3d") == 0) {
    *value = tune_get_resident3d();
    return STN_OK;
  }
  if (strcmp(knob, "fp64_double_word") == 0) {
    *value = tune_get_double_word();
    return STN_OK;
  }
  if (strcmp(knob, "fault_withhold_3d") == 0) {
    *value = tune_get_withhold3d();
    return STN_OK;
  }
  const SchedFaults& f = sched_faults();
  if (strcmp(knob, "fault_withhold_last") == 0) {
    *value = f.withhold_last;
    return STN_OK;
  }
  if (strcmp(knob, "sched_idle_ms") == 0) {
    *value = f.idle_ms;
    return STN_OK;
  }
  if (strcmp(knob, "last_star_variant") == 0) {
    *value = star_last().variant;
    return STN_OK;
  }
  if (strcmp(knob, "last_star_chunks") == 0) {
    *value = star_last().chunks;
    return STN_OK;
  }
  if (strcmp(knob, "last_temporal_depth") == 0) {
    *value = star_last().depth;
    return STN_OK;
  }
  if (strcmp(knob, "fault_admit_fail") == 0) {
    *value = f.admit_fail;
    return STN_OK;
  }
  if (strcmp(knob, "fault_admit_failed") == 0) {
    *value = f.admit_failed;
    return STN_OK;
  }
  return einval("unknown knob");
}

int stencil_sched_stats(uint64_t* out, int n) {
  clear_error();
  if (!out || n < 1) return einval("NULL or empty stats buffer");
  unsigned long long v[SCHED_NSTATS];
  sched_last_stats(v);
  for (int i = 0; i < n && i < SCHED_NSTATS; i++) out[i] = v[i];
  return n < SCHED_NSTATS ? n : SCHED_NSTATS;
}

int stencil_release_workspace(void) {
  clear_error();
  return release_all();
}

int stencil_sweep_f64(double* in, double* out, int64_t nx, int64_t ny, int64_t nz,
                      const double* coeffs, int radius, int64_t iters, void* stream) {
  return sweep_impl<double>(in, out, nx, ny, nz, coeffs, radius, iters, stream);
}

int stencil_sweep_f32(float* in, float* out, int64_t nx, int64_t ny, int64_t nz,
                      const double* coeffs, int radius, int64_t iters, void* stream) {
  return sweep_impl<float>(in, out, nx, ny, nz, coeffs, radius, iters, stream);
}

int stencil_apply_f64(const double* u, const double* b, double* out, int64_t nx, int64_t ny,
                      int64_t nz, const double* coeffs, int radius, void* stream) {
  return apply_impl<double>(u, b, out, nx, ny, nz, coeffs, radius, stream);
}

int stencil_apply_f32(const float* u, const float* b, float* out, int64_t nx, int64_t ny,
                      int64_t nz, const double* coeffs, int radius, void* stream) {
  return apply_impl<float>(u, b, out, nx, ny, nz, coeffs, radius, stream);
}

int residual_norm_f64(const double* u, const double* b, int64_t nx, int64_t ny, int64_t nz,
                      const double* coeffs, int radius, double* norm_out, void* stream) {
  return residual_impl<double>(u, b, nx, ny, nz, coeffs, radius, norm_out, stream);
}

int residual_norm_f32(const float* u, const float* b, int64_t nx, int64_t ny, int64_t nz,
                      const double* coeffs, int radius, double* norm_out, void* stream) {
  return residual_impl<float>(u, b, nx, ny, nz, coeffs, radius, norm_out, stream);
}

int jacobi_solve_f64(const double* rhs, double* u, int64_t nx, int64_t ny, int64_t nz,
                     const double* coeffs, int radius, double tol, int64_t max_iters,
                     int64_t check_every, stn_solve_info* info, void* stream) {
  return jacobi_impl(rhs, u, nx, ny, nz, coeffs, radius, tol, max_iters, check_every, info, stream);
}

int jacobi_solve_refined_f64(const double* rhs, double* u, int64_t nx, int64_t ny, int64_t nz,
                             const double* coeffs, int radius, double tol, int64_t inner_sweeps,
                             double inner_tol, int64_t check_every, int64_t max_outer,
                             stn_solve_info* info, void* stream) {
  clear_error();
  if (!u) return einval("NULL grid");
  if (g_refined_engine == 1)
    return refined_direct_impl(rhs, u, nx, ny, nz, coeffs, radius, tol, inner_sweeps, inner_tol, check_every,
                               max_outer, info, stream);
  stn_problem p;
  p.nx = nx;
  p.ny = ny;
  p.nz = nz;
  p.rhs = rhs;
  p.u = u;
  return batch_impl(&p, 1, coeffs, radius, tol, inner_sweeps, check_every, inner_tol, max_outer, true,
                    info, stream);
}

int jacobi_solve_batched_f64(const stn_problem* probs, int64_t count, const double* coeffs,
                             int radius, double tol, int64_t max_iters, int64_t check_every,
                             stn_solve_info* infos, void* stream) {
  return batch_impl(probs, count, coeffs, radius, tol, max_iters, check_every, 0.0, 0, false, infos,
                    stream);
}

int jacobi_solve_batched_refined(const stn_problem* probs, int64_t count, const double* coeffs,
                                 int radius, double tol, int64_t inner_sweeps, double inner_tol,
                                 int64_t check_every, int64_t max_outer, stn_solve_info* infos,
                                 void* stream) {
  return batch_impl(probs, count, coeffs, radius, tol, inner_sweeps, check_every, inner_tol,
                    max_outer, true, infos, stream);
}

int varcoef_apply_f64(const double* u, const double* a, double* out, int64_t nx, int64_t ny,
                      int64_t nz, const double* w, int radius, void* stream) {
  return var_apply_impl(u, a, out, nx, ny, nz, w, radius, stream);
}

int varcoef_sweep_f64(double* in, double* out, const double* a, const double* f, int64_t nx,
                      int64_t ny, int64_t nz, const double* w, int radius, int64_t iters,
                      void* stream) {
  return var_sweep_impl<double>(in, out, a, f, nx, ny, nz, w, radius, iters, stream);
}

int varcoef_sweep_f32(float* in, float* out, const float* a, const float* f, int64_t nx,
                      int64_t ny, int64_t nz, const double* w, int radius, int64_t iters,
                      void* stream) {
  return var_sweep_impl<float>(in, out, a, f, nx, ny, nz, w, radius, iters, stream);
}

int varcoef_residual_norm_f64(const double* u, const double* a, const double* f, int64_t nx,
                              int64_t ny, int64_t nz, const double* w, int radius,
                              double* norm_out, void* stream) {
  return var_residual_impl(u, a, f, nx, ny, nz, w, radius, norm_out, stream);
}

int jacobi_solve_varcoef_f64(const double* a, const double* f, double* u, int64_t nx, int64_t ny,
                             int64_t nz, const double* w, int radius, double tol,
                             int64_t max_iters, int64_t check_every, stn_solve_info* info,
                             void* stream) {
  return var_jacobi_impl(a, f, u, nx, ny, nz, w, radius, tol, max_iters, check_every, info, stream);
}

int jacobi_solve_varcoef_refined(const double* a, const double* f, double* u, int64_t nx,
                                 int64_t ny, int64_t nz, const double* w, int radius, double tol,
                                 int64_t inner_sweeps, int64_t max_outer, stn_solve_info* info,
                                 void* stream) {
  return refined_impl(a, f, u, nx, ny, nz, w, radius, tol, inner_sweeps, max_outer, info, stream);
}

int stencil_sweep2d_f64(double* in, double* out, int64_t nx, int64_t ny, const double* coeffs,
                        int radius, int64_t iters, void* stream) {
  return sweep2d_impl<double>(in, out, nx, ny, coeffs, radius, iters, stream);
}

int stencil_sweep2d_f32(float* in, float* out, int64_t nx, int64_t ny, const double* coeffs,
                        int radius, int64_t iters, void* stream) {
  return sweep2d_impl<float>(in, out, nx, ny, coeffs, radius, iters, stream);
}

int residual_norm2d_f64(const double* u, const double* b, int64_t nx, int64_t ny,
                        const double* coeffs, int radius, double* norm_out, void* stream) {
  return residual2d_impl<double>(u, b, nx, ny, coeffs, radius, norm_out, stream);
}

int residual_norm2d_f32(const float* u, const float* b, int64_t nx, int64_t ny,
                        const double* coeffs, int radius, double* norm_out, void* stream) {
  return residual2d_impl<float>(u, b, nx, ny, coeffs, radius, norm_out, stream);
}

int reduce_sum_f64(const double* x, int64_t n, double* out, void* stream) {
  return vec_reduce_impl(x, nullptr, n, out, stream);
}

int dot_f64(const double* x, const double* y, int64_t n, double* out, void* stream) {
  if (n > 0 && !y) {
    clear_error();
    return einval("NULL array");
  }
  return vec_reduce_impl(x, y, n, out, stream);
}

int advect_f64(const double* u, const double* v, const double* w, const double* const* q, int nq,
               double* const* s, int64_t nx, int64_t ny, int64_t nz, const double* c, void* stream) {
  return advect_impl<double>(u, v, w, q, nq, s, nx, ny, nz, c, stream);
}

int advect_f32(const float* u, const float* v, const float* w, const float* const* q, int nq,
               float* const* s, int64_t nx, int64_t ny, int64_t nz, const double* c, void* stream) {
  return advect_impl<float>(u, v, w, q, nq, s, nx, ny, nz, c, stream);
}

}  // extern "C"
