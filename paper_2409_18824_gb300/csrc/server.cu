// Serving loop: Jacobi/Poisson solve requests arrive at any time, are
// admitted against a device-memory budget, and run concurrently on the GPU
// inside the persistent work-unit scheduler (sched.cu) -- continuous
// batching: a request admitted while others are on the GPU joins the running
// kernel through its queue, and its passes interleave with theirs.
//
// Host side: stn_submit copies the request into server memory and returns a
// ticket.  One server thread owns every CUDA call: it admits pending
// requests in arrival order while their grids fit in the budget (device
// grids from a stream-ordered pool, right-hand side copied in, problem
// descriptor written, queue tail advanced with a system-scope release), keeps
// the scheduler kernel running while work is outstanding (the kernel exits
// after a bounded idle period; the thread relaunches it), and collects
// finished requests from host-mapped done flags (solution copied out, grids
// freed, budget returned, waiters woken).
//
// A result depends only on its own request: the scheduler's passes are the
// batched passes, reduced in a fixed order whatever else is in flight.
#include <string.h>
#include <time.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "work_sched.h"

namespace stn {
namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
  uint64_t ticket = 0;
  i64 nx = 0, ny = 0, nz = 0;
  std::vector<double> rhs;  // padded grid
  std::vector<double> u;    // padded grid: initial guess in, solution out
  int state = 0;            // 0 pending, 1 on device, 2 done
  int pi = -1;              // problem-table entry
  size_t bytes = 0;
  char* dev = nullptr;      // device block
  double t_submit = 0, t_admit = 0, t_done = 0;
  stn_solve_info info{};
  int rc = STN_OK;
};

}  // namespace

struct ServerImpl {
  stn_server_opts opts{};
  int device = 0;
  cudaStream_t sk = nullptr, sc = nullptr;  // kernel stream, copy stream
  cudaEvent_t kev = nullptr;
  bool kernel_launched = false;
  int ctas = 0, nslots = 0, cap = 0;
  // device state
  SchedProblem* probs = nullptr;
  SchedSlot* slots = nullptr;
  unsigned long long* words = nullptr;
  int* ctr = nullptr;  // qhead, finished, error, free_slots
  // host-mapped state
  int* queue = nullptr;
  int* qtail = nullptr;
  SchedResult* results = nullptr;
  int* done_flags = nullptr;
  int* queue_d = nullptr;
  int* qtail_d = nullptr;
  SchedResult* results_d = nullptr;
  int* done_flags_d = nullptr;
  int tail = 0;
  std::vector<int> free_pi;
  // requests
  std::mutex mu;
  std::condition_variable cv;
  std::map<uint64_t, Req*> reqs;
  std::deque<Req*> pending;
  std::vector<Req*> running;
  uint64_t next_ticket = 1;
  size_t in_use = 0;
  bool stop = false;
  int fatal = STN_OK;
  std::string fatal_msg;
  std::thread th;
  long long submitted = 0, completed = 0;

  size_t need_bytes(const Req& r) const {
    const size_t n = (size_t)((r.nx + 2 * opts.radius) * (r.ny + 2 * opts.radius) * (r.nz + 2 * opts.radius));
    const size_t n8 = (n * 8 + 255) / 256 * 256, n4 = (n * 4 + 255) / 256 * 256;
    // pool engine: u, rhs, one double scratch grid and, refined, three float ones
    if (opts.engine == 1) return 3 * n8 + (opts.refined ? 3 * n4 : 0);
    const size_t units = (size_t)sched_units(r.nx, r.ny, r.nz);
    return 3 * n8 + (opts.refined ? 3 * n4 : 0) + (units * 8 + 255) / 256 * 256;
  }

  // --- stream-pool engine ----------------------------------------------------
  // Worker w owns stream ws_[w].  It takes the oldest pending request when
  // its grids fit the budget (arrival order: a request that does not fit
  // holds back the ones behind it), runs it on the full-grid kernels, copies
  // the solution out and frees the grids.  max_inflight workers run their
  // requests at the same time, so requests arriving while others are on the
  // GPU are admitted as workers and memory free up and their kernels overlap
  // with the running ones.  A result depends only on its request.
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> wstreams;

  void pool_worker(int w) {
    cudaSetDevice(device);
    cudaStream_t st = wstreams[(size_t)w];
    {
      // partial-sum slots for any request up to 256^3-class grids, sized once:
      // growing them later would synchronise the device under the others
      Workspace* ws;
      if (get_workspace(st, (i64)1 << 17, 0, &ws) != STN_OK) {
        std::lock_guard<std::mutex> lk(mu);
        fail(STN_ENOMEM, "server worker workspace");
        cv.notify_all();
        return;
      }
    }
    while (true) {
      Req* r = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] {
          if (fatal != STN_OK) return true;
          if (pending.empty()) return stop;
          return in_use + pending.front()->bytes <= opts.hbm_budget;
        });
        if (fatal != STN_OK) {  // the server cannot run: fail what is left
          for (Req* q : pending) {
            q->rc = fatal;
            q->t_done = now_s();
            q->state = 2;
          }
          pending.clear();
          cv.notify_all();
          return;
        }
        if (pending.empty()) return;
        r = pending.front();
        pending.pop_front();
        in_use += r->bytes;
        running.push_back(r);
        r->state = 1;
        r->t_admit = now_s();
      }
      const int rc = pool_run(r, st);
      {
        std::lock_guard<std::mutex> lk(mu);
        if (rc == -1) {  // device pool busy (or an injected failure): back to the head, retry
          in_use -= r->bytes;
          running.erase(std::find(running.begin(), running.end(), r));
          r->state = 0;
          r->t_admit = 0;
          pending.push_front(r);
          cv.notify_all();
        } else {
          r->rc = rc;
          in_use -= r->bytes;
          running.erase(std::find(running.begin(), running.end(), r));
          r->t_done = now_s();
          r->state = 2;
          completed++;
          cv.notify_all();
        }
      }
      if (rc == -1) std::this_thread::sleep_for(std::chrono::milliseconds(1));
    }
  }

  // One request on stream st: -1 when the grids could not be allocated now,
  // else the solve's status or an error.
  int pool_run(Req* r, cudaStream_t st) {
    const int R = opts.radius;
    const Grid g{r->nx, r->ny, r->nz, R};
    const size_t n = (size_t)g.count();
    const size_t n8 = (n * 8 + 255) / 256 * 256;
    {
      SchedFaults& f = sched_faults();
      std::lock_guard<std::mutex> lk(mu);
      if (f.admit_fail > 0) {  // injected allocation failure: same path as a busy pool
        f.admit_fail--;
        f.admit_failed++;
        return -1;
      }
    }
    char* dev = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&dev, r->bytes, st);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return -1;
    }
    double* du = (double*)dev;
    double* db = (double*)(dev + n8);
    double* dt = (double*)(dev + 2 * n8);
    float* f32 = (float*)(dev + 3 * n8);
    int rc = STN_OK;
    if ((e = cudaMemcpyAsync(du, r->u.data(), n * 8, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(db, r->rhs.data(), n * 8, cudaMemcpyHostToDevice, st)))
      rc = cuda_fail(e, "server admission copy");
    stn_solve_info info{};
    if (rc == STN_OK) {
      rc = opts.refined ? solve_refined_core(db, du, dt, f32, g, opts.coeffs, opts.tol, opts.inner_sweeps,
                                             opts.inner_tol, opts.check_every, opts.max_outer, &info, st)
                        : solve_jacobi_core(db, du, dt, g, opts.coeffs, opts.tol, opts.max_iters, opts.check_every,
                                            &info, st);
    }
    if (rc >= 0) {
      if ((e = cudaMemcpyAsync(r->u.data(), du, n * 8, cudaMemcpyDeviceToHost, st))) rc = cuda_fail(e, "server copy-out");
    }
    cudaFreeAsync(dev, st);
    if ((e = cudaStreamSynchronize(st)) && rc >= 0) rc = cuda_fail(e, "server request");
    r->info = info;
    return rc;
  }

  int fail(int rc, const std::string& m) {
    fatal = rc;
    fatal_msg = m;
    return rc;
  }

  // --- server thread -------------------------------------------------------
  int admit_one(Req* r) {
    const size_t n = (size_t)((r->nx + 2 * opts.radius) * (r->ny + 2 * opts.radius) * (r->nz + 2 * opts.radius));
    const size_t n8 = (n * 8 + 255) / 256 * 256, n4 = (n * 4 + 255) / 256 * 256;
    cudaError_t e;
    {
      SchedFaults& f = sched_faults();
      if (f.admit_fail > 0) {  // injected allocation failure: same path as a busy pool
        f.admit_fail--;
        f.admit_failed++;
        return -1;
      }
    }
    e = cudaMallocAsync((void**)&r->dev, r->bytes, sc);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return -1;  // pool could not serve it right now: retry later
    }
    SchedProblem p;
    memset(&p, 0, sizeof(p));
    p.nx = (int)r->nx;
    p.ny = (int)r->ny;
    p.nz = (int)r->nz;
    p.nunits = (int)sched_units(r->nx, r->ny, r->nz);
    p.u = (double*)r->dev;
    p.b = (const double*)(r->dev + n8);
    p.t = (double*)(r->dev + 2 * n8);
    size_t off = 3 * n8;
    if (opts.refined) {
      p.e = (float*)(r->dev + off);
      p.e2 = (float*)(r->dev + off + n4);
      p.r32 = (float*)(r->dev + off + 2 * n4);
      off += 3 * n4;
    }
    p.partials = (double*)(r->dev + off);
    const int pi = free_pi.back();
    free_pi.pop_back();
    r->pi = pi;
    done_flags[pi] = 0;
    if ((e = cudaMemcpyAsync(p.u, r->u.data(), n * 8, cudaMemcpyHostToDevice, sc)) ||
        (e = cudaMemcpyAsync((void*)p.b, r->rhs.data(), n * 8, cudaMemcpyHostToDevice, sc)) ||
        (e = cudaMemcpyAsync(p.t, r->u.data(), n * 8, cudaMemcpyHostToDevice, sc)) ||
        (opts.refined && (e = cudaMemsetAsync(p.e, 0, 3 * n4, sc))) ||
        (e = cudaMemcpyAsync(&probs[pi], &p, sizeof(p), cudaMemcpyHostToDevice, sc)) ||
        (e = cudaStreamSynchronize(sc)))
      return fail(cuda_fail(e, "server admission"), "admission copy failed");
    queue[tail % cap] = pi;
    tail++;
    __atomic_store_n(qtail, tail, __ATOMIC_RELEASE);
    r->state = 1;
    r->t_admit = now_s();
    return 0;
  }

  void collect() {
    for (size_t k = 0; k < running.size();) {
      Req* r = running[k];
      if (__atomic_load_n(&done_flags[r->pi], __ATOMIC_ACQUIRE) == 0) {
        k++;
        continue;
      }
      const SchedResult res = results[r->pi];
      const size_t n = (size_t)((r->nx + 2 * opts.radius) * (r->ny + 2 * opts.radius) * (r->nz + 2 * opts.radius));
      cudaError_t e = cudaMemcpyAsync(r->u.data(), r->dev, n * 8, cudaMemcpyDeviceToHost, sc);
      if (e == cudaSuccess) e = cudaFreeAsync(r->dev, sc);
      if (e == cudaSuccess) e = cudaStreamSynchronize(sc);
      std::lock_guard<std::mutex> lk(mu);
      if (e != cudaSuccess) {
        r->rc = cuda_fail(e, "server collection");
      } else {
        r->rc = res.status;
      }
      r->info.iters = res.iters;
      r->info.outer = res.outer;
      r->info.rel_res = res.rel_res;
      r->info.res_norm = res.res_norm;
      r->info.rhs_norm = res.rhs_norm;
      r->info.status = res.status;
      r->dev = nullptr;
      in_use -= r->bytes;
      free_pi.push_back(r->pi);
      r->t_done = now_s();
      r->state = 2;
      completed++;
      running[k] = running.back();
      running.pop_back();
      cv.notify_all();
    }
  }

  bool kernel_running() {
    if (!kernel_launched) return false;
    cudaError_t q = cudaEventQuery(kev);
    if (q == cudaErrorNotReady) return true;
    kernel_launched = false;
    if (q != cudaSuccess) fail(cuda_fail(q, "scheduler kernel"), "scheduler kernel failed");
    return false;
  }

  void launch_kernel() {
    SchedArgs a;
    memset(&a, 0, sizeof(a));
    a.probs = probs;
    a.slots = slots;
    a.words = words;
    a.nslots = nslots;
    a.count = cap;
    a.qlen = 0;
    a.queue = queue_d;
    a.qcap = cap;
    a.qhead = ctr + 0;
    a.finished = ctr + 1;
    a.error = ctr + 2;
    a.free_slots = ctr + 3;
    a.qtail = qtail_d;
    a.serving = 1;
    a.results = results_d;
    a.done_flags = done_flags_d;
    for (int d = 0; d < 3; d++) a.coeffs[d] = opts.coeffs[d];
    a.tol = opts.tol;
    a.max_iters = opts.refined ? opts.inner_sweeps : opts.max_iters;
    a.check_every = opts.check_every;
    a.inner_tol = opts.inner_tol;
    a.max_outer = opts.max_outer;
    a.refined = opts.refined;
    a.idle_cycles = 100000000ll;  // about 50 ms without work, then exit (relaunched on demand)
    int rc = sched_launch(a, opts.radius, opts.coeffs[0] != 0.0, ctas, sk);
    if (rc != STN_OK) {
      fail(rc, "scheduler launch failed");
      return;
    }
    cudaEventRecord(kev, sk);
    kernel_launched = true;
  }

  void loop() {
    cudaSetDevice(device);
    while (true) {
      {
        std::unique_lock<std::mutex> lk(mu);
        if (stop && pending.empty() && running.empty()) break;
        if (fatal != STN_OK) break;
        // admission in arrival order while the budget allows
        while (!pending.empty() && !free_pi.empty()) {
          Req* r = pending.front();
          if (in_use + r->bytes > opts.hbm_budget) break;
          in_use += r->bytes;
          lk.unlock();
          const int rc = admit_one(r);
          lk.lock();
          if (rc < 0) {  // device pool busy: retry on the next turn
            in_use -= r->bytes;
            break;
          }
          if (rc > 0 || fatal != STN_OK) break;
          pending.pop_front();
          running.push_back(r);
        }
      }
      if (fatal != STN_OK) break;
      if (!running.empty() && !kernel_running() && fatal == STN_OK) launch_kernel();
      collect();
      bool idle;
      {
        std::lock_guard<std::mutex> lk(mu);
        idle = pending.empty() && running.empty();
      }
      if (idle) {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait_for(lk, std::chrono::milliseconds(2), [&] { return stop || !pending.empty(); });
      } else {
        std::this_thread::sleep_for(std::chrono::microseconds(50));
      }
    }
    // wait for the kernel to go idle and exit (bounded by its idle timeout)
    if (kernel_launched) cudaEventSynchronize(kev);
    std::lock_guard<std::mutex> lk(mu);
    if (fatal != STN_OK) {
      for (Req* r : pending) {
        r->rc = fatal;
        r->state = 2;
      }
      for (Req* r : running) {
        r->rc = fatal;
        r->state = 2;
      }
      pending.clear();
      running.clear();
    }
    cv.notify_all();
  }
};

}  // namespace stn

using namespace stn;

extern "C" {

stn_server* stn_server_create(const stn_server_opts* o) {
  clear_error();
  if (!o) {
    set_error("invalid argument: NULL options");
    return nullptr;
  }
  if ((o->radius != 1 && o->radius != 2) || !(o->tol >= 0.0) || o->check_every < 1 ||
      o->max_inflight < 1 || o->max_iters < 0 || o->inner_sweeps < 0 || o->max_outer < 0 ||
      !(o->inner_tol >= 0.0) || o->hbm_budget == 0 || o->queue_capacity < 1 || o->engine < 0 || o->engine > 1 ||
      (o->engine == 1 && o->max_inflight > 64)) {
    set_error("invalid argument: server options out of range");
    return nullptr;
  }
  ServerImpl* s = new ServerImpl();
  s->opts = *o;
  cudaError_t e;
  auto bad = [&](cudaError_t err, const char* what) {
    cuda_fail(err, what);
    delete s;
    return (stn_server*)nullptr;
  };
  if ((e = cudaGetDevice(&s->device))) return bad(e, "cudaGetDevice");
  keep_pool_memory();
  if (o->engine == 1) {
    for (int w = 0; w < o->max_inflight; w++) {
      cudaStream_t st;
      if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking))) {
        for (cudaStream_t x : s->wstreams) cudaStreamDestroy(x);
        s->wstreams.clear();
        return bad(e, "stream");
      }
      s->wstreams.push_back(st);
    }
    for (int w = 0; w < o->max_inflight; w++) s->workers.emplace_back([s, w] { s->pool_worker(w); });
    return (stn_server*)s;
  }
  s->ctas = sched_ctas(o->radius, o->coeffs[0] != 0.0, o->refined != 0);
  if (s->ctas < 1) {
    set_error("scheduler kernel does not fit on an SM");
    delete s;
    return nullptr;
  }
  s->nslots = o->max_inflight;
  s->cap = o->queue_capacity;
  if ((e = cudaStreamCreateWithFlags(&s->sk, cudaStreamNonBlocking))) return bad(e, "stream");
  if ((e = cudaStreamCreateWithFlags(&s->sc, cudaStreamNonBlocking))) return bad(e, "stream");
  if ((e = cudaEventCreateWithFlags(&s->kev, cudaEventDisableTiming))) return bad(e, "event");
  if ((e = cudaMalloc(&s->probs, sizeof(SchedProblem) * s->cap))) return bad(e, "cudaMalloc");
  if ((e = cudaMalloc(&s->slots, sizeof(SchedSlot) * s->nslots))) return bad(e, "cudaMalloc");
  if ((e = cudaMalloc(&s->words, sizeof(unsigned long long) * s->nslots))) return bad(e, "cudaMalloc");
  if ((e = cudaMalloc(&s->ctr, sizeof(int) * 8))) return bad(e, "cudaMalloc");
  if ((e = cudaHostAlloc(&s->queue, sizeof(int) * s->cap, cudaHostAllocMapped))) return bad(e, "cudaHostAlloc");
  if ((e = cudaHostAlloc(&s->qtail, sizeof(int) * 32, cudaHostAllocMapped))) return bad(e, "cudaHostAlloc");
  if ((e = cudaHostAlloc(&s->results, sizeof(SchedResult) * s->cap, cudaHostAllocMapped))) return bad(e, "cudaHostAlloc");
  if ((e = cudaHostAlloc(&s->done_flags, sizeof(int) * s->cap, cudaHostAllocMapped))) return bad(e, "cudaHostAlloc");
  if ((e = cudaHostGetDevicePointer(&s->queue_d, s->queue, 0))) return bad(e, "mapped pointer");
  if ((e = cudaHostGetDevicePointer(&s->qtail_d, s->qtail, 0))) return bad(e, "mapped pointer");
  if ((e = cudaHostGetDevicePointer(&s->results_d, s->results, 0))) return bad(e, "mapped pointer");
  if ((e = cudaHostGetDevicePointer(&s->done_flags_d, s->done_flags, 0))) return bad(e, "mapped pointer");
  memset(s->queue, 0, sizeof(int) * s->cap);
  memset(s->qtail, 0, sizeof(int) * 32);
  memset(s->done_flags, 0, sizeof(int) * s->cap);
  std::vector<SchedSlot> hs((size_t)s->nslots);
  for (auto& sl : hs) {
    memset(&sl, 0, sizeof(sl));
    sl.claim_free = 1;
  }
  const int c0[8] = {0, 0, 0, s->nslots, 0, 0, 0, 0};
  if ((e = cudaMemcpy(s->slots, hs.data(), sizeof(SchedSlot) * s->nslots, cudaMemcpyHostToDevice)) ||
      (e = cudaMemset(s->words, 0, sizeof(unsigned long long) * s->nslots)) ||
      (e = cudaMemcpy(s->ctr, c0, sizeof(c0), cudaMemcpyHostToDevice)))
    return bad(e, "server state init");
  for (int i = s->cap - 1; i >= 0; i--) s->free_pi.push_back(i);
  s->th = std::thread([s] { s->loop(); });
  return (stn_server*)s;
}

int stn_submit(stn_server* sv, const stn_request* req, uint64_t* ticket) {
  clear_error();
  ServerImpl* s = (ServerImpl*)sv;
  if (!s || !req || !ticket || !req->rhs) {
    set_error("invalid argument: NULL server, request, rhs or ticket");
    return STN_EINVAL;
  }
  const int r = s->opts.radius;
  if (req->nx < 1 || req->ny < 1 || req->nz < 1 || req->nx > 4096 || req->ny > 4096 || req->nz > 4096) {
    set_error("invalid argument: request extents out of range");
    return STN_EINVAL;
  }
  Req* q = new Req();
  q->nx = req->nx;
  q->ny = req->ny;
  q->nz = req->nz;
  const size_t n = (size_t)((q->nx + 2 * r) * (q->ny + 2 * r) * (q->nz + 2 * r));
  q->bytes = s->need_bytes(*q);
  if (q->bytes > s->opts.hbm_budget) {
    delete q;
    set_error("request needs more device memory than the whole server budget");
    return STN_EBUSY;
  }
  q->rhs.assign(req->rhs, req->rhs + n);
  if (req->u0) q->u.assign(req->u0, req->u0 + n);
  else q->u.assign(n, 0.0);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->fatal != STN_OK) {
    delete q;
    set_error("server failed: " + s->fatal_msg);
    return s->fatal;
  }
  if (s->stop) {
    delete q;
    set_error("server is shutting down");
    return STN_EBUSY;
  }
  q->ticket = s->next_ticket++;
  q->t_submit = now_s();
  s->reqs[q->ticket] = q;
  s->pending.push_back(q);
  s->submitted++;
  *ticket = q->ticket;
  s->cv.notify_all();
  return STN_OK;
}

static int fill_result(ServerImpl* s, Req* q, stn_result* res) {
  if (res) {
    res->info = q->info;
    res->latency_s = q->t_done - q->t_submit;
    res->queue_s = q->t_admit > 0 ? q->t_admit - q->t_submit : q->t_done - q->t_submit;
    res->rc = q->rc;
  }
  (void)s;
  return q->rc < 0 ? q->rc : STN_OK;
}

int stn_poll(stn_server* sv, uint64_t ticket, stn_result* res) {
  clear_error();
  ServerImpl* s = (ServerImpl*)sv;
  if (!s) return STN_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) {
    set_error("invalid argument: unknown ticket");
    return STN_EINVAL;
  }
  if (it->second->state != 2) return STN_PENDING;
  return fill_result(s, it->second, res);
}

int stn_wait(stn_server* sv, uint64_t ticket, double timeout_s, stn_result* res) {
  clear_error();
  ServerImpl* s = (ServerImpl*)sv;
  if (!s) return STN_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) {
    set_error("invalid argument: unknown ticket");
    return STN_EINVAL;
  }
  Req* q = it->second;
  const bool ok = s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s < 0 ? 1e9 : timeout_s),
                                 [&] { return q->state == 2; });
  if (!ok) {
    set_error("timed out waiting for the request");
    return STN_ETIMEOUT;
  }
  return fill_result(s, q, res);
}

int stn_result_copy(stn_server* sv, uint64_t ticket, double* u_out) {
  clear_error();
  ServerImpl* s = (ServerImpl*)sv;
  if (!s || !u_out) return STN_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) {
    set_error("invalid argument: unknown ticket");
    return STN_EINVAL;
  }
  if (it->second->state != 2) return STN_PENDING;
  memcpy(u_out, it->second->u.data(), it->second->u.size() * sizeof(double));
  return STN_OK;
}

int stn_release(stn_server* sv, uint64_t ticket) {
  clear_error();
  ServerImpl* s = (ServerImpl*)sv;
  if (!s) return STN_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return STN_EINVAL;
  if (it->second->state != 2) return STN_PENDING;
  delete it->second;
  s->reqs.erase(it);
  return STN_OK;
}

int stn_server_stats(stn_server* sv, stn_server_stats_t* st) {
  ServerImpl* s = (ServerImpl*)sv;
  if (!s || !st) return STN_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->pending = (int64_t)s->pending.size();
  st->running = (int64_t)s->running.size();
  st->bytes_in_use = s->in_use;
  st->status = s->fatal;
  return STN_OK;
}

void stn_server_destroy(stn_server* sv) {
  ServerImpl* s = (ServerImpl*)sv;
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->th.joinable()) s->th.join();
  for (auto& t : s->workers)
    if (t.joinable()) t.join();
  if (s->opts.engine == 1) {
    for (cudaStream_t x : s->wstreams) cudaStreamDestroy(x);
    for (auto& kv : s->reqs) delete kv.second;
    delete s;
    return;
  }
  cudaStreamSynchronize(s->sk);
  cudaStreamSynchronize(s->sc);
  for (auto& kv : s->reqs) {
    if (kv.second->dev) cudaFree(kv.second->dev);
    delete kv.second;
  }
  cudaFree(s->probs);
  cudaFree(s->slots);
  cudaFree(s->words);
  cudaFree(s->ctr);
  cudaFreeHost(s->queue);
  cudaFreeHost(s->qtail);
  cudaFreeHost(s->results);
  cudaFreeHost(s->done_flags);
  cudaEventDestroy(s->kev);
  cudaStreamDestroy(s->sk);
  cudaStreamDestroy(s->sc);
  delete s;
}

}  // extern "C"
