// Shared declarations of the persistent scheduler (sched.cu) and its hosts
// (batched solves in batched.cu, the serving loop in server.cpp).
#pragma once

#include "internal.h"

namespace stn {

// One problem: u = S u + b on a padded grid, with its scratch.
struct SchedProblem {
  int nx, ny, nz, nunits;
  double* u;         // iterate (in/out)
  const double* b;   // source term (may be null)
  double* t;         // double scratch grid; its halo must equal u's halo
  float* e;          // refined: correction grids (zeroed, halo included)
  float* e2;
  float* r32;
  double* partials;  // one per work unit
};

// Scheduler state of one slot (one problem in flight).
struct SchedSlot {
  int problem;          // index into the problem / result arrays
  int phase;            // pass kind (sched.cu Phase)
  int status;
  int parity;           // which grid of a ping-pong pair holds the iterate
  int resid;            // the current sweep also reduces its residual
  int nunits;           // units of the current pass (0 when idle)
  int done;             // units completed in the current pass
  int claim_free;       // 1 when the slot holds no problem
  unsigned pass;        // id of the published pass (high word of the claim word)
  int pad;
  long long group, group_pos;
  long long iters, outer, sweeps, inner;
  long long start_clock;
  double bnorm, scale, res, rel, smax, r32norm;
};

struct SchedResult {
  long long iters;
  long long outer;
  double rel_res;
  double res_norm;
  double rhs_norm;
  long long clocks;  // device clock cycles from admission to completion
  int status;
  int pad;
};

struct SchedArgs {
  SchedProblem* probs;
  SchedSlot* slots;
  unsigned long long* words;  // per slot: claim word (pass id, units of the pass, next unit)
  int nslots;
  int count;                  // problems in total (batch) / queue capacity bound (serving)
  int qlen;                   // batch: queue entries available (count, or fewer under fault injection)
  const int* queue;           // problem indices in admission order (ring of qcap)
  int qcap;
  int* qhead;                 // device counter of taken queue entries
  const int* qtail;           // serving: host-advanced count of queued entries
  int serving;
  SchedResult* results;       // per problem
  int* done_flags;            // per problem: 1 once its result is written
  int* finished;              // problems finished
  int* free_slots;            // slots holding no problem
  int* error;                 // first error (STN_ETIMEOUT, ...), 0 if none
  double coeffs[3];
  double tol;
  long long max_iters;        // plain: sweeps; refined: float sweeps per outer step
  long long check_every;
  double inner_tol;
  long long max_outer;
  int refined;
  long long idle_cycles;      // give up after this many clock cycles without work
  unsigned long long* stats;  // optional SCHED_NSTATS counters (cycles and counts), or null
};

// Scheduler counters (summed over CTAs): clock cycles spent finding and
// claiming units, computing units, completing units (publish of the partial
// and the done count), in pass epilogues, idle; units done; epilogues run;
// claim attempts that found nothing.
enum {
  SCHED_CYC_CLAIM = 0,
  SCHED_CYC_UNIT = 1,
  SCHED_CYC_DONE = 2,
  SCHED_CYC_EPI = 3,
  SCHED_CYC_IDLE = 4,
  SCHED_N_UNITS = 5,
  SCHED_N_EPI = 6,
  SCHED_N_MISS = 7,
  SCHED_N_FAST = 8,   // units claimed on the same slot and pass as the CTA's previous unit
  SCHED_N_TRIES = 9,  // claim atomics issued by slot scans (successful or not)
  SCHED_NSTATS = 10
};
// Counters of the last scheduler launch made by this process.
void sched_last_stats(unsigned long long* out);

int sched_launch(const SchedArgs& a, int radius, bool has_c0, int ctas, cudaStream_t s);
// Allocates the launch counters once (before a launch is captured into a
// graph), and names the stream the counters are read back on.
int sched_prepare();
void sched_set_stats_stream(cudaStream_t s);

// Fault injection and limits for tests (process-wide; all default to off).
struct SchedFaults {
  int withhold_last = 0;      // batch: never queue the last problem (the CTAs then time out)
  long long idle_ms = 2000;   // batch: idle limit before STN_ETIMEOUT
  int admit_fail = 0;         // server: fail this many admission allocations (retried later)
  long long admit_failed = 0; // server: admission failures seen so far
};
SchedFaults& sched_faults();
// CTAs of one full wave of the scheduler kernel (-1 on error); refined
// launches use an instantiation with more resident blocks per SM.
int sched_ctas(int radius, bool has_c0, bool refined);
// Work units of a problem's pass.
i64 sched_units(i64 nx, i64 ny, i64 nz);

// A slot's claim word: the published pass's id (low 16 bits of it; compared
// for equality only), its unit count (24 bits) and the next unit to hand out
// (24 bits).  A claim is one atomicAdd, valid when the returned next unit is
// below the returned count, so a failed claim costs no further reads.
// Problems are limited to kMaxPassUnits units per pass, which leaves the
// next-unit field 3 x 2^22 increments of headroom for claims that lose races
// after a pass runs out (at most a few per CTA and pass).
constexpr i64 kMaxPassUnits = (i64)1 << 22;
__host__ __device__ inline unsigned long long claim_word(unsigned pass, int nunits) {
  return ((unsigned long long)(pass & 0xffffu) << 48) | ((unsigned long long)(unsigned)nunits << 24);
}
__host__ __device__ inline unsigned claim_pass(unsigned long long w) { return (unsigned)(w >> 48); }
__host__ __device__ inline int claim_units(unsigned long long w) { return (int)((w >> 24) & 0xffffffu); }
__host__ __device__ inline int claim_next(unsigned long long w) { return (int)(w & 0xffffffu); }

}  // namespace stn
