/*
 * stencil.h -- C ABI of libstencil.so: iterated 3D structured-grid Jacobi
 * stencil sweeps with a fused residual-norm reduction, on one NVIDIA GB300
 * (sm_103a).
 *
 * The operation is the "jacobi" benchmark of arXiv 2409.18824 (Sec. 4: a
 * Jacobi iteration solving Laplace's equation on a structured grid), which
 * the paper's compiler flow expresses as a stencil (Sec. 2.2) plus a sum
 * reduction (Sec. 5.3, Listing 8).  Here it is three-dimensional.
 *
 * ---------------------------------------------------------------- layout ---
 * Every grid argument is a Fortran array  u(1:nx+2r, 1:ny+2r, 1:nz+2r)  in
 * column-major order: element (i,j,k) (1-based) sits at 0-based offset
 *     (i-1) + (j-1)*NX + (k-1)*NX*NY,   NX = nx+2r, NY = ny+2r, NZ = nz+2r
 * (Sec. 5.2, Listing 7: subtract the lower bound, first index fastest).
 * nx, ny, nz are the INTERIOR extents; r is the stencil radius.  The outer r
 * layers on every face are the Dirichlet halo: read, never written by a
 * sweep.  A C caller sees the same memory as a row-major array [NZ][NY][NX].
 * A grid holds NX*NY*NZ elements; no padding, no pitch.
 *
 * ---------------------------------------------------------------- stencil ---
 * Constant-coefficient star stencil, radius r in {1, 2}, coefficients
 * coeffs[0..r] (a HOST array of r+1 doubles): for each interior point
 *     out = c0*u + sum_{d=1..r} c_d * S_d  (+ b)
 *     S_d = ((u(i-d)+u(i+d)) + (u(j-d)+u(j+d))) + (u(k-d)+u(k+d))
 * evaluated in exactly this order: acc = c_r*S_r, then acc += c_d*S_d for
 * d = r-1..1, then acc += c0*u if c0 != 0, then acc += b if b is given; every
 * product and sum rounded separately (no fused multiply-add), so the double
 * path is bitwise reproducible.  The 7-point Laplace update is r = 1,
 * coeffs = {0, 1/6}.  The _f32 entry points round the coefficients to float
 * and compute in float.
 *
 * ------------------------------------------------------- pointers/streams ---
 * Grid pointers may be DEVICE memory (cudaMalloc, a torch CUDA tensor) or
 * HOST memory (pageable or pinned).  When every grid argument of a call is in
 * device memory the call is asynchronous on `stream` (a cudaStream_t passed as
 * void*; NULL = the legacy default stream) unless stated otherwise.  When any
 * grid argument is host memory the library stages all of them through device
 * memory it allocates for the call, runs on `stream`, copies the outputs back
 * and synchronises `stream` before returning.  Mixing host and device grids in
 * one call is allowed.  The caller owns every pointer it passes; the library
 * keeps none of them after the call returns.
 *
 * Workspace: the library owns a small per-(device, stream) workspace
 * (reduction partials, status words, one grid-sized ping-pong buffer for the
 * solvers), allocated on first use and reused; stencil_release_workspace()
 * frees it.  Calls on the same stream are ordered; calls on different streams
 * use different workspaces.
 *
 * ------------------------------------------------------------------ errors ---
 * Every entry point returns an int status.  It never aborts, exits or traps.
 * On a negative status nothing asynchronous was left running by the call;
 * outputs are unspecified.  stencil_last_error() gives a message for the last
 * failing call on the calling thread.  Extents are accepted up to 2^28 each,
 * but a 3-D kernel launch holds at most 65535 tiles of rows (j) and 65535
 * chunks of planes (k).  The sweeps, norms, solvers and advection return
 * STN_EINVAL, before launching anything, for extents beyond that: ny above
 * 65535 times the kernel's tile height (4 to 64 rows, so from 262140 rows
 * up), or nz above 65535 chunks of 64 planes for advection.
 * stencil_plan_query tells in advance for the sweeps.
 */
#ifndef STENCIL_H_
#define STENCIL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  STN_OK = 0,             /* success */
  STN_NOT_CONVERGED = 1,  /* solver: result valid, tolerance not reached */
  STN_EINVAL = -1,        /* bad argument: NULL, extent < 1, radius not 1/2, iters < 0,
                             in == out or overlapping, unsupported pointer kind */
  STN_ENOMEM = -2,        /* device or host allocation failed */
  STN_ECUDA = -3,         /* a CUDA runtime call failed (message in stencil_last_error) */
  STN_ETIMEOUT = -4,      /* a device-side wait reached its spin limit */
  STN_EBUSY = -5,         /* admission refused (server over its memory budget) */
  STN_PENDING = 2         /* server: request not finished yet */
};

/* Result of a solve (host struct filled by the solvers). */
typedef struct stn_solve_info {
  int64_t iters;     /* sweeps performed (inner float sweeps for the refined solver) */
  int64_t outer;     /* refinement steps (0 for plain Jacobi) */
  double rel_res;    /* last measured ||rho||/||rhs|| (absolute ||rho|| if ||rhs|| = 0) */
  double res_norm;   /* last measured ||rho||_2 */
  double rhs_norm;   /* ||rhs||_2 over the interior */
  int status;        /* STN_OK or STN_NOT_CONVERGED */
} stn_solve_info;

/* Message for the last failing call on this thread ("" if none). */
const char* stencil_last_error(void);

/* Library version string. */
const char* stencil_version(void);

/* Frees every workspace the library holds on the current device.  Returns
 * STN_OK, or STN_ECUDA.  Not safe while calls are in flight on that device. */
int stencil_release_workspace(void);

/*
 * stencil_tune_set / stencil_tune_get -- process-wide kernel-selection knobs
 * (no paper counterpart; the paper's own tuning is compile-time, Sec. 6).
 *   "star_variant": -1 automatic (default: for float grids of at least 3e7
 *                   points 3, else 1 at radius 1 and 2 at radius 2; 0 for
 *                   double),
 *                   0 shared-memory plane kernel (one point per thread),
 *                   1 register/shuffle column kernel (8 j rows per thread,
 *                   no shared memory), 2 plane kernel taking two k planes
 *                   per step (more independent work per thread), 3 staged
 *                   kernel (whole rows of a block's planes stream through a
 *                   shared-memory ring filled by asynchronous 16-byte copies;
 *                   grids whose rows are too long for the ring use another).
 *   "star_chunks":  0 automatic (default: the tuning cache's entry, else the
 *                   built-in plan), else the number of k chunks each
 *                   column of tiles is split into (one block per tile and
 *                   chunk; clamped to chunks of >= 4 planes).  Changes the
 *                   grid, never the iterates; the residual's partial sums
 *                   follow the grid, so its last bits may change.
 *   "repeat_graph": 1 (default): sweep loops of grids up to 2^22 points and at
 *                   least 16 sweeps (stencil_sweep_*, varcoef_sweep_*, the
 *                   refined solver's inner sweeps) run as a CUDA graph whose
 *                   while node repeats 16 sweeps on the device; 0: one stream
 *                   launch per sweep.  Same kernels, same results.
 *   "var_chunks":   k chunks per tile column of the TMA-staged variable-
 *                   coefficient sweep (0 = planned: about six waves of
 *                   blocks).  Changes the grid, never the results.
 *   "refined_engine": jacobi_solve_refined_f64: 1 (default) full-grid kernels
 *                   per step; 0 a batch of one in the persistent scheduler.
 *   "var_variant":  variable-coefficient kernels: -1 automatic (default: float
 *                   radius-2 sweeps on grids whose padded rows are a multiple
 *                   of 16 bytes, with u, a and f 16-byte and out 8-byte
 *                   aligned, and at least four waves of its blocks, take the
 *                   TMA-staged kernel; everything else the
 *                   register/shuffle column kernel that computes each face
 *                   coefficient once), 0 the shared-memory plane kernel, 1
 *                   column, 2 TMA-staged where it applies (column elsewhere).
 *                   Bitwise the same results (face coefficients in the normal
 *                   floating-point range).
 *   "sweep2d_resident": 2-D sweeps: -1 automatic (default: shared-memory
 *                   resident whenever the grid fits), 0 always through HBM,
 *                   1 resident whenever it fits.
 *   "sweep2d_chunk": most sweeps per resident 2-D launch (default 32768;
 *                   longer runs take several launches).
 *   "sweep2d_ctas_per_sm": resident 2-D bands per SM, 1 (default) to 4; fewer
 *                   when their shared memory does not fit (1024^2 double: 2 at
 *                   most).  Same results.
 *   "sweep2d_tma":  resident 2-D sweeps fetch the neighbours' rows by bulk
 *                   copy when a row's interior is a multiple of 16 bytes (1,
 *                   default) or always through registers (0).
 *   "temporal_depth": sweeps fused per pass over HBM in stencil_sweep_*
 *                   (temporal blocking): 0 automatic (the tuning cache's
 *                   entry for the extents, else 1), 1 off, 2..4 (double
 *                   radius 2: at most 3).
 *   "solve_graph":  jacobi_solve_f64 iterates inside a CUDA graph whose while
 *                   node repeats {check_every sweeps, device-side convergence
 *                   decision} with no host round trip (1, default), or in a
 *                   host loop that reads the residual every check (0).
 *   "batch_engine": batched solvers: 0 dynamic work-unit scheduler (default:
 *                   any CTA may take any unit of any problem in flight),
 *                   1 one thread-block cluster per problem, 2 a pool of
 *                   eight worker streams taking the problems largest first,
 *                   each solved as jacobi_solve_f64 / jacobi_solve_refined_f64
 *                   solve it alone (full-grid or resident kernels).
 *   "resident3d":   1 (default): sweep loops of at least two sweeps over 3-D
 *                   grids of at most 2^18 interior points (stencil_sweep_*,
 *                   a solve's group of sweeps, the refined solver's inner
 *                   loop, when no kernel variant, chunk count or tuning-cache
 *                   entry is forced) run in one cooperative launch, sweeps
 *                   separated by a bounded grid barrier; 0: per-sweep kernels.
 *                   Same results.
 *   "fp64_double_word": 0 (default): double sweeps take the canonical
 *                   update.  1: radius-1 double sweeps without source term or
 *                   centre coefficient evaluate the update in double-word
 *                   float arithmetic on the FP32 pipe (error per sweep at most
 *                   40 * 2^-48 of the largest |u| next to the point; NOT
 *                   bitwise; points next to values outside the float split's
 *                   range take the canonical update).
 *   "batch_graph":  the batch scheduler's persistent launch as a CUDA graph
 *                   captured and launched on the call's stream (1, default;
 *                   a failure to capture falls back to a plain launch), or a
 *                   plain launch (0).  Same kernel, same results.
 * Every variant, depth and engine computes bitwise the same iterates (with a
 * fixed number of inner sweeps, for refined solves; with inner_tol > 0 the
 * engines' inner stopping sums may round differently).
 * Limits and host-side fault injection (for tests of failure handling; no
 * GPU fault is ever caused):
 *   "sched_idle_ms": batched scheduler idle limit (default 2000 ms); CTAs
 *                   that find no work for this long end the launch with
 *                   STN_ETIMEOUT.
 *   "fault_withhold_last": 1 = batched scheduler never queues the last
 *                   problem, so the launch times out (STN_ETIMEOUT).
 *   "fault_withhold_2d": 1 = the last band of a resident 2-D sweep never
 *                   publishes its rows, so its neighbour's wait runs out and
 *                   the call returns STN_ETIMEOUT.
 *   "fault_withhold_3d": 1 = the last block of the next resident 3-D sweep
 *                   launches never arrives at the grid barrier, so the other
 *                   blocks' bounded waits run out and the next synchronising
 *                   call on the stream returns STN_ETIMEOUT.
 *   "fault_admit_fail": the server's next N admission allocations fail
 *                   (retried later, like a busy pool); "fault_admit_failed"
 *                   (read only) counts the injected failures.
 * Read only, per calling thread: "last_star_variant" and "last_star_chunks"
 * (kernel variant and k chunks of the last star-kernel launch),
 * "last_temporal_depth" (depth used by the last stencil_sweep_* call).  Not thread-safe against
 * concurrent launches.  Unknown knob or value: STN_EINVAL.
 */
int stencil_tune_set(const char* knob, int64_t value);
/* Counters of the last batched/served scheduler launch in this process
 * (summed over CTAs): cycles claiming, computing units, completing units, in
 * pass epilogues, idle; units; epilogues; empty claim scans; units claimed
 * on the slot and pass of the CTA's previous unit; claim atomics issued by
 * slot scans.  Returns the number of counters written (at most n). */
int stencil_sched_stats(uint64_t* out, int n);
int stencil_tune_get(const char* knob, int64_t* value);

/*
 * Autotuner and tuning cache for the star sweeps (stencil_sweep_*,
 * stencil_apply_*, residual_norm_*, jacobi_solve_f64; no paper counterpart:
 * the paper's loop tiling and unrolling are compile-time passes, Sec. 6 and
 * 6.1, where this picks tile shapes by timing them).  One entry per (device name, element
 * size, radius, nx, ny, nz) holds the kernel variant (the tile shape: 0 the
 * 32 x 8 plane kernel, 1 the 30 x 32-row column kernel, 2 the plane kernel
 * taking two planes per step, 3 the staged kernel's whole-row blocks), the
 * k chunks each tile column is split into,
 * and the temporal depth (sweeps fused per pass over HBM, 1 = none).  When
 * the "star_variant", "star_chunks" and "temporal_depth" knobs are automatic,
 * a call on grids of those extents uses the entry; with no entry the built-in
 * plan applies.  Every configuration computes bitwise the same iterates;
 * residual norms may differ in their last bits (their partial sums follow
 * the grid).  Changing the cache while calls on the same extents are in
 * flight is not safe (like the knobs).
 */
typedef struct stn_tune_entry {
  char device[64];        /* device name the entry applies to ("" = the current device's) */
  int64_t nx, ny, nz;     /* interior extents */
  int32_t esize;          /* element bytes: 8 double, 4 float */
  int32_t radius;         /* 1 or 2 */
  int32_t variant;        /* 0, 1, 2 or 3 (see above) */
  int32_t chunks;         /* k chunks per tile column, >= 1 */
  int32_t depth;          /* temporal depth 1..4 */
  int32_t reserved;
  double glups;           /* measured rate of this configuration (0 if set by hand) */
  double default_glups;   /* measured rate of the built-in plan */
} stn_tune_entry;

/* Times the candidate configurations for sweeps of these extents on two
 * scratch grids the call allocates (2 x (nx+2r)(ny+2r)(nz+2r) x esize bytes of
 * device memory, zero-filled, freed before return) on the current device and
 * `stream`: every kernel variant at k-chunk counts around the built-in plan
 * (its own, half, twice and four times it, and the counts giving 2, 4, 6, 8
 * and 16 blocks per SM), and temporal depths 2..4; each candidate runs 12 sweeps (`trial_sweeps` > 0 overrides) after
 * two untimed ones, timed by CUDA events, in two rounds (the faster round
 * counts).  The fastest configuration is stored in the cache and copied to
 * *best; the built-in plan is kept unless another is more than 2 % faster.
 * coeffs: host array of radius+1 doubles, or NULL for {0, 1/6[, 0]}.
 * When the environment variable STN_TUNE_CACHE names a file, the cache is
 * written there after tuning.  Synchronises `stream`.
 * Errors: STN_EINVAL (bad extents, radius or esize, NULL best), STN_ENOMEM,
 * STN_ECUDA. */
int stencil_autotune_sweep(int64_t nx, int64_t ny, int64_t nz, int esize, int radius,
                           const double* coeffs, int trial_sweeps, stn_tune_entry* best, void* stream);
/* Adds or replaces an entry (device "" = the current device's name).
 * STN_EINVAL for bad extents, radius, esize, variant (0..3), chunks (1..65535)
 * or depth (1..4). */
int stencil_tune_cache_put(const stn_tune_entry* entry);
/* Looks up the entry for (device, extents, esize, radius); device NULL or ""
 * = the current device's name.  Returns 1 and fills *out when found, 0 when
 * not, STN_EINVAL on bad arguments.  The first lookup in a process loads
 * the file named by STN_TUNE_CACHE, if set and readable. */
int stencil_tune_cache_get(const char* device, int64_t nx, int64_t ny, int64_t nz, int esize, int radius,
                           stn_tune_entry* out);
/* Number of entries. */
int64_t stencil_tune_cache_size(void);
/* Removes every entry. */
int stencil_tune_cache_clear(void);
/* Writes every entry to `path` as JSON ({"stencil_tune_cache": 1, "entries":
 * [{...}, ...]}, one entry per line).  STN_EINVAL for a NULL path or a file
 * that cannot be written (the reason in stencil_last_error). */
int stencil_tune_cache_save(const char* path);
/* Reads entries written by stencil_tune_cache_save and adds them (replacing
 * entries with the same key).  Returns the number of entries read (>= 0), or
 * STN_EINVAL for a NULL path, an unreadable file or a malformed entry (then
 * nothing is added). */
int stencil_tune_cache_load(const char* path);

/* The launch one sweep of these extents would make on the current device,
 * computed on the host by the same planners the sweeps use (the knobs and the
 * tuning cache apply); nothing is launched or allocated.  Without a device
 * the planners assume 152 SMs and a fixed number of resident blocks per SM.
 * op: "sweep" (stencil_sweep_f64/_f32: variant as the star_variant knob,
 * 0..3), "varcoef_sweep" (the variable-coefficient sweep: variant 0 the
 * plane kernel, 1 the column kernel), "sweep2d" (stencil_sweep2d_f64/_f32,
 * nz = 1: variant 1 the shared-memory-resident kernel, 0 one launch per
 * sweep) or "batch_unit" (how the batched solvers and the server split one
 * problem into work units, radius-independent: variant = tile shape, 0
 * 32 x 8, 1 16 x 16, 2 8 x 32 columns; grid_x x grid_y tiles times grid_z
 * chunks of kchunk planes are the units; stage_elems = the elements of the
 * shared plane every shape fits; extents at most 2^20).  Block (x, y, z) covers the interior columns [x tile_w,
 * (x+1) tile_w), rows [y tile_h, (y+1) tile_h) and planes [z kchunk,
 * (z+1) kchunk), clipped to the grid; the per-sweep 2-D kernel loops over
 * its 32 x 8 tiles with grid_x blocks, and the resident one gives band b the
 * rows [b ny / grid_x, (b+1) ny / grid_x), at most tile_h.  The staged kernel
 * (variant 3 of "sweep") streams whole rows through a ring of 2r+2 stages of
 * stage_elems elements, smem_bytes of dynamic shared memory in all.  The
 * resident 2-D kernel keeps two copies of its band's rows with row stride
 * row_stride elements, padded column c at row_pad + c; bulk_copy = 1 when
 * the halo rows arrive by bulk copy; it needs scratch_bytes of global scratch
 * with the exchange slots from xchg_offset on.
 * Errors: STN_EINVAL (NULL op or out, unknown op, bad extents, esize or
 * radius, or a plan beyond CUDA's launch-grid limits: the sweep itself
 * rejects those extents the same way). */
typedef struct stn_launch_plan {
  int32_t variant;
  int32_t grid_x, grid_y, grid_z; /* blocks */
  int32_t block_threads;
  int32_t tile_w, tile_h;         /* interior columns (i) and rows (j) per block */
  int32_t kchunk;                 /* interior planes per block */
  int32_t stage_elems;            /* staged kernel: elements per ring stage, else 0 */
  int32_t smem_bytes;             /* dynamic shared memory per block */
  int32_t row_stride, row_pad;    /* resident 2-D kernel: shared-memory row layout, else 0 */
  int32_t bulk_copy;              /* resident 2-D kernel: halo rows by bulk copy (1) or not (0) */
  int32_t reserved;
  int64_t scratch_bytes;          /* resident 2-D kernel: global scratch, else 0 */
  int64_t xchg_offset;            /* resident 2-D kernel: offset of the exchange slots in it */
} stn_launch_plan;
int stencil_plan_query(const char* op, int64_t nx, int64_t ny, int64_t nz, int esize, int radius,
                       stn_launch_plan* out);

/*
 * stencil_sweep_f64 / _f32 -- `iters` Jacobi sweeps of the constant-
 * coefficient star stencil (no source term).  Sec. 4 (the benchmark repeats
 * the sweep a fixed number of iterations).
 *   in      grid holding the starting iterate (its halo is the boundary);
 *           its INTERIOR is clobbered when iters > 1 (used as the ping-pong
 *           buffer); unchanged when iters <= 1.
 *   out     grid receiving the result: interior = iterate number `iters`,
 *           halo = in's halo.  iters == 0 copies in to out.
 *   coeffs  host, radius+1 doubles {c0, c1[, c2]}.
 *   radius  1 or 2.
 *   iters   >= 0.
 * Errors: STN_EINVAL (NULL grid or coeffs, extents < 1, radius not 1/2,
 * iters < 0, in and out overlap), STN_ENOMEM, STN_ECUDA.
 */
int stencil_sweep_f64(double* in, double* out, int64_t nx, int64_t ny, int64_t nz,
                      const double* coeffs, int radius, int64_t iters, void* stream);
int stencil_sweep_f32(float* in, float* out, int64_t nx, int64_t ny, int64_t nz,
                      const double* coeffs, int radius, int64_t iters, void* stream);

/*
 * stencil_apply_f64 / _f32 -- ONE application of the star stencil (the
 * stencil.apply of Sec. 2.2): out = S u + b on the interior, one kernel
 * launch, asynchronous on `stream`.  The halo of `out` is not written.
 *   u       grid (read only); b: source grid or NULL (read only).
 *   out     grid; must not overlap u or b.  Device memory only (no staging).
 * Errors: STN_EINVAL (NULL u/out/coeffs, bad extents/radius, overlap, a host
 * pointer), STN_ECUDA.
 */
int stencil_apply_f64(const double* u, const double* b, double* out, int64_t nx, int64_t ny,
                      int64_t nz, const double* coeffs, int radius, void* stream);
int stencil_apply_f32(const float* u, const float* b, float* out, int64_t nx, int64_t ny,
                      int64_t nz, const double* coeffs, int radius, void* stream);

/*
 * residual_norm_f64 / _f32 -- ||rho||_2 with rho = (S u + b) - u over the
 * interior, i.e. the change one more sweep would make (Sec. 5.3, Listing 8:
 * sum reduction from zero with an add combiner, here of rho^2, accumulated in
 * double in a fixed order that depends only on the extents, then sqrt).
 *   u         grid (read only).
 *   b         grid of the source term, or NULL for none (read only; its halo
 *             is not read).
 *   norm_out  HOST double receiving the norm.  The call synchronises `stream`.
 * For _f32 the stencil value is computed in float; rho and its square in
 * double.
 * Errors: STN_EINVAL (NULL u/coeffs/norm_out, bad extents or radius),
 * STN_ENOMEM, STN_ECUDA.
 */
int residual_norm_f64(const double* u, const double* b, int64_t nx, int64_t ny, int64_t nz,
                      const double* coeffs, int radius, double* norm_out, void* stream);
int residual_norm_f32(const float* u, const float* b, int64_t nx, int64_t ny, int64_t nz,
                      const double* coeffs, int radius, double* norm_out, void* stream);

/*
 * residual_norm_f64_noalloc -- residual_norm_f64 for callers that may not let
 * the library allocate memory (the paper has no counterpart: this is a
 * deployment variant).  Such callers include serving processes that have
 * already given their whole device-memory budget to their own pools, code
 * that must not call cudaMalloc because it can synchronise the device and
 * stall the process's other streams, and loops that have no way to report an
 * allocation failure.  This call allocates nothing: its scratch (up to 65536
 * per-block partial sums plus a few result slots, 512 KiB in all) is a fixed
 * array in the library's device image, which every GPU that loads the library
 * holds until the process exits.
 *   u, b      DEVICE grids only (host grids: STN_EINVAL, no staging).
 *   norm_out  HOST double receiving the norm; the call synchronises `stream`.
 * Same result as residual_norm_f64 (same kernels, same fixed reduction
 * order).  Grids whose launch plan needs more than 65536 partial sums (one
 * per 64 x 8 or 32 x 8 tile of the (i, j) plane once the plane has enough
 * tiles to fill the GPU: nx*ny above roughly 17 to 34 million, e.g.
 * 8192 x 8192) are rejected with STN_EINVAL before any GPU work.  The limit
 * is checked against the very plan the call then launches and reduces (formed
 * once per call), so a tuning knob or tuning-cache entry set meanwhile on
 * another host thread cannot push a launch past the array.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) for that device; make that first call before any
 * stream capture.  Every call on a device shares the one array: calls that
 * overlap on the GPU (other streams, other host threads) race and must be
 * ordered by the caller.  Each call writes every scratch slot it reads, so no
 * state carries over from one call to the next.
 */
int residual_norm_f64_noalloc(const double* u, const double* b, int64_t nx, int64_t ny,
                              int64_t nz, const double* coeffs, int radius, double* norm_out,
                              void* stream);

/*
 * jacobi_solve_f64 -- solve u = S u + rhs by Jacobi iteration (Sec. 4).
 * Sweeps run in groups of `check_every` (>= 1); the last sweep of each group
 * is fused with the residual reduction of the iterate it starts from.  The
 * solve stops after the first group whose measured ||rho|| <= tol*||rhs||
 * (absolute ||rho|| <= tol when ||rhs|| = 0 or rhs == NULL), or after
 * max_iters sweeps.
 *   rhs       grid of the source term b (read only), or NULL for b = 0.
 *   u         in: initial guess and Dirichlet halo; out: the last iterate
 *             (one sweep past the iterate whose residual was measured).
 *   info      HOST, filled on return (may be NULL).
 * The call synchronises `stream`.  Returns STN_OK, STN_NOT_CONVERGED, or an
 * error (STN_EINVAL for tol < 0, max_iters < 0, check_every < 1, ...).
 */
int jacobi_solve_f64(const double* rhs, double* u, int64_t nx, int64_t ny, int64_t nz,
                     const double* coeffs, int radius, double tol, int64_t max_iters,
                     int64_t check_every, stn_solve_info* info, void* stream);

/*
 * jacobi_solve_refined_f64 -- mixed-precision iterative refinement of
 * u = S u + rhs (not in the paper; double only for the residual and the
 * update):
 *   outer (double): t = S u + rhs, rho = t - u; stop if ||rho|| <= tol*||rhs||
 *                   (absolute if ||rhs|| = 0); s = max|rho|; r32 = float(rho/s)
 *   inner (float) : sweeps of e = S e + r32 from e = 0 (coefficients rounded to
 *                   float), in groups of check_every; stop after a group whose
 *                   last sweep changed e by <= inner_tol*||r32|| (inner_tol = 0:
 *                   never), or after inner_sweeps sweeps
 *   update(double): u = u + s * double(e)
 * up to max_outer outer steps.  info->outer = outer steps, info->iters =
 * float sweeps, info->rel_res = last double relative residual.  The steps
 * run as full-grid kernels (the double sweep with its fused residual, the
 * float sweeps of stencil_sweep_f32, small grids' inner loops as
 * device-repeated CUDA graphs); knob "refined_engine" = 0 runs the request as
 * a batch of one in the persistent scheduler instead (same arithmetic; with
 * inner_tol > 0 the inner stopping sums may round differently).  Device or
 * host grids.  Synchronises.  Returns STN_OK or STN_NOT_CONVERGED.
 */
int jacobi_solve_refined_f64(const double* rhs, double* u, int64_t nx, int64_t ny, int64_t nz,
                             const double* coeffs, int radius, double tol, int64_t inner_sweeps,
                             double inner_tol, int64_t check_every, int64_t max_outer,
                             stn_solve_info* info, void* stream);

/*
 * Batched solves: many independent problems of different extents (a C4-style
 * batch) in ONE persistent kernel launch (captured in a CUDA graph and
 * launched on `stream`; knob "batch_graph").  By default (knob
 * "batch_engine" = 0) a dynamic work-unit scheduler runs one wave of CTAs:
 * up to 96 problems are in flight at a time, largest estimated work first;
 * each problem advances pass by pass (a sweep, a residual sweep or a
 * refinement step), a pass is split into units (a tile of columns times a
 * chunk of 128-256 planes, from the extents alone) that any CTA claims, and
 * the CTA that completes a pass's last unit reduces its partials in unit
 * order and publishes the next pass.  Every sweep is the single-problem
 * path's canonical update and every reduction has a fixed order, so each
 * result is bitwise independent of the rest of the batch.  Engine 1 gives
 * each problem one thread-block cluster (sweeps separated by the cluster's
 * barrier), engine 2 a pool of worker streams running the one-problem
 * solves; both give the same iterates.
 *   probs   HOST array of `count` problems; their grids are DEVICE memory, each
 *           its own (problems must not share or overlap grids).
 *   infos   HOST array of `count` results (may be NULL).
 * Extents are at most 2^20 per axis and a problem at most 2^22 units per pass
 * (STN_EINVAL otherwise); a batch whose scratch exceeds any device's memory
 * returns STN_ENOMEM before any allocation.  The library allocates the
 * scratch grids of the batch (stream-ordered) and frees them before
 * returning.  Synchronises `stream`.  Returns STN_OK when every problem
 * converged, STN_NOT_CONVERGED when one did not, STN_ETIMEOUT when the
 * scheduler's CTAs found no work for the idle limit (a lost unit; never
 * expected), or an error.
 */
typedef struct stn_problem {
  int64_t nx, ny, nz;  /* interior extents */
  const double* rhs;   /* source term grid (device), or NULL */
  double* u;           /* initial guess in, last iterate out (device) */
} stn_problem;

/* Plain double Jacobi for each problem; same stopping rule as jacobi_solve_f64. */
int jacobi_solve_batched_f64(const stn_problem* probs, int64_t count, const double* coeffs,
                             int radius, double tol, int64_t max_iters, int64_t check_every,
                             stn_solve_info* infos, void* stream);

/* Refinement of jacobi_solve_refined_f64 for each problem. */
int jacobi_solve_batched_refined(const stn_problem* probs, int64_t count, const double* coeffs,
                                 int radius, double tol, int64_t inner_sweeps, double inner_tol,
                                 int64_t check_every, int64_t max_outer, stn_solve_info* infos,
                                 void* stream);

/*
 * Serving loop (continuous batching; not in the paper).  A server owns a
 * device-memory budget.  Requests (one Poisson/Jacobi solve u = S u + rhs
 * each, extents per request) are submitted at any time from any thread; the
 * server admits them in arrival order as their grids fit in the budget, runs
 * the admitted requests concurrently on the GPU, and hands back the
 * solution.  Two engines:
 *   0  a persistent scheduler kernel: every admitted request's passes are
 *      split into work units that any CTA claims; requests admitted while
 *      others run join the running kernel.  Its results are those of
 *      jacobi_solve_batched_refined / _f64 on the request alone.
 *   1  max_inflight worker streams: each takes the oldest admitted request,
 *      runs it with the full-grid kernels of jacobi_solve_refined_f64 (or
 *      jacobi_solve_f64 when not refined) and takes the next; the kernels of
 *      different requests overlap on the device.  Its results are those of
 *      jacobi_solve_refined_f64 / jacobi_solve_f64 on the request alone.  The
 *      budget counts each running request's grids and scratch (3 double and,
 *      refined, 3 float grids); each worker also keeps 2 MiB of reduction
 *      slots and a few scalars outside it.
 * A result depends only on its request: it is the same alone and in any mix
 * of concurrent requests.
 */
typedef struct stn_server stn_server;

typedef struct stn_server_opts {
  size_t hbm_budget;       /* bytes of device memory for request grids and scratch */
  int radius;              /* 1 or 2 */
  double coeffs[3];        /* {c0, c1, c2}; entries beyond radius ignored */
  double tol;              /* stop at ||rho|| <= tol*||rhs|| (as jacobi_solve_f64) */
  int refined;             /* 1: float sweeps + double refinement; 0: double Jacobi */
  int64_t max_iters;       /* plain: sweep limit */
  int64_t inner_sweeps;    /* refined: float sweep limit per outer step */
  double inner_tol;        /* refined: inner stop (0 = run inner_sweeps) */
  int64_t check_every;     /* sweeps per convergence check */
  int64_t max_outer;       /* refined: outer step limit */
  int max_inflight;        /* requests on the GPU at once (engine 1: worker streams, <= 64) */
  int queue_capacity;      /* engine 0: admitted-but-unfinished requests the device queue holds */
  int engine;              /* 0: the persistent work-unit scheduler kernel;
                              1: a pool of max_inflight worker streams, each running one
                                 request at a time on the full-grid kernels (the steps of
                                 jacobi_solve_refined_f64 / jacobi_solve_f64) */
} stn_server_opts;

typedef struct stn_request {
  int64_t nx, ny, nz;      /* interior extents */
  const double* rhs;       /* HOST padded grid (copied at submit) */
  const double* u0;        /* HOST padded initial guess and halo, or NULL for zeros */
} stn_request;

typedef struct stn_result {
  stn_solve_info info;
  double latency_s;        /* submit -> result ready */
  double queue_s;          /* submit -> admitted to the GPU */
  int rc;                  /* STN_OK, STN_NOT_CONVERGED or an error */
} stn_result;

typedef struct stn_server_stats_t {
  int64_t submitted, completed, pending, running;
  size_t bytes_in_use;
  int status;              /* STN_OK, or the error that stopped the server */
} stn_server_stats_t;

/* Creates a server on the current device (NULL on error; see
 * stencil_last_error). */
stn_server* stn_server_create(const stn_server_opts* opts);
/* Submits a request; *ticket identifies it.  STN_EBUSY if it can never fit in
 * the budget or the server is stopping. */
int stn_submit(stn_server* s, const stn_request* req, uint64_t* ticket);
/* STN_PENDING while the request runs; else fills *res (may be NULL) and returns
 * STN_OK (the solve's own status is in res->info.status / res->rc). */
int stn_poll(stn_server* s, uint64_t ticket, stn_result* res);
/* Waits up to timeout_s seconds (negative: forever); STN_ETIMEOUT if it did not
 * finish in time. */
int stn_wait(stn_server* s, uint64_t ticket, double timeout_s, stn_result* res);
/* Copies a finished request's solution (padded grid) to HOST memory u_out. */
int stn_result_copy(stn_server* s, uint64_t ticket, double* u_out);
/* Forgets a finished request (frees its host copy). */
int stn_release(stn_server* s, uint64_t ticket);
int stn_server_stats(stn_server* s, stn_server_stats_t* stats);
/* Stops accepting requests, finishes the ones submitted, frees everything. */
void stn_server_destroy(stn_server* s);

/*
 * Variable-coefficient operator, radius R in {1, 2}, weights w[0..R] (HOST;
 * w[0] unused), per-point coefficient field a on the full padded grid:
 *   (A u)(p) = sum_{d=1..R} w_d sum_{q = p +- d e_x, e_y, e_z} kappa(p,q) (u(p) - u(q)),
 *   kappa(p,q) = (a(p) + a(q)) / 2.
 * With D(p) = sum w_d kappa and N(p) = sum w_d kappa u(q), both accumulated
 * over d = 1..R, then axes x, y, z, minus neighbour before plus neighbour:
 *   Jacobi update  u'(p) = (f(p) + N(p)) / D(p);   (A u)(p) = D(p) u(p) - N(p).
 * The paper states only Laplace's equation (Sec. 4); this symmetric
 * M-matrix form is the reading used for the variable-coefficient Poisson
 * workload (a ~ U[0.5,1.5], w = {-, 1, 1/4}).
 */

/* out = A u on the interior; the halo of out is not written. */
int varcoef_apply_f64(const double* u, const double* a, double* out, int64_t nx, int64_t ny,
                      int64_t nz, const double* w, int radius, void* stream);

/* `iters` Jacobi sweeps for A u = f; in/out semantics as stencil_sweep_f64
 * (in's interior clobbered when iters > 1).  _f32 takes float a, f, grids;
 * weights rounded to float.  Float sweeps of radius 2 whose padded rows are
 * a multiple of 16 bytes (nx + 4 divisible by 4), with 16-byte-aligned in,
 * out (both serve as u), a and f, stage their tiles
 * through shared memory by tensor-map copies (TMA); the results are the same
 * bits as every other variant.  Their device-side waits are bounded: a wait
 * that gave up (never expected) stops that sweep early and is reported as
 * STN_ETIMEOUT by the next synchronising variable-coefficient call on the
 * device (residual norm, solves). */
int varcoef_sweep_f64(double* in, double* out, const double* a, const double* f, int64_t nx,
                      int64_t ny, int64_t nz, const double* w, int radius, int64_t iters,
                      void* stream);
int varcoef_sweep_f32(float* in, float* out, const float* a, const float* f, int64_t nx,
                      int64_t ny, int64_t nz, const double* w, int radius, int64_t iters,
                      void* stream);

/* ||f - A u||_2 over the interior, in double (host result; synchronises). */
int varcoef_residual_norm_f64(const double* u, const double* a, const double* f, int64_t nx,
                              int64_t ny, int64_t nz, const double* w, int radius,
                              double* norm_out, void* stream);

/* Plain double Jacobi solve of A u = f, same grouping/stopping rule as
 * jacobi_solve_f64 with rho = f - A u.  Synchronises. */
int jacobi_solve_varcoef_f64(const double* a, const double* f, double* u, int64_t nx, int64_t ny,
                             int64_t nz, const double* w, int radius, double tol,
                             int64_t max_iters, int64_t check_every, stn_solve_info* info,
                             void* stream);

/*
 * jacobi_solve_varcoef_refined -- mixed-precision iterative refinement for
 * A u = f (not in the paper; double kept only for the residual and update):
 *   outer (double): rho = f - A u; stop if ||rho||/||f|| <= tol;
 *                   s = max|rho|; r32 = float(rho / s)
 *   inner (float) : `inner_sweeps` Jacobi sweeps on A e = r32 from e = 0
 *                   (a and w rounded to float once per call)
 *   update(double): u = u + s * double(e)
 * up to max_outer outer steps.  info->outer = outer steps, info->iters =
 * total float sweeps, info->rel_res = the last double relative residual.
 * Synchronises.  Returns STN_OK or STN_NOT_CONVERGED.
 */
int jacobi_solve_varcoef_refined(const double* a, const double* f, double* u, int64_t nx,
                                 int64_t ny, int64_t nz, const double* w, int radius, double tol,
                                 int64_t inner_sweeps, int64_t max_outer, stn_solve_info* info,
                                 void* stream);

/*
 * ---------------------------------------------------------------------------
 * Two-dimensional grids: the paper's own jacobi benchmark (Sec. 4: a Jacobi
 * iteration for Laplace's equation on one 2-D 1024 x 1024 grid, 100000
 * iterations).  A 2-D grid is a padded (ny+2r) x (nx+2r) array with i fastest
 * (the Fortran array u(1:nx+2r, 1:ny+2r), Sec. 5.2 indexing), the same
 * Dirichlet halo as the 3-D grids.  Canonical order of one update:
 *     S_d = (u[i-d]+u[i+d]) + (u[j-d]+u[j+d]);  acc = c_r*S_r;
 *     acc = acc + c_d*S_d (d = r-1..1);  acc = acc + c0*u if c0 != 0;
 *     acc = acc + b if b is given.
 * With c = {0, 1/4} and r = 1 this is the 5-point Laplace Jacobi update.
 *
 * stencil_sweep2d_f64 / _f32 -- `iters` 2-D Jacobi sweeps (no source term).
 *   in      grid holding the starting iterate (its halo is the boundary).
 *           Grids that fit in the SMs' shared memory (1024 x 1024 doubles
 *           does) are swept there, one band of rows per SM, and `in` is not
 *           modified; larger grids are swept through HBM and `in`'s interior
 *           is clobbered when iters > 1.
 *   out     receives the result: interior = iterate number `iters`, halo =
 *           in's halo.  iters == 0 copies in to out.
 *   coeffs  host, radius+1 doubles {c0, c1[, c2]}; radius 1 or 2.
 * Device or host grids.  The call synchronises `stream`.
 * Errors: STN_EINVAL (NULL grid or coeffs, extents < 1 or > 2^28, radius not
 * 1/2, iters < 0, in and out overlap), STN_ENOMEM, STN_ECUDA, STN_ETIMEOUT (a
 * band's device-side wait for its neighbour's rows gave up after 2 s; the
 * context stays usable, `out` is undefined).
 */
int stencil_sweep2d_f64(double* in, double* out, int64_t nx, int64_t ny, const double* coeffs,
                        int radius, int64_t iters, void* stream);
int stencil_sweep2d_f32(float* in, float* out, int64_t nx, int64_t ny, const double* coeffs,
                        int radius, int64_t iters, void* stream);

/*
 * residual_norm2d_f64 / _f32 -- ||rho||_2, rho = (S u + b) - u over the 2-D
 * interior (the Sec. 5.3 add-reduction of rho^2 in double, fixed order for
 * given extents, then sqrt).  b may be NULL.  norm_out is a HOST double; the
 * call synchronises `stream`.  For _f32 the stencil value is float, rho and
 * its square double.  Errors as residual_norm_f64.
 */
int residual_norm2d_f64(const double* u, const double* b, int64_t nx, int64_t ny,
                        const double* coeffs, int radius, double* norm_out, void* stream);
int residual_norm2d_f32(const float* u, const float* b, int64_t nx, int64_t ny,
                        const double* coeffs, int radius, double* norm_out, void* stream);

/*
 * reduce_sum_f64 / dot_f64 -- the Fortran `sum` and `dotproduct` intrinsics
 * (Sec. 5.4, Table 3: the sum of a 32768 x 32768 double array, the dot
 * product of two 134-million-element double vectors), i.e. the linalg.reduce
 * of Sec. 5.3 / Listing 8 with a zero initial value and an add combiner.
 *   x, y   n contiguous doubles, device or host, 8-byte aligned (read only);
 *          a 2-D array is summed as its n = nx*ny elements.
 *   n      >= 0 (n == 0 gives 0).
 *   out    HOST double receiving the result.  The call synchronises `stream`.
 * The order of the additions is fixed for given n and for the operands'
 * offsets modulo 16 bytes (blocked partial sums added in index order), so
 * the result is reproducible; it differs from a left-to-right sum only by
 * rounding (dot products use fused multiply-adds).
 * Errors: STN_EINVAL (NULL out or array with n > 0, n < 0, misaligned
 * pointer), STN_ENOMEM, STN_ECUDA.
 */
int reduce_sum_f64(const double* x, int64_t n, double* out, void* stream);
int dot_f64(const double* x, const double* y, int64_t n, double* out, void* stream);

/*
 * advect_f64 / _f32 -- multi-field advection, a synthetic stand-in for the
 * paper's pw-advection and tra-adv workloads (Sec. 4: fields carried by a
 * wind on 2048 x 1024 x 1024 and 1024 x 512 x 512 grids; the paper gives no
 * formulas).  Second-order centred flux-form advection of a field q by the
 * velocity (u, v, w) on a halo-1 grid (the 3-D layout above, radius 1); for
 * each axis a with velocity component V and interior point p:
 *     F- = (V(p-e)+V(p)) * (q(p-e)+q(p)),   F+ = (V(p)+V(p+e)) * (q(p)+q(p+e)),
 *     T_a = c_a * (F- - F+),                 s(p) = (T_x + T_y) + T_z,
 * each operation rounded separately in this order.  With c_a = 1/(4 h_a) this
 * is -div(V q) in flux form.
 *   u, v, w  velocity components (device grids, read only).
 *   q        NULL: the velocity components advect themselves (the pw-like
 *            case) and s[0..2] receive their tendencies; otherwise nq (1..6)
 *            fields, s[0..nq-1] their tendencies (the tra-adv-like case).
 *   s        output grids; only the interior is written.  Must not overlap
 *            any input or each other.
 *   c        host, 3 doubles {c_x, c_y, c_z}.
 * Device grids only.  Asynchronous on `stream`.
 * Errors: STN_EINVAL (NULL pointers, nq out of range, non-finite c, bad
 * extents, overlap, a host pointer), STN_ECUDA.
 */
int advect_f64(const double* u, const double* v, const double* w, const double* const* q, int nq,
               double* const* s, int64_t nx, int64_t ny, int64_t nz, const double* c, void* stream);
int advect_f32(const float* u, const float* v, const float* w, const float* const* q, int nq,
               float* const* s, int64_t nx, int64_t ny, int64_t nz, const double* c, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* STENCIL_H_ */
