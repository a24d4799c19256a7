// Internal declarations shared by the translation units of libstencil.so.
// Nothing here is part of the public ABI (include/stencil.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/stencil.h"

namespace stn {

using i64 = int64_t;

// Thread-local error message behind stencil_last_error().
void set_error(const std::string& msg);
void clear_error();

// Returns STN_ECUDA with a message when `e` is an error.
int cuda_fail(cudaError_t e, const char* what);

#define STN_CUDA_TRY(expr)                                  \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return ::stn::cuda_fail(_e, #expr); \
  } while (0)

// CUDA's limits on a launch grid: gridDim.x < 2^31, gridDim.y and .z <= 65535.
// A launcher whose plan would exceed them (extents with more than 65535 tiles
// of rows, or of k chunks) returns STN_EINVAL before launching anything.
inline int check_launch_grid(i64 gx, i64 gy, i64 gz) {
  if (gx < 1 || gy < 1 || gz < 1 || gx >= ((i64)1 << 31) || gy > 65535 || gz > 65535) {
    set_error("invalid argument: extents too large for one launch grid (more than 65535 row tiles or k chunks)");
    return STN_EINVAL;
  }
  return STN_OK;
}

// Geometry of one padded grid.
struct Grid {
  i64 nx, ny, nz;  // interior extents
  int r;           // halo width
  i64 NX() const { return nx + 2 * r; }
  i64 NY() const { return ny + 2 * r; }
  i64 NZ() const { return nz + 2 * r; }
  i64 count() const { return NX() * NY() * NZ(); }
  i64 interior() const { return nx * ny * nz; }
};

// Launch configuration of the z-streaming kernels: tiles of TX x TY columns,
// each block streams a chunk of `kchunk` planes.
struct ZPlan {
  int tiles_x, tiles_y, chunks;
  int kchunk;
  int variant = 0;
  // staged variant: interior rows per block, elements per ring stage, and
  // the dynamic shared memory of its ring
  int rg = 0, stage_elems = 0, smem = 0;
  i64 blocks() const { return (i64)tiles_x * tiles_y * chunks; }
};

// Per-(device, stream) workspace.
struct Workspace {
  double* partials = nullptr;  // per-block partial sums
  i64 partials_cap = 0;
  double* scalars = nullptr;   // small device scalars (norms, flags); 64 doubles
  void* grid = nullptr;        // ping-pong grid for solvers
  size_t grid_bytes = 0;
  void* grid2 = nullptr;       // second solver buffer (refinement)
  size_t grid2_bytes = 0;
  void* grid3 = nullptr;
  size_t grid3_bytes = 0;
  double* host_scalars = nullptr;  // pinned host mirror of scalars
};

// Lets the current device's default stream-ordered memory pool keep up to
// kPoolKeepBytes of freed memory instead of returning it to the driver at
// every synchronisation (its default), so the library's per-call
// allocations (host-grid staging, batch scratch, served requests) reuse
// mapped memory.  Once per device and process; the setting belongs to this
// process's CUDA context and ends with it.
constexpr unsigned long long kPoolKeepBytes = 16ull << 30;
void keep_pool_memory();

// Returns the workspace of the current device and `stream`, with at least
// `partials` partial slots and (if grid_bytes > 0) a grid buffer of that size.
int get_workspace(cudaStream_t stream, i64 partials, size_t grid_bytes, Workspace** ws);
int ensure_grid2(Workspace* ws, size_t bytes);
int ensure_grid3(Workspace* ws, size_t bytes);

// ---- constant-coefficient star stencil (sweep.cu) --------------------------
enum SweepMode { kSweep = 0, kSweepResidual = 1, kResidualOnly = 2 };

// Star-kernel variants: the shared-memory plane kernel (one point per
// thread), the shuffle/register column kernel, and the plane kernel taking
// two planes per step.
// The staged kernel: whole rows of a block's planes fetched into a
// shared-memory ring by asynchronous 16-byte copies.
enum StarVariant { kStarScalar = 0, kStarColumn = 1, kStarPlane2 = 2, kStarStaged = 3 };
// Shared-memory ring of a staged block: most of an SM's (one block per SM).
constexpr int kStagedSmemMax = 220 * 1024;
ZPlan plan_star(const Grid& g, int variant, size_t esize);
// Whether the staged kernel's ring fits for this grid (rows not too long).
bool staged_applicable(const Grid& g, size_t esize);
int star_variant(const Grid& g, size_t esize, const void* a, const void* b, const void* c);
// Tuning override of the variant choice (-1 = automatic).
int tune_set_star_variant(int v);
int tune_get_star_variant();
// A star-sweep configuration: kernel variant (-1 = not set), k chunks per
// tile column (0 = not set), temporal depth (0 = not set); no_cache makes
// the planners ignore the tuning cache.
struct StarChoice {
  int variant = -1;
  int chunks = 0;
  int depth = 0;
  bool no_cache = false;
};
// The configuration the autotuner forces on this thread while it times a
// candidate (takes precedence over the knobs and the cache).
StarChoice& star_force();
// The configuration of this thread's last star launch (variant, chunks) and
// last stencil_sweep call (depth): read through stencil_tune_get.
StarChoice& star_last();
// The tuning-cache entry for sweeps of g's extents and radius with elements
// of `esize` bytes on the current device, if any (tune.cu).
bool tune_cache_lookup(const Grid& g, size_t esize, StarChoice* out);
// SM count of the current device (152 when there is none: planning only).
int device_sms();
// Number of per-block partials launch_star writes for these arguments.
i64 star_blocks(const Grid& g, size_t esize, const void* u, const void* b, const void* out);

// Host-side description of the launch one sweep makes (nothing is launched):
// the kernel variant, grid and block, the interior columns (i) and rows (j)
// one block covers, planes per k chunk, and the staged kernel's ring.
struct LaunchPlan {
  int variant = 0;
  int grid_x = 0, grid_y = 0, grid_z = 0, block_threads = 0;
  int tile_w = 0, tile_h = 0, kchunk = 0;
  int stage_elems = 0, smem = 0;
  // the resident 2-D sweep: shared-memory row stride and pad, halo rows by
  // bulk copy, global scratch and the offset of its exchange slots
  int row_stride = 0, row_pad = 0, bulk_copy = 0;
  i64 scratch = 0, xchg_off = 0;
};
LaunchPlan sweep_launch_plan(const Grid& g, size_t esize);
LaunchPlan var_launch_plan(const Grid& g, size_t esize);
// The work units of one batched problem (the scheduler's split: tile shape,
// tiles, k chunks); the same on the host and in the scheduler kernel.
LaunchPlan batch_unit_plan(i64 nx, i64 ny, i64 nz);
// One launch: out = S u + b over the interior; in residual modes also the
// per-block partial sums of rho^2 into `partials` (ZPlan::blocks() entries).
// The plan is formed once per call.  In residual modes a plan needing more
// than `max_partials` partials (when >= 0) is refused with STN_EINVAL before
// anything launches, and `nparts` (when not NULL) receives the number of
// partials the launch writes: the count to reduce.
template <typename T>
int launch_star(const T* u, const T* b, T* out, const Grid& g, const double* coeffs,
                SweepMode mode, double* partials, cudaStream_t s, i64 max_partials = -1,
                i64* nparts = nullptr);
// Copies the halo cells of `src` into `dst` (same geometry).
template <typename T>
int launch_copy_halo(const T* src, T* dst, const Grid& g, cudaStream_t s);

// ---- opt-in double sweep in double-word float arithmetic (sweep_dw.cu) ------
bool dw_applicable(const Grid& g, const double* coeffs, const void* b);
int launch_star_dw(const double* u, double* out, const Grid& g, const double* coeffs, cudaStream_t s);
int tune_set_double_word(int v);
int tune_get_double_word();

// ---- many sweeps of a small grid in one cooperative launch (resident3d.cu) --
constexpr int kResidentTimeout = 1;
// Whether the grid is small enough (every interior point one of at most 8
// per thread of two 512-thread blocks per SM; the sweeps' data stay in L2).
bool resident3d_applicable(const Grid& g, size_t esize);
// Blocks (and residual partials) of the resident launch for this grid.
i64 resident3d_blocks(const Grid& g);
// `sweeps` sweeps ping-ponging a -> b2 -> a ... (b2's halo must equal a's;
// the result is in b2 when sweeps is odd), rhs optional; with resid_last the
// last sweep writes one partial sum of rho^2 per block (*nparts of them).
// bar: two zero-initialised words the launch resets; status: set to
// kResidentTimeout when a grid barrier's bounded wait ran out.
template <typename T>
int launch_star_resident(T* a, T* b2, const T* rhs, const Grid& g, const double* coeffs, i64 sweeps,
                         bool resid_last, double* partials, i64* nparts, unsigned* bar, int* status,
                         cudaStream_t s);
int tune_set_resident3d(int v);
int tune_get_resident3d();
int tune_set_withhold3d(int v);
int tune_get_withhold3d();

// ---- two-dimensional star stencil (jacobi2d.cu) ------------------------------
// Padded (ny+2r) x (nx+2r) grid, i fastest.
struct Grid2 {
  i64 nx, ny;
  int r;
  i64 NX() const { return nx + 2 * r; }
  i64 NY() const { return ny + 2 * r; }
  i64 count() const { return NX() * NY(); }
};
// Blocks of the per-sweep 2-D kernel (grid-stride over 32 x 8 tiles).
constexpr i64 kJ2dBlocks = 152 * 8;
// Launch plan of the shared-memory-resident 2-D sweep: `nblk` bands of at
// most `nbmax` rows, one CTA each; `scratch` bytes of global exchange space
// (counters, status, then the exchange slots at `xchg_off`).
struct Plan2d {
  bool ok = false;
  bool tma = false;     // halo rows by bulk copy (rows a multiple of 16 bytes)
  int pad = 0, ns = 0;  // shared-memory row layout: column c of a row at pad + c, stride ns
  int nblk = 0, nbmax = 0, threads = 0;
  size_t smem = 0, xchg_off = 0, scratch = 0;
};
Plan2d plan_resident2d(const Grid2& g, size_t esize);
bool use_resident2d(const Plan2d& p);
LaunchPlan sweep2d_launch_plan(const Grid2& g, size_t esize);
// One launch of the per-sweep kernel: out = S u + b over the interior; in
// residual modes one partial per block (star2d_blocks(g) entries).
template <typename T>
int launch_star2d(const T* u, const T* b, T* out, const Grid2& g, const double* coeffs,
                  SweepMode mode, double* partials, cudaStream_t s);
i64 star2d_blocks(const Grid2& g);
// `iters` sweeps in -> out, resident (scratch of plan.scratch bytes) or per
// sweep (ping-ponging through `pingpong`, which may be `in`).  Synchronises
// `s`; STN_ETIMEOUT when a resident band's wait ran out.
template <typename T>
int sweep2d_run(const T* in, T* out, const Grid2& g, const double* coeffs, i64 iters,
                unsigned char* scratch, const Plan2d& p, bool resident, T* pingpong,
                cudaStream_t s);
int tune_set_resident2d(int v);
int tune_get_resident2d();
int tune_set_chunk2d(i64 v);
i64 tune_get_chunk2d();
int tune_set_withhold2d(int v);
int tune_get_withhold2d();
int tune_set_tma2d(int v);
int tune_get_tma2d();
int tune_set_ctas2d(int v);
int tune_get_ctas2d();

// ---- sum / dotproduct intrinsics (intrinsics.cu) ---------------------------
// Number of per-block partials launch_vec_reduce writes for n elements.
i64 vec_reduce_blocks(i64 n);
// Partials of sum(x[0..n)) (y == NULL) or sum(x[i]*y[i]); fixed order.
int launch_vec_reduce(const double* x, const double* y, i64 n, double* partials, cudaStream_t s);

// ---- multi-field advection (advect.cu) --------------------------------------
// Tendencies s[m] of fields q[m] (m < nq <= 3) under the velocity (u, v, w);
// q == NULL: the velocity components advect themselves (s[0..2]).
template <typename T>
int launch_advect(const T* u, const T* v, const T* w, const T* const* q, int nq, T* const* s,
                  const Grid& g, const double* c, cudaStream_t st);

// ---- temporal blocking (temporal.cu) -----------------------------------------
// `depth` sweeps of the star stencil (no source term) in one pass: out =
// S^depth(u) on the interior; bitwise equal to depth separate sweeps.
template <typename T>
int launch_temporal(const T* u, T* out, const Grid& g, const double* coeffs, int depth,
                    cudaStream_t s);
// The depth actually used for a request (1 = no temporal blocking).
int temporal_depth_supported(int depth, size_t esize, int radius);
ZPlan plan_temporal(const Grid& g, int depth, int resident);
// Tuning: temporal depth for stencil_sweep (0 = automatic).
int tune_set_temporal_depth(int d);
int tune_get_temporal_depth();
int tune_set_star_chunks(int c);
int tune_get_star_chunks();

// ---- batched solves (batched.cu) --------------------------------------------
// One persistent cluster launch over `count` problems (device grids).
// refined = false: plain double Jacobi, `iters` = max sweeps per problem.
// refined = true: `iters` = max float sweeps per outer step, inner_tol the
// inner stop, max_outer the outer steps.  Synchronises `s`.
int batched_solve(const stn_problem* probs, i64 count, const double* coeffs, int radius, double tol,
                  i64 iters, i64 check_every, double inner_tol, i64 max_outer, bool refined,
                  stn_solve_info* infos, cudaStream_t s);

// Batch engine 2: the problems, largest first, on a pool of worker streams,
// each solved by solve_refined_core / solve_jacobi_core (batched_pool.cu).
int batched_pool(const stn_problem* probs, i64 count, const double* coeffs, int radius, double tol, i64 iters,
                 i64 check_every, double inner_tol, i64 max_outer, bool refined, stn_solve_info* infos,
                 cudaStream_t s);
// Tuning: batched engine (0 = dynamic unit scheduler, 1 = one cluster per
// problem, 2 = worker streams running the one-problem solves).
int tune_set_batch_engine(int v);
int tune_get_batch_engine();
// Tuning: the batch's persistent scheduler launch as a CUDA graph (1, default) or plain (0).
int tune_set_batch_graph(int v);
int tune_get_batch_graph();

// ---- reductions (reduce.cu) -------------------------------------------------
// Sums partials[0..n) in a fixed order into dst[0] = sum, dst[1] = sqrt(sum),
// and, if scale_src is not NULL, dst[2] = sqrt(sum) / scale with
// scale = *scale_src (1 when that is 0), and dst[3] = (dst[2] <= tol).
int launch_finalize(const double* partials, i64 n, double* dst, const double* scale_src,
                    double tol, cudaStream_t s);
// Graph-driven solve: finalize + convergence decision + iteration count +
// while-node condition (continue while not converged and another group of
// `group` sweeps fits under max_full).
int launch_decide(const double* partials, i64 n, double* dst, double tol, i64 group, i64 max_full,
                  cudaGraphConditionalHandle h, cudaStream_t s);
// Counter node of a device-repeated graph body (see graph_repeat in api.cu).
int launch_count(unsigned long long* ctr, i64 n, cudaGraphConditionalHandle h, cudaStream_t s);
// Tuning: 1 = jacobi_solve_f64 iterates inside a CUDA graph (default), 0 = host loop.
int tune_set_solve_graph(int v);
int tune_get_solve_graph();
// Interior sum of squares of a grid (per-block partials) then finalize.
template <typename T>
int launch_interior_sumsq(const T* x, const Grid& g, double* partials, i64* nparts,
                          cudaStream_t s);

// ---- variable coefficient (varcoef.cu) --------------------------------------
enum VarMode { kVarSweep = 0, kVarApply = 1, kVarResidual = 2, kVarRefine = 3 };
ZPlan plan_var(const Grid& g, size_t esize);
// Variable-coefficient kernel choice: -1 automatic (column), 0 plane, 1 column.
int tune_set_var_variant(int v);
int tune_get_var_variant();
// k chunks per tile column of the TMA-staged variable-coefficient sweep (0 = planned).
int tune_set_var_chunks(int v);
int tune_get_var_chunks();
// kVarRefine writes rho = f - A u (double) into out's interior and per-block
// partial sums of rho^2 / maxima of |rho| into partials / partials_max.
template <typename T>
int launch_var(const T* u, const T* a, const T* f, T* out, const Grid& g, const double* w,
               VarMode mode, double* partials, double* partials_max, cudaStream_t s);

// TMA-staged float sweep of radius 2 (varcoef_tma.cu): applicable when the
// rows are a multiple of 16 bytes and u, a, f are 16-byte and out 8-byte
// aligned (NULL pointers: not checked, for planning).
bool var_tma_applicable(const Grid& g, size_t esize, const void* u, const void* a, const void* f,
                        const void* out);
ZPlan plan_var_tma(const Grid& g);
int launch_var_tma(const float* u, const float* a, const float* f, float* out, const Grid& g, const double* w,
                   cudaStream_t s);
// The status word of the TMA-staged sweeps: nonzero once a bounded wait ran
// out (the sweep stopped early); `clear` resets it.  Synchronous.
int var_tma_status(bool clear, int* status);

// ---- one-problem solves on the full-grid kernels (api.cu) -------------------
// Double Jacobi of one device problem (db may be NULL); tmp: a scratch grid
// of the problem's size.  Synchronises `s`; returns STN_OK,
// STN_NOT_CONVERGED or an error.
int solve_jacobi_core(const double* db, double* du, double* tmp, const Grid& g, const double* coeffs, double tol,
                      i64 max_iters, i64 check_every, stn_solve_info* info, cudaStream_t s);
// The refinement of jacobi_solve_refined_f64 for one device problem; t: a
// double scratch grid, f32: three float scratch grids (r32, e, e'), all of
// the problem's size.  Synchronises `s`.
int solve_refined_core(const double* db, double* du, double* t, float* f32, const Grid& g, const double* coeffs,
                       double tol, i64 inner_sweeps, double inner_tol, i64 check_every, i64 max_outer,
                       stn_solve_info* info, cudaStream_t s);

// ---- refinement helpers (refine.cu) ----------------------------------------
// r32 = float(rho / s), s = dst_scalar[0] (device); e = 0 on the interior.
int launch_refine_scale(const double* rho, float* r32, const Grid& g, const double* smax,
                        cudaStream_t s);
// u += s * double(e) on the interior.
int launch_refine_update(double* u, const float* e, const Grid& g, const double* smax,
                         cudaStream_t s);
int launch_max_finalize(const double* partials, i64 n, double* dst, cudaStream_t s);
// Block maxima of |t - u| over the interior (at most 152 * 16 partials; the
// count in *nparts), for the constant-coefficient refinement's scale.
int launch_diff_max(const double* t, const double* u, const Grid& g, double* partials, i64* nparts,
                    cudaStream_t s);
// r32 = float((t - u) / s) on the interior, s = *smax (device).
int launch_refine_scale_diff(const double* t, const double* u, float* r32, const Grid& g, const double* smax,
                             cudaStream_t s);
template <typename T, typename U>
int launch_convert(const T* src, U* dst, i64 n, cudaStream_t s);

}  // namespace stn
