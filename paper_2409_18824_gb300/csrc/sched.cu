// Dynamic persistent scheduler for many Jacobi solves (batched and served).
//
// One persistent kernel runs one wave of CTAs.  Every active problem advances
// pass by pass (a pass = one data-parallel step: a sweep, a residual sweep, an
// element-wise refinement step).  A pass is split into work units (32 x 8
// column tiles x a chunk of k planes) that any CTA may claim, so a large
// problem soaks up every CTA the small ones leave idle, and a problem's
// critical path shrinks to its own work divided by the whole GPU.
//
//   claim     : 64-bit word per slot = pass id, the pass's unit count and
//               the next unit; one atomicAdd claims a unit AND names the pass
//               it belongs to, and tells whether the claim is valid.
//   complete  : per-unit partial results are written to the problem's
//               partials array, then a release fence and an atomicAdd on the
//               slot's done counter; the CTA that completes the last unit
//               runs the pass epilogue.
//   epilogue  : reduces the partials in unit order (a fixed tree: results do
//               not depend on which CTA did what), advances the problem's
//               state machine, resets the counters and publishes the next
//               pass with an atomic exchange of the claim word (release).
// Sweeps are computed by star_tile, the code of the single-problem kernels,
// or at radius 1 by star_tile_async, its arithmetic with the planes staged
// asynchronously, so every sweep is bitwise the single-problem sweep.  There is no device
// wait on another CTA's progress except the bounded idle back-off of a CTA
// that found no work; it gives up after `idle_ns` and records STN_ETIMEOUT
// (batch) or simply returns (serving, where the host relaunches on demand).
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "work_sched.h"
#include "star.cuh"

namespace stn {

namespace {

constexpr int BT = TX * TY;
constexpr int kSchedMinBlocksRefined = 5;
constexpr int kSchedMinBlocksPlain = 4;

enum Phase : int {
  PH_IDLE = 0,
  PH_INIT = 1,    // sum b^2 (rhs norm)
  PH_SWEEP = 2,   // plain double sweep cur -> nxt (residual on a group's last)
  PH_COPY = 3,    // u <- t (interior)
  PH_RES = 4,     // refined: t = S u + b, sum rho^2
  PH_MAX = 5,     // refined: max |t - u|
  PH_SCALE = 6,   // refined: r32 = float((t-u)/s), e = 0, sum r32^2
  PH_INNER = 7,   // refined: float sweep e -> e' (residual on a group's last)
  PH_UPDATE = 8,  // refined: u += s * e
};

// Unit tile shapes, all of BT columns: 32 x 8, 16 x 16 or 8 x 32, whichever
// covers the problem's (nx, ny) with the fewest tiles (ties to the wider
// shape: longer contiguous rows).  The block's threads map to the tile flat.
// Over the 2048-problem mix (sizes log-uniform in [16, 128]) the interior
// share of the units' columns is 0.759 with 32 x 8 alone, 0.808 with 16 x 16
// added, 0.834 with 8 x 32 too.
__host__ __device__ inline int tile_width(int shape) { return shape == 0 ? TX : (shape == 1 ? 16 : 8); }

struct Geo {
  int tiles_x, tiles_y, kc, klen, n, shape;  // shape: 0 = 32 x 8, 1 = 16 x 16, 2 = 8 x 32 tiles
};

__host__ __device__ inline Geo make_geo(int nx, int ny, int nz) {
  Geo g;
  // the shape depends on the extents only, so a problem's reduction order
  // (and hence its iteration count) is the same in any batch
  g.shape = 0;
  long long best = -1;
  for (int sh = 0; sh < 3; sh++) {
    const int tw = tile_width(sh), th = BT / tw;
    const long long t = (long long)((nx + tw - 1) / tw) * ((ny + th - 1) / th);
    if (best < 0 || t < best) {
      best = t;
      g.shape = sh;
    }
  }
  const int tw = tile_width(g.shape), th = BT / tw;
  g.tiles_x = (nx + tw - 1) / tw;
  g.tiles_y = (ny + th - 1) / th;
  // k chunks sized from the extents alone (the unit split fixes the order of
  // every reduction): aim at ~256 units per pass, with chunks of 128..256
  // planes.  Measured on the 2048-solve mix (refined / FP64 solves/s), with
  // the plane kernel's units: 16..64 planes, 2048 units per pass: 90.6 / -;
  // 32..64, 1024: 114.3 / 43.8; 64..128, 512: 125.4 / 45.1; 96..128: 125.7;
  // 128..256, 256: 127.5.  With the ring units: 64..128, 512: 146.3-147.4 /
  // 45.5; 128..256, 256: 151.4 / 45.9.  Longer units cost less claiming per
  // point (22 % -> 16 % of CTA cycles, refined) and fewer ring start-ups.
  const long long tiles = (long long)g.tiles_x * g.tiles_y;
  long long klen = ((long long)nz * tiles + 255) / 256;
  if (klen < 128) klen = 128;
  if (klen > 256) klen = 256;
  if (klen > nz) klen = nz;
  g.klen = (int)klen;
  g.kc = (nz + g.klen - 1) / g.klen;
  // unsigned: wraps instead of overflowing for extents the entry points
  // reject (they use the exact 64-bit count); equal to the product otherwise
  g.n = (int)((unsigned)g.tiles_x * (unsigned)g.tiles_y * (unsigned)g.kc);
  return g;
}

__device__ __forceinline__ int tid_flat() { return threadIdx.x + TX * threadIdx.y; }

// Reads a state struct through volatile 8-byte loads (never a stale L1 line):
// slot and problem records are written by other SMs and, when serving, by
// the host.
template <typename S>
__device__ __forceinline__ S vload(const S* p) {
  static_assert(sizeof(S) % 8 == 0, "state records are whole 8-byte words");
  S out;
  const volatile unsigned long long* src = reinterpret_cast<const volatile unsigned long long*>(p);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(&out);
#pragma unroll 4
  for (int i = 0; i < (int)(sizeof(S) / 8); i++) dst[i] = src[i];
  return out;
}

__device__ __forceinline__ double bmax(double v, double* red) {
  const int lane = tid_flat() & 31, warp = tid_flat() >> 5;
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

// Fixed-order reduction of n partials by the whole CTA (tree shape depends
// on n only); result valid in thread 0.
__device__ __forceinline__ double reduce_parts(const double* p, int n, bool is_max, double* red) {
  double v = 0.0;
  for (int i = tid_flat(); i < n; i += BT) {
    const double x = __ldcg(p + i);
    v = is_max ? fmax(v, x) : v + x;
  }
  if (is_max) return bmax(v, red);
  const double s = block_sum_fixed<BT>(v, red);
  __syncthreads();
  return s;
}

// Calls f(p) for every interior point of unit q, k outer; each thread owns
// one column of the unit's tile.
template <int R, typename F>
__device__ __forceinline__ void for_unit_points(const SchedProblem& P, const Geo& g, int q, F&& f) {
  const int tiles = g.tiles_x * g.tiles_y;
  const int kci = q / tiles, tq = q - kci * tiles;
  const int tyi = tq / g.tiles_x, txi = tq - tyi * g.tiles_x;
  const int tw = tile_width(g.shape), th = BT / tw, t = tid_flat();
  const int i = txi * tw + t % tw + R, j = tyi * th + t / tw + R;
  if (i >= P.nx + R || j >= P.ny + R) return;
  const i64 NX = P.nx + 2 * R, NY = P.ny + 2 * R;
  const int k0 = R + kci * g.klen, k1 = min(k0 + g.klen, P.nz + R);
  for (int k = k0; k < k1; k++) f((i64)i + NX * ((i64)j + NY * k));
}

// one shared plane of any tile shape (radius <= 2): 12 x 36 = 36 x 12 = 432
// elements for 32 x 8 and 8 x 32, 20 x 20 for 16 x 16
constexpr int kPlaneElems = (TY + 4) * (TX + 4);
static_assert((BT / 16 + 4) * (16 + 4) <= kPlaneElems && (BT / 8 + 4) * (8 + 4) <= kPlaneElems,
              "every tile shape's plane fits");
constexpr int kPlaneBytes = kPlaneElems * 8;

// ---------------------------------------------------------------------------
// Radius-1 unit sweeps stream their planes through a shared-memory ring
// filled by element-wise asynchronous copies (cp.async.ca: the grids were
// written by other CTAs in earlier passes, and the unit's acquire fence
// precedes the copies as it preceded the loads), PF planes ahead of the
// 2R+1 in use, with one block barrier per plane (per two planes where the
// ring has room: star_tile_async2, below).  The per-plane tile sweep
// with a one-plane register prefetch (star_tile) spent most of its time at
// its two barriers per plane and on long-scoreboard stalls: in ncu, 64 warps
// per SM were resident and issued only 36 % of the cycles.  A stage holds the
// tile's plane with its halo and, after it, the source term of the tile's
// points; z neighbours come from the neighbouring stages.  Every value and
// operation is star_tile's, in its order, so the results are its bits.
// The ring is 27.5 KB: 5 double stages or 10 float stages.  Larger rings
// were slower on the refined 2048-solve mix at 5 blocks per SM (8 double
// stages: 128.0 solves/s against 147.0; 4 stages: 147.8), most likely
// because shared memory taken from the unified L1 leaves less cache for the
// units' element-wise copies and the spills.
constexpr int kStageElems = kPlaneElems + BT;  // plane with halo, then b
template <int MINB>
__host__ __device__ constexpr int ring_bytes() {
  static_assert(MINB * (5 * kStageElems * 8 + 1024 + 512) <= 233472, "the rings of MINB blocks fit an SM");
  return 5 * kStageElems * 8;
}
// stages of T the ring holds (at most 12)
template <typename T, int MINB>
__host__ __device__ constexpr int ring_stages() {
  return ring_bytes<MINB>() / (kStageElems * (int)sizeof(T)) > 12 ? 12
                                                                  : ring_bytes<MINB>() / (kStageElems * (int)sizeof(T));
}
// planes in flight beyond those in use: two planes are computed per block
// barrier when the ring leaves at least one plane in flight that way
template <typename T, int MINB>
__host__ __device__ constexpr bool ring_pairs() { return ring_stages<T, MINB>() >= 6; }
template <typename T, int MINB>
__host__ __device__ constexpr int ring_pf() {
  return ring_pairs<T, MINB>() ? ring_stages<T, MINB>() - 5 : ring_stages<T, MINB>() - 3;
}
// the unit's shared buffer: the ring at radius 1, one plane at radius 2
template <int R, int MINB>
__host__ __device__ constexpr int unit_smem_bytes() { return R == 1 ? ring_bytes<MINB>() : kPlaneBytes; }

__device__ __forceinline__ void cp_el(void* dst_smem, const void* src, int bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename T, bool HAS_B, bool HAS_C0, int MODE, int PF>
__device__ __forceinline__ void star_tile_async(const T* u, const T* b, T* out, int nx, int ny, int NX, int NY,
                                                int tile_x, int tile_y, int k0, int k1, const StarCoeffs<T, 1>& cf,
                                                int tw, int th, T* ring, double* rsum_io) {
  using A = Arith<T>;
  constexpr int R = 1, S = 2 * R + 1 + PF;
  static_assert(PF >= 1, "at least one plane ahead");
  const int flat = (int)(threadIdx.x + blockDim.x * threadIdx.y);
  const int tx = flat % tw, ty = flat / tw;
  const int pitch = tw + 2 * R;
  const int gi = tile_x * tw + tx + R, gj = tile_y * th + ty + R;
  const i64 sy = NX, sz = (i64)NX * NY;
  const bool inx = gi < NX, iny = gj < NY;
  const bool active = (gi < nx + R) && (gj < ny + R);
  const bool hx = (tx < R) || (tx >= tw - R);
  const int hx_i = (tx < R) ? gi - R : gi + R;
  const int hx_lx = (tx < R) ? tx : tx + 2 * R;
  const bool hx_ok = hx && hx_i < NX && iny;
  const bool hy = (ty < R) || (ty >= th - R);
  const int hy_j = (ty < R) ? gj - R : gj + R;
  const int hy_ly = (ty < R) ? ty : ty + 2 * R;
  const bool hy_ok = hy && hy_j < NY && inx;
  const bool ld_c = inx && iny;
  const int me = (ty + R) * pitch + tx + R;
  const T* pc = u + gi + gj * sy;
  const T* px = u + hx_i + gj * sy;
  const T* py = u + gi + (i64)hy_j * sy;
  const T* pb = HAS_B ? b + gi + gj * sy : nullptr;
  const int pfirst = k0 - R, plast = k1 - 1 + R;
  auto stage = [&](int p) -> T* { return ring + ((p - pfirst) % S) * kStageElems; };
  auto issue = [&](int p) {  // every thread: its cells of plane p (one commit group, maybe empty)
    if (p <= plast) {
      T* st = stage(p);
      const i64 po = (i64)p * sz;
      if (ld_c) cp_el(st + me, pc + po, (int)sizeof(T));
      if (hx_ok) cp_el(st + (ty + R) * pitch + hx_lx, px + po, (int)sizeof(T));
      if (hy_ok) cp_el(st + hy_ly * pitch + tx + R, py + po, (int)sizeof(T));
      if (HAS_B && active && p >= k0 && p < k1) cp_el(st + kPlaneElems + flat, pb + po, (int)sizeof(T));
    }
    cp_commit();
  };
  // planes k0 - R .. k0 + R + PF - 1 before the first plane
  for (int i = 0; i < S - 1; i++) issue(pfirst + i);
  double rsum = *rsum_io;
  for (int k = k0; k < k1; k++) {
    cp_wait<PF - 1>();  // this thread's copies of planes <= k + R have landed
    __syncthreads();          // everyone's, and plane k - 1 - R is no longer read
    issue(k + R + PF);  // into the stage of plane k - 1 - R
    if (active) {
      const T* c0p = stage(k);
      const T* cm = stage(k - 1);
      const T* cp = stage(k + 1);
      const T sx = A::add(c0p[me - 1], c0p[me + 1]);
      const T sy_ = A::add(c0p[me - pitch], c0p[me + pitch]);
      const T szz = A::add(cm[me], cp[me]);
      T acc = A::mul(cf.c[1], A::add(A::add(sx, sy_), szz));
      const T c = c0p[me];
      if (HAS_C0) acc = A::add(acc, A::mul(cf.c[0], c));
      if (HAS_B) acc = A::add(acc, c0p[kPlaneElems + flat]);
      if (MODE != kResidualOnly) out[gi + gj * sy + (i64)k * sz] = acc;
      if (MODE != kSweep) {
        const double rho = (double)acc - (double)c;
        rsum = __fma_rn(rho, rho, rsum);
      }
    }
  }
  cp_wait<0>();
  __syncthreads();  // the ring is free again when this returns
  *rsum_io = rsum;
}

// The same tile sweep with two planes per block barrier: the ring holds the
// 2R+2 planes a pair reads and PF more in flight; each thread updates its
// column at planes k and k+1 (k's residual term first, as in the one-plane
// loop), which halves the waits and barriers per point and gives each thread
// two independent updates to overlap.  Plane p sits in stage (p - first
// staged plane) mod S; stage indices advance instead of being recomputed.
template <typename T, bool HAS_B, bool HAS_C0, int MODE, int PF>
__device__ __forceinline__ void star_tile_async2(const T* u, const T* b, T* out, int nx, int ny, int NX, int NY,
                                                 int tile_x, int tile_y, int k0, int k1,
                                                 const StarCoeffs<T, 1>& cf, int tw, int th, T* ring,
                                                 double* rsum_io) {
  using A = Arith<T>;
  constexpr int R = 1, S = 2 * R + 3 + PF;
  static_assert(PF >= 1, "at least one plane ahead");
  const int flat = (int)(threadIdx.x + blockDim.x * threadIdx.y);
  const int tx = flat % tw, ty = flat / tw;
  const int pitch = tw + 2 * R;
  const int gi = tile_x * tw + tx + R, gj = tile_y * th + ty + R;
  const i64 sz = (i64)NX * NY;
  const bool inx = gi < NX, iny = gj < NY;
  const bool active = (gi < nx + R) && (gj < ny + R);
  const bool hx = (tx < R) || (tx >= tw - R);
  const int hx_i = (tx < R) ? gi - R : gi + R;
  const int hx_lx = (tx < R) ? tx : tx + 2 * R;
  const bool hx_ok = hx && hx_i < NX && iny;
  const bool hy = (ty < R) || (ty >= th - R);
  const int hy_j = (ty < R) ? gj - R : gj + R;
  const int hy_ly = (ty < R) ? ty : ty + 2 * R;
  const bool hy_ok = hy && hy_j < NY && inx;
  const bool ld_c = inx && iny;
  const int me = (ty + R) * pitch + tx + R;
  const int hx_at = (ty + R) * pitch + hx_lx, hy_at = hy_ly * pitch + tx + R;
  const i64 col = gi + (i64)gj * NX;
  const T* pc = u + col;
  const T* px = u + (hx_i + (i64)gj * NX);
  const T* py = u + (gi + (i64)hy_j * NX);
  const T* pb = HAS_B ? b + col : nullptr;
  const int pfirst = k0 - R, plast = k1 - 1 + R;
  int p_iss = pfirst, s_iss = 0;  // next plane to issue and its stage
  auto issue_next = [&]() {  // every thread: its cells of the next plane (one commit group, maybe empty)
    if (p_iss <= plast) {
      T* st = ring + s_iss * kStageElems;
      const i64 po = (i64)p_iss * sz;
      if (ld_c) cp_el(st + me, pc + po, (int)sizeof(T));
      if (hx_ok) cp_el(st + hx_at, px + po, (int)sizeof(T));
      if (hy_ok) cp_el(st + hy_at, py + po, (int)sizeof(T));
      if (HAS_B && active && p_iss >= k0 && p_iss < k1) cp_el(st + kPlaneElems + flat, pb + po, (int)sizeof(T));
    }
    cp_commit();
    p_iss++;
    s_iss = s_iss + 1 == S ? 0 : s_iss + 1;
  };
  // planes k0 - R .. k0 + R + PF before the first pair
  for (int i = 0; i < 2 * R + 1 + PF; i++) issue_next();
  double rsum = *rsum_io;
  int sk = R;  // stage of plane k
  T* outk = out + col + (i64)k0 * sz;
  for (int k = k0; k < k1; k += 2) {
    cp_wait<PF - 1>();  // this thread's copies of planes <= k + 1 + R have landed
    __syncthreads();    // everyone's, and planes <= k - 1 - R are no longer read
    issue_next();       // planes k + R + PF + 1 and + 2, into the stages of k - 2 - R and k - 1 - R
    issue_next();
    if (active) {
      const int sm = sk == 0 ? S - 1 : sk - 1;
      const int sp = sk + 1 == S ? 0 : sk + 1;
      const int spp = sp + 1 == S ? 0 : sp + 1;
      const T* c0p = ring + sk * kStageElems;
      const T* cm = ring + sm * kStageElems;
      const T* cp = ring + sp * kStageElems;
      const T c = c0p[me];
      const T c1 = cp[me];
      {
        const T sx = A::add(c0p[me - 1], c0p[me + 1]);
        const T sy_ = A::add(c0p[me - pitch], c0p[me + pitch]);
        const T szz = A::add(cm[me], c1);
        T acc = A::mul(cf.c[1], A::add(A::add(sx, sy_), szz));
        if (HAS_C0) acc = A::add(acc, A::mul(cf.c[0], c));
        if (HAS_B) acc = A::add(acc, c0p[kPlaneElems + flat]);
        if (MODE != kResidualOnly) outk[0] = acc;
        if (MODE != kSweep) {
          const double rho = (double)acc - (double)c;
          rsum = __fma_rn(rho, rho, rsum);
        }
      }
      if (k + 1 < k1) {
        const T* cpp = ring + spp * kStageElems;
        const T sx = A::add(cp[me - 1], cp[me + 1]);
        const T sy_ = A::add(cp[me - pitch], cp[me + pitch]);
        const T szz = A::add(c, cpp[me]);
        T acc = A::mul(cf.c[1], A::add(A::add(sx, sy_), szz));
        if (HAS_C0) acc = A::add(acc, A::mul(cf.c[0], c1));
        if (HAS_B) acc = A::add(acc, cp[kPlaneElems + flat]);
        if (MODE != kResidualOnly) outk[sz] = acc;
        if (MODE != kSweep) {
          const double rho = (double)acc - (double)c1;
          rsum = __fma_rn(rho, rho, rsum);
        }
      }
    }
    sk = sk + 2 >= S ? sk + 2 - S : sk + 2;
    outk += 2 * sz;
  }
  cp_wait<0>();
  __syncthreads();  // the ring is free again when this returns
  *rsum_io = rsum;
}

template <typename T, int R, bool HAS_C0, int MODE, int MINB>
__device__ __forceinline__ double unit_sweep(const T* cur, const T* b, T* nxt, const SchedProblem& P,
                                             const Geo& g, int q, const StarCoeffs<T, R>& cf, T* plane) {
  const int tiles = g.tiles_x * g.tiles_y;
  const int kci = q / tiles, tq = q - kci * tiles;
  const int tyi = tq / g.tiles_x, txi = tq - tyi * g.tiles_x;
  const int k0 = R + kci * g.klen, k1 = min(k0 + g.klen, P.nz + R);
  const int NX = P.nx + 2 * R, NY = P.ny + 2 * R;
  const int tw = tile_width(g.shape);
  double rs = 0.0;
  if constexpr (R == 1) {
    // `plane` is the kernel's ring buffer at radius 1
    if constexpr (ring_pairs<T, MINB>()) {
      if (b)
        star_tile_async2<T, true, HAS_C0, MODE, ring_pf<T, MINB>()>(cur, b, nxt, P.nx, P.ny, NX, NY, txi, tyi, k0,
                                                                    k1, cf, tw, BT / tw, plane, &rs);
      else
        star_tile_async2<T, false, HAS_C0, MODE, ring_pf<T, MINB>()>(cur, nullptr, nxt, P.nx, P.ny, NX, NY, txi,
                                                                     tyi, k0, k1, cf, tw, BT / tw, plane, &rs);
      return rs;
    }
    if (b)
      star_tile_async<T, true, HAS_C0, MODE, ring_pf<T, MINB>()>(cur, b, nxt, P.nx, P.ny, NX, NY, txi, tyi, k0, k1, cf, tw, BT / tw,
                                             plane, &rs);
    else
      star_tile_async<T, false, HAS_C0, MODE, ring_pf<T, MINB>()>(cur, nullptr, nxt, P.nx, P.ny, NX, NY, txi, tyi, k0, k1, cf, tw,
                                              BT / tw, plane, &rs);
    return rs;
  }
  if (b)
    star_tile<T, R, true, HAS_C0, MODE>(cur, b, nxt, P.nx, P.ny, NX, NY, txi, tyi, k0, k1, cf, tw, BT / tw, plane,
                                        &rs);
  else
    star_tile<T, R, false, HAS_C0, MODE>(cur, nullptr, nxt, P.nx, P.ny, NX, NY, txi, tyi, k0, k1, cf, tw, BT / tw,
                                         plane, &rs);
  return rs;
}

// Processes unit q of the slot's current pass; returns the partial (valid in
// thread 0) to store at partials[q].
template <int R, bool HAS_C0, int MINB>
__device__ double run_unit(const SchedArgs& a, const SchedSlot& S, const SchedProblem& P, int q,
                           unsigned char* smem, double* red) {
  const Geo g = make_geo(P.nx, P.ny, P.nz);
  StarCoeffs<double, R> c64;
  StarCoeffs<float, R> c32;
#pragma unroll
  for (int d = 0; d <= R; d++) {
    c64.c[d] = a.coeffs[d];
    c32.c[d] = (float)a.coeffs[d];
  }
  double* t64 = (double*)smem;
  float* t32 = (float*)smem;
  double v = 0.0;
  switch (S.phase) {
    case PH_INIT: {
      if (P.b) for_unit_points<R>(P, g, q, [&](i64 p) {
          const double x = P.b[p];
          v = __fma_rn(x, x, v);
        });
      return block_sum_fixed<BT>(v, red);
    }
    case PH_SWEEP: {
      double* cur = S.parity ? P.t : P.u;
      double* nxt = S.parity ? P.u : P.t;
      if (S.resid)
        v = unit_sweep<double, R, HAS_C0, kSweepResidual, MINB>(cur, P.b, nxt, P, g, q, c64, t64);
      else
        unit_sweep<double, R, HAS_C0, kSweep, MINB>(cur, P.b, nxt, P, g, q, c64, t64);
      return block_sum_fixed<BT>(v, red);
    }
    case PH_COPY: {
      for_unit_points<R>(P, g, q, [&](i64 p) { P.u[p] = P.t[p]; });
      return 0.0;
    }
    case PH_RES: {
      v = unit_sweep<double, R, HAS_C0, kSweepResidual, MINB>(P.u, P.b, P.t, P, g, q, c64, t64);
      return block_sum_fixed<BT>(v, red);
    }
    case PH_MAX: {
      for_unit_points<R>(P, g, q, [&](i64 p) { v = fmax(v, fabs(__dsub_rn(P.t[p], P.u[p]))); });
      return bmax(v, red);
    }
    case PH_SCALE: {
      const double s = S.smax;
      for_unit_points<R>(P, g, q, [&](i64 p) {
        const float x = __double2float_rn(__ddiv_rn(__dsub_rn(P.t[p], P.u[p]), s));
        P.r32[p] = x;
        P.e[p] = 0.0f;
        v = __fma_rn((double)x, (double)x, v);
      });
      return block_sum_fixed<BT>(v, red);
    }
    case PH_INNER: {
      float* cur = S.parity ? P.e2 : P.e;
      float* nxt = S.parity ? P.e : P.e2;
      if (S.resid)
        v = unit_sweep<float, R, HAS_C0, kSweepResidual, MINB>(cur, P.r32, nxt, P, g, q, c32, t32);
      else
        unit_sweep<float, R, HAS_C0, kSweep, MINB>(cur, P.r32, nxt, P, g, q, c32, t32);
      return block_sum_fixed<BT>(v, red);
    }
    case PH_UPDATE: {
      const double s = S.smax;
      const float* e = S.parity ? P.e2 : P.e;
      for_unit_points<R>(P, g, q, [&](i64 p) { P.u[p] = __dadd_rn(P.u[p], __dmul_rn(s, (double)e[p])); });
      return 0.0;
    }
    default:
      return 0.0;
  }
}

// Sets up a group of sweeps of the slot (counts are set; the caller publishes).
__device__ __forceinline__ void start_group(const SchedArgs& a, SchedSlot& S, long long done_so_far,
                                            long long limit) {
  long long left = limit - done_so_far;
  S.group = a.check_every < left ? a.check_every : left;
  S.group_pos = 0;
  S.resid = S.group == 1 ? 1 : 0;
}

// Advances the slot's state machine after a completed pass.  `red_val` is
// the reduced partial of that pass.  Returns true when the problem finished.
__device__ bool advance(const SchedArgs& a, SchedSlot& S, const SchedProblem& P, double red_val) {
  switch (S.phase) {
    case PH_INIT: {
      S.bnorm = sqrt(red_val);
      S.scale = S.bnorm > 0.0 ? S.bnorm : 1.0;
      S.iters = 0;
      S.outer = 0;
      S.sweeps = 0;
      S.parity = 0;
      if (a.refined) {
        S.phase = PH_RES;
        S.resid = 1;
        return false;
      }
      if (a.max_iters <= 0) {
        S.status = STN_NOT_CONVERGED;
        return true;
      }
      S.phase = PH_SWEEP;
      start_group(a, S, 0, a.max_iters);
      return false;
    }
    case PH_SWEEP: {
      S.iters++;
      S.parity ^= 1;
      S.group_pos++;
      if (S.group_pos == S.group) {
        S.res = sqrt(red_val);
        S.rel = S.res / S.scale;
        if (S.rel <= a.tol) S.status = STN_OK;
        else if (S.iters >= a.max_iters) S.status = STN_NOT_CONVERGED;
        else {
          start_group(a, S, S.iters, a.max_iters);
          return false;
        }
        if (S.parity) {  // the last iterate is in t
          S.phase = PH_COPY;
          return false;
        }
        return true;
      }
      S.resid = S.group_pos == S.group - 1 ? 1 : 0;
      return false;
    }
    case PH_COPY:
      return true;
    case PH_RES: {
      S.res = sqrt(red_val);
      S.rel = S.res / S.scale;
      if (S.rel <= a.tol) {
        S.status = STN_OK;
        return true;
      }
      if (S.outer >= a.max_outer) {
        S.status = STN_NOT_CONVERGED;
        return true;
      }
      S.phase = PH_MAX;
      return false;
    }
    case PH_MAX: {
      S.smax = red_val;
      if (!(S.smax > 0.0)) {
        S.status = STN_NOT_CONVERGED;
        return true;
      }
      S.phase = PH_SCALE;
      return false;
    }
    case PH_SCALE: {
      S.r32norm = sqrt(red_val);
      S.inner = 0;
      S.parity = 0;
      if (a.max_iters <= 0) {
        S.phase = PH_UPDATE;
        return false;
      }
      S.phase = PH_INNER;
      start_group(a, S, 0, a.max_iters);
      if (!(a.inner_tol > 0.0)) S.resid = 0;
      return false;
    }
    case PH_INNER: {
      S.inner++;
      S.parity ^= 1;
      S.group_pos++;
      bool stop = false;
      if (S.group_pos == S.group) {
        if (a.inner_tol > 0.0 && sqrt(red_val) <= a.inner_tol * S.r32norm) stop = true;
        if (S.inner >= a.max_iters) stop = true;
        if (!stop) start_group(a, S, S.inner, a.max_iters);
      } else {
        S.resid = S.group_pos == S.group - 1 ? 1 : 0;
      }
      if (!(a.inner_tol > 0.0)) S.resid = 0;
      if (stop) S.phase = PH_UPDATE;
      return false;
    }
    case PH_UPDATE: {
      S.sweeps += S.inner;
      S.outer++;
      S.phase = PH_RES;
      S.resid = 1;
      return false;
    }
    default:
      return true;
  }
}

__device__ __forceinline__ int ld_acquire_sys_s32(const int* p) {
  int v;
  asm volatile("ld.acquire.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Takes unit q of the pass named by claim word w of slot si (one thread; q
// is below the word's unit count).  The pass's state was written before the
// word (release), and the pass cannot end while this unit is held, so the
// state read after the fence is that pass's.  The check below cannot fail
// under that protocol; if it did, the unit would be left unrun and the
// batch would end by its idle limit (STN_ETIMEOUT) rather than run a unit
// of the wrong pass.
__device__ __forceinline__ int take_claim(const SchedArgs& a, int si, unsigned long long w, int q,
                                          SchedSlot& s_state, SchedProblem& s_prob, int& s_unit) {
  __threadfence();
  const SchedSlot S = vload(&a.slots[si]);
  if ((S.pass & 0xffffu) != claim_pass(w) || q >= S.nunits) return 0;
  s_state = S;
  s_prob = vload(&a.probs[S.problem]);
  s_unit = q;
  return 1;
}

// Publishes the next pass of slot si (one thread; the slot state for that
// pass has been written).  Release: state writes before the word exchange.
__device__ __forceinline__ void publish(const SchedArgs& a, int si) {
  SchedSlot& S = a.slots[si];
  const unsigned pass = *(volatile unsigned*)&S.pass + 1;
  const int nunits = *(volatile int*)&S.nunits;
  S.pass = pass;
  S.done = 0;
  __threadfence();
  atomicExch(&a.words[si], claim_word(pass, nunits));
}

// Loads problem `pi` into slot `si` (one thread) and publishes its first pass.
__device__ void admit(const SchedArgs& a, int si, int pi) {
  SchedSlot& S = a.slots[si];
  const SchedProblem P = vload(&a.probs[pi]);
  S.problem = pi;
  S.phase = PH_INIT;
  S.status = STN_NOT_CONVERGED;
  S.parity = 0;
  S.resid = 0;
  S.rel = INFINITY;
  S.res = INFINITY;
  S.nunits = P.nunits;
  S.claim_free = 0;
  S.start_clock = clock64();
  publish(a, si);
}

// Takes the next queued problem index, or -1.  For serving the host appends
// entries and then advances *qtail (system-scope release).
__device__ int pop_queue(const SchedArgs& a) {
  const int tail = a.serving ? ld_acquire_sys_s32(a.qtail) : a.qlen;
  int h = atomicAdd(a.qhead, 0);
  while (h < tail) {
    const int got = atomicCAS(a.qhead, h, h + 1);
    if (got == h) return *(const volatile int*)&a.queue[h % a.qcap];
    h = got;
  }
  return -1;
}

// Tries to start a queued problem in a free slot (one thread).  The slot is
// claimed first, so a popped problem always has a home.
__device__ bool try_admit(const SchedArgs& a) {
  if (*(volatile int*)a.free_slots <= 0) return false;
  for (int k = 0; k < a.nslots; k++) {
    if (*(volatile int*)&a.slots[k].claim_free != 1) continue;
    if (atomicCAS(&a.slots[k].claim_free, 1, 2) != 1) continue;  // 2 = being filled
    const int pi = pop_queue(a);
    if (pi < 0) {
      atomicExch(&a.slots[k].claim_free, 1);
      return false;
    }
    atomicSub(a.free_slots, 1);
    admit(a, k, pi);
    return true;
  }
  return false;
}

// The CTA that completed the last unit of slot si's pass: reduce the unit
// partials in order, advance the state machine, publish the next pass or
// finish the problem and start the next queued one in this slot.
template <int R, bool HAS_C0>
__device__ void epilogue(const SchedArgs& a, int si, const SchedProblem& P, const SchedSlot& S0,
                         double* red) {
  const bool is_max = S0.phase == PH_MAX;
  const double v = reduce_parts(P.partials, S0.nunits, is_max, red);
  if (tid_flat() == 0) {
    SchedSlot S = vload(&a.slots[si]);
    const bool finished = advance(a, S, P, v);
    a.slots[si] = S;  // written back before anything is published
    if (finished) {
      SchedResult r;
      r.iters = a.refined ? S.sweeps : S.iters;
      r.outer = S.outer;
      r.rel_res = S.rel;
      r.res_norm = S.res;
      r.rhs_norm = S.bnorm;
      r.clocks = clock64() - S.start_clock;
      r.status = S.status;
      r.pad = 0;
      a.results[S.problem] = r;
      __threadfence_system();
      atomicExch(&a.done_flags[S.problem], 1);
      __threadfence_system();
      atomicAdd(a.finished, 1);
      SchedSlot& G = a.slots[si];
      G.phase = PH_IDLE;
      G.nunits = 0;
      const int nxt = pop_queue(a);
      if (nxt >= 0) {
        admit(a, si, nxt);
      } else {
        publish(a, si);  // an empty pass: nothing to claim
        __threadfence();
        atomicExch(&G.claim_free, 1);
        atomicAdd(a.free_slots, 1);
      }
    } else {
      publish(a, si);
    }
  }
  __syncthreads();
}

// MINB: blocks per SM the register allocation must allow.  With the plane
// kernel's units, refined work (float inner sweeps) was latency-bound and ran
// faster with more resident warps (a batch of 256 refined solves: 68.7 solves/s
// at 4 blocks per SM, 101.9 at 7).  With the ring units, the refined
// 2048-solve mix runs 132.7 solves/s at 7 blocks (32 registers, spills),
// 128.9 at 6 (40), 147.0 at 5 (48 registers, few spills) and 143.0 at 4, so
// refined launches use MINB = 5.  Double launches use MINB = 4 (64 registers,
// no spills; bound by the FP64 pipe; leaving the allocation unconstrained gave
// 96 registers and 2 blocks per SM).
template <int R, bool HAS_C0, int MINB>
__global__ void __launch_bounds__(BT, MINB) sched_kernel(SchedArgs a) {
  __shared__ __align__(16) unsigned char smem[unit_smem_bytes<R, MINB>()];
  __shared__ double red[BT / 32];
  __shared__ SchedSlot s_state;
  __shared__ SchedProblem s_prob;
  __shared__ int s_slot, s_unit, s_last, s_flag, s_fast;
  const int nslots = a.nslots;
  int cursor = (int)(blockIdx.x % (unsigned)(nslots > 0 ? nslots : 1));
  // slot of this CTA's last unit while its pass may have units left, else -1
  int sticky = -1;
  long long idle_since = -1;
  unsigned long long st[SCHED_NSTATS] = {};
  long long t0 = clock64();
  for (;;) {
    if (tid_flat() < 32) {
      // warp 0 looks at 32 slots per round trip (from the cursor on), then
      // tries the ones with units left in slot order, one lane at a time: the
      // claim and its validation are those of a single thread's scan.
      // (Starting each CTA's tries at a lane of its own spread the CTAs over
      // the slots, but the refined 2048-solve mix ran 3 % slower.)
      const int lane = tid_flat();
      // first the slot of the last unit: one atomic.  A unit of the same
      // pass keeps the slot state, the problem and the acquired grids (pass
      // ids of a slot only grow, so an equal id is the same pass); a unit of
      // a later pass (the pass ended meanwhile) is taken like a scan's claim.
      // Either must be run: a valid claim is never dropped.
      int got = 0, fast = 0;
      if (sticky >= 0) {
        if (lane == 0) {
          const unsigned long long w = atomicAdd(&a.words[sticky], 1ull);
          const int q = claim_next(w);
          if (q < claim_units(w)) {
            if (claim_pass(w) == (s_state.pass & 0xffffu)) {
              s_unit = q;
              got = fast = 1;
            } else {
              got = take_claim(a, sticky, w, q, s_state, s_prob, s_unit);
            }
          }
        }
        got = __shfl_sync(0xffffffffu, got, 0);
        fast = __shfl_sync(0xffffffffu, fast, 0);
        if (!got) sticky = -1;
      }
      // -1 none yet, -3 stop; lane 0 reads the error word so that every lane
      // takes the same path through the ballots below
      int found = got ? sticky : (lane == 0 && *(volatile int*)a.error != 0 ? -3 : -1);
      found = __shfl_sync(0xffffffffu, found, 0);
      for (int base = 0; found == -1 && base < nslots; base += 32) {
        const int si = (cursor + base + lane) % nslots;
        bool cand = false;
        if (base + lane < nslots) {
          const unsigned long long w0 = *(volatile unsigned long long*)&a.words[si];
          cand = claim_next(w0) < claim_units(w0);
        }
        unsigned mask = __ballot_sync(0xffffffffu, cand);
        while (mask && found == -1) {
          const int l = __ffs(mask) - 1;
          mask &= mask - 1;
          int ok = 0;
          st[SCHED_N_TRIES]++;
          if (lane == l) {
            const unsigned long long w = atomicAdd(&a.words[si], 1ull);
            const int q = claim_next(w);
            if (q < claim_units(w)) ok = take_claim(a, si, w, q, s_state, s_prob, s_unit);
          }
          if (__shfl_sync(0xffffffffu, ok, l)) found = __shfl_sync(0xffffffffu, si, l);
        }
      }
      if (lane == 0) {
        s_slot = found;
        s_fast = fast;
        if (found >= 0) {
          cursor = found;
        } else if (found == -1) {
          if (try_admit(a)) s_slot = -2;
          else if (!a.serving && *(volatile int*)a.finished >= a.count) s_slot = -3;
        }
      }
      cursor = __shfl_sync(0xffffffffu, cursor, 0);
    }
    __syncthreads();
    const int si = s_slot;
    long long t1 = clock64();
    if (si == -3) break;
    if (si == -2) {
      st[SCHED_CYC_CLAIM] += t1 - t0;
      t0 = t1;
      continue;
    }
    if (si < 0) {
      // no work anywhere: bounded back-off, then give up
      st[SCHED_N_MISS]++;
      if (tid_flat() == 0) {
        const long long now = clock64();
        if (idle_since < 0) idle_since = now;
        s_flag = (now - idle_since) > a.idle_cycles ? 1 : 0;
        if (!s_flag) __nanosleep(1000);
      }
      __syncthreads();
      const long long t2 = clock64();
      st[SCHED_CYC_IDLE] += t2 - t0;
      t0 = t2;
      if (s_flag) {
        if (tid_flat() == 0 && !a.serving) atomicCAS(a.error, 0, STN_ETIMEOUT);
        break;
      }
      continue;
    }
    st[SCHED_CYC_CLAIM] += t1 - t0;
    st[SCHED_N_FAST] += s_fast;
    idle_since = -1;
    if (!s_fast) __threadfence();  // acquire for every thread: the previous pass's grids
    const SchedSlot S = s_state;
    const SchedProblem P = s_prob;
    const double part = run_unit<R, HAS_C0, MINB>(a, S, P, s_unit, smem, red);
    __syncthreads();  // every thread's writes of this unit precede the release
    const long long t2 = clock64();
    st[SCHED_CYC_UNIT] += t2 - t1;
    st[SCHED_N_UNITS]++;
    if (tid_flat() == 0) {
      P.partials[s_unit] = part;
      __threadfence();
      const int prev = atomicAdd(&a.slots[si].done, 1);
      s_last = prev == S.nunits - 1 ? 1 : 0;
      if (s_last) __threadfence();
    }
    __syncthreads();
    const long long t3 = clock64();
    st[SCHED_CYC_DONE] += t3 - t2;
    sticky = s_last ? -1 : si;  // the last unit's CTA moves the slot to its next pass
    if (s_last) {
      __threadfence();  // acquire for every thread: the other units' partials
      epilogue<R, HAS_C0>(a, si, P, S, red);
      st[SCHED_N_EPI]++;
      const long long t4 = clock64();
      st[SCHED_CYC_EPI] += t4 - t3;
      t0 = t4;
    } else {
      t0 = t3;
    }
  }
  if (a.stats && tid_flat() == 0)
    for (int i = 0; i < SCHED_NSTATS; i++) atomicAdd(&a.stats[i], st[i]);
}

}  // namespace

static unsigned long long* g_stats_dev = nullptr;
static unsigned long long g_stats_host[SCHED_NSTATS];
static cudaStream_t g_stats_stream = nullptr;

void sched_last_stats(unsigned long long* out) {
  if (g_stats_dev && cudaMemcpyAsync(g_stats_host, g_stats_dev, sizeof(g_stats_host), cudaMemcpyDeviceToHost,
                                     g_stats_stream) == cudaSuccess &&
      cudaStreamSynchronize(g_stats_stream) == cudaSuccess)
    memcpy(out, g_stats_host, sizeof(g_stats_host));
  else
    memset(out, 0, sizeof(g_stats_host));
}

int sched_prepare() {
  if (!g_stats_dev) STN_CUDA_TRY(cudaMalloc(&g_stats_dev, sizeof(unsigned long long) * SCHED_NSTATS));
  return STN_OK;
}

void sched_set_stats_stream(cudaStream_t s) { g_stats_stream = s; }

int sched_launch(const SchedArgs& a0, int radius, bool has_c0, int ctas, cudaStream_t s) {
  SchedArgs a = a0;
  if (int rc = sched_prepare()) return rc;
  STN_CUDA_TRY(cudaMemsetAsync(g_stats_dev, 0, sizeof(unsigned long long) * SCHED_NSTATS, s));
  g_stats_stream = s;
  a.stats = g_stats_dev;
#define STN_SCHED(R_, C0_)                                                     \
  do {                                                                         \
    if (a.refined)                                                             \
      sched_kernel<R_, C0_, kSchedMinBlocksRefined><<<ctas, dim3(TX, TY), 0, s>>>(a); \
    else                                                                       \
      sched_kernel<R_, C0_, kSchedMinBlocksPlain><<<ctas, dim3(TX, TY), 0, s>>>(a); \
  } while (0)
  if (radius == 1) {
    if (has_c0) STN_SCHED(1, true);
    else STN_SCHED(1, false);
  } else {
    if (has_c0) STN_SCHED(2, true);
    else STN_SCHED(2, false);
  }
#undef STN_SCHED
  STN_CUDA_TRY(cudaGetLastError());
  return STN_OK;
}

template <int MINB>
static cudaError_t sched_occupancy(int* per_sm, int radius, bool has_c0) {
  if (radius == 1)
    return has_c0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, sched_kernel<1, true, MINB>, BT, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, sched_kernel<1, false, MINB>, BT, 0);
  return has_c0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, sched_kernel<2, true, MINB>, BT, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, sched_kernel<2, false, MINB>, BT, 0);
}

int sched_ctas(int radius, bool has_c0, bool refined) {
  int per_sm = 0;
  const cudaError_t e = refined ? sched_occupancy<kSchedMinBlocksRefined>(&per_sm, radius, has_c0)
                                : sched_occupancy<kSchedMinBlocksPlain>(&per_sm, radius, has_c0);
  if (e != cudaSuccess || per_sm < 1) return -1;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * sms;
}

LaunchPlan batch_unit_plan(i64 nx, i64 ny, i64 nz) {
  const Geo g = make_geo((int)nx, (int)ny, (int)nz);
  LaunchPlan q;
  q.variant = g.shape;
  q.grid_x = g.tiles_x;
  q.grid_y = g.tiles_y;
  q.grid_z = g.kc;
  q.block_threads = BT;
  q.tile_w = tile_width(g.shape);
  q.tile_h = BT / q.tile_w;
  q.kchunk = g.klen;
  q.stage_elems = kPlaneElems;
  return q;
}

// The exact count (each factor fits an int for extents <= 2^20; their product
// need not, and the batched entry points reject problems above 2^22).
i64 sched_units(i64 nx, i64 ny, i64 nz) {
  const Geo g = make_geo((int)nx, (int)ny, (int)nz);
  return (i64)g.tiles_x * g.tiles_y * g.kc;
}

SchedFaults& sched_faults() {
  static SchedFaults f;
  return f;
}

}  // namespace stn
