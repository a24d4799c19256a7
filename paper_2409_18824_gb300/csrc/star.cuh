// Constant-coefficient star-stencil sweep (radius 1 or 2) with an optional
// fused residual reduction -- the Jacobi update of arXiv 2409.18824 Sec. 4
// (Laplace's equation), in the stencil form of Sec. 2.2, with the sum
// reduction of Sec. 5.3 / Listing 8 fused into the same pass.
//
// Design (z-streaming, "2.5D" blocking):
//   * a block owns a TX x TY tile of (i, j) columns and streams a chunk of k
//     planes; i is the contiguous Fortran index, so a warp reads 32
//     consecutive elements of one row (fully coalesced).
//   * each thread keeps its column's k-2R..k+R values in a register queue; the
//     in-plane neighbours (i +- d, j +- d) come from a shared-memory copy of
//     plane k with an R-wide halo;  the next plane's values are loaded before
//     the current plane is computed, so loads overlap arithmetic.
//   * every product and sum is rounded separately in the canonical order (see
//     include/stencil.h and arith.cuh) so double results are bitwise
//     reproducible.
//   * residual modes accumulate rho^2 per thread in double, reduce each block
//     in a fixed shuffle/shared-memory order and write one partial per block;
//     reduce.cu adds the partials in index order, so the norm is deterministic
//     for given extents.
#pragma once
#include <atomic>

#include "arith.cuh"
#include "internal.h"

namespace stn {

namespace {

constexpr int TX = 32;
constexpr int TY = 8;

template <typename T, int R>
struct StarCoeffs {
  T c[R + 1];
};

// Block-wide sum of a per-thread double in a fixed order; result valid in
// thread (0, 0).
template <int NT>
__device__ __forceinline__ double block_sum_fixed(double v, double* red) {
  const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
  const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < NT / 32 ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;
}

// One 32 x 8 tile of columns (tile_x, tile_y) over planes [k0, k1): the body
// of star_kernel, also called in loops by the persistent batched solver.
// Accumulates rho^2 of its points into *rsum in residual modes.  Every thread
// of the block must call it (it uses __syncthreads); `tile` is the block's
// TY+2R x TX+2R shared plane.  The pointers carry no __restrict__: the
// batched solver reads grids that other CTAs of its launch wrote, which must
// go through the coherent load path.
// The tile is tw x th columns (32 x 8 for the standalone kernel, where the
// shape folds to constants; the batched scheduler also uses 16 x 16 for
// narrow problems) with the block's tw * th threads numbered flat, x
// fastest; `plane` is a (th+2R) x (tw+2R) shared array, row pitch tw+2R.
template <typename T, int R, bool HAS_B, bool HAS_C0, int MODE>
__device__ __forceinline__ void star_tile(const T* u, const T* b, T* out, int nx, int ny, int NX, int NY,
                                          int tile_x, int tile_y, int k0, int k1,
                                          const StarCoeffs<T, R>& cf, int tw, int th, T* plane,
                                          double* rsum_io) {
  using A = Arith<T>;
  const int flat = (int)(threadIdx.x + blockDim.x * threadIdx.y);
  const int tx = flat % tw, ty = flat / tw;
  const int pitch = tw + 2 * R;
  const int gi = tile_x * tw + tx + R;  // padded 0-based column index
  const int gj = tile_y * th + ty + R;
  const i64 sy = NX, sz = (i64)NX * NY;
  const bool inx = gi < NX, iny = gj < NY;
  const bool active = (gi < nx + R) && (gj < ny + R);

  // halo duties: x halo for the first/last R lanes, y halo for the first/last R rows
  const bool hx = (tx < R) || (tx >= tw - R);
  const int hx_i = (tx < R) ? gi - R : gi + R;
  const int hx_lx = (tx < R) ? tx : tx + 2 * R;
  const bool hx_ok = hx && hx_i < NX && iny;
  const bool hy = (ty < R) || (ty >= th - R);
  const int hy_j = (ty < R) ? gj - R : gj + R;
  const int hy_ly = (ty < R) ? ty : ty + 2 * R;
  const bool hy_ok = hy && hy_j < NY && inx;

  const T* pc = u + gi + gj * sy;         // this column
  const T* px = u + hx_i + gj * sy;       // x-halo column
  const T* py = u + gi + (i64)hy_j * sy;  // y-halo column
  const bool ld_c = inx && iny;
  T* const me = plane + (ty + R) * pitch + tx + R;  // this column's cell

  T q[2 * R + 1];
#pragma unroll
  for (int m = 0; m < 2 * R + 1; m++) q[m] = ld_c ? pc[(i64)(k0 - R + m) * sz] : T(0);
  T hxv = hx_ok ? px[(i64)k0 * sz] : T(0);
  T hyv = hy_ok ? py[(i64)k0 * sz] : T(0);
  double rsum = *rsum_io;

  for (int k = k0; k < k1; k++) {
    const bool more = k + 1 < k1;
    T qn = T(0), hxn = T(0), hyn = T(0);
    if (more) {
      if (ld_c) qn = pc[(i64)(k + 1 + R) * sz];
      if (hx_ok) hxn = px[(i64)(k + 1) * sz];
      if (hy_ok) hyn = py[(i64)(k + 1) * sz];
    }
    __syncthreads();
    me[0] = q[R];
    if (hx) plane[(ty + R) * pitch + hx_lx] = hxv;
    if (hy) plane[hy_ly * pitch + tx + R] = hyv;
    __syncthreads();
    if (active) {
      T acc = T(0);
#pragma unroll
      for (int d = R; d >= 1; d--) {
        T sx = A::add(me[-d], me[d]);
        T sy_ = A::add(me[-d * pitch], me[d * pitch]);
        T szz = A::add(q[R - d], q[R + d]);
        T s = A::add(A::add(sx, sy_), szz);
        T t = A::mul(cf.c[d], s);
        acc = (d == R) ? t : A::add(acc, t);
      }
      if (HAS_C0) acc = A::add(acc, A::mul(cf.c[0], q[R]));
      if (HAS_B) acc = A::add(acc, b[gi + gj * sy + (i64)k * sz]);
      if (MODE != kResidualOnly) out[gi + gj * sy + (i64)k * sz] = acc;
      if (MODE != kSweep) {
        const double rho = (double)acc - (double)q[R];
        rsum = __fma_rn(rho, rho, rsum);
      }
    }
#pragma unroll
    for (int m = 0; m < 2 * R; m++) q[m] = q[m + 1];
    q[2 * R] = qn;
    hxv = hxn;
    hyv = hyn;
  }
  __syncthreads();  // the tile buffer is free again when this returns
  *rsum_io = rsum;
}

// Two planes per step: the same tile sweep as star_tile, but planes k and
// k+1 are staged together (two shared planes, one pair of barriers per two
// planes) and their two independent updates are interleaved, which doubles
// the independent double operations each thread has in flight.  Same
// arithmetic, same order per point.
template <typename T, int R, bool HAS_B, bool HAS_C0, int MODE>
__device__ __forceinline__ void star_tile2(const T* u, const T* b, T* out, int nx, int ny, int NX,
                                           int NY, int tile_x, int tile_y, int k0, int k1,
                                           const StarCoeffs<T, R>& cf,
                                           T (*tile)[TY + 2 * R][TX + 2 * R], double* rsum_io) {
  using A = Arith<T>;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int gi = tile_x * TX + tx + R;
  const int gj = tile_y * TY + ty + R;
  const i64 sy = NX, sz = (i64)NX * NY;
  const bool inx = gi < NX, iny = gj < NY;
  const bool active = (gi < nx + R) && (gj < ny + R);
  const bool hx = (tx < R) || (tx >= TX - R);
  const int hx_i = (tx < R) ? gi - R : gi + R;
  const int hx_lx = (tx < R) ? tx : tx + 2 * R;
  const bool hx_ok = hx && hx_i < NX && iny;
  const bool hy = (ty < R) || (ty >= TY - R);
  const int hy_j = (ty < R) ? gj - R : gj + R;
  const int hy_ly = (ty < R) ? ty : ty + 2 * R;
  const bool hy_ok = hy && hy_j < NY && inx;
  const T* pc = u + gi + gj * sy;
  const T* px = u + hx_i + gj * sy;
  const T* py = u + gi + (i64)hy_j * sy;
  const bool ld_c = inx && iny;
  constexpr int Q = 2 * R + 2;  // planes k-R .. k+1+R
  T q[Q];
#pragma unroll
  for (int m = 0; m < Q; m++) {
    const int kk = k0 - R + m;
    q[m] = (ld_c && kk <= k1 - 1 + R) ? pc[(i64)kk * sz] : T(0);
  }
  T hx0 = hx_ok ? px[(i64)k0 * sz] : T(0), hy0 = hy_ok ? py[(i64)k0 * sz] : T(0);
  T hx1 = (hx_ok && k0 + 1 < k1) ? px[(i64)(k0 + 1) * sz] : T(0);
  T hy1 = (hy_ok && k0 + 1 < k1) ? py[(i64)(k0 + 1) * sz] : T(0);
  double rsum = *rsum_io;
  for (int k = k0; k < k1; k += 2) {
    const bool two = k + 1 < k1;
    // prefetch the next pair: centre planes k+2+R, k+3+R; halo planes k+2, k+3
    T qn0 = T(0), qn1 = T(0), hxn0 = T(0), hxn1 = T(0), hyn0 = T(0), hyn1 = T(0);
    if (k + 2 < k1) {
      if (ld_c) qn0 = pc[(i64)(k + 2 + R) * sz];
      if (hx_ok) hxn0 = px[(i64)(k + 2) * sz];
      if (hy_ok) hyn0 = py[(i64)(k + 2) * sz];
    }
    if (k + 3 < k1) {
      if (ld_c) qn1 = pc[(i64)(k + 3 + R) * sz];
      if (hx_ok) hxn1 = px[(i64)(k + 3) * sz];
      if (hy_ok) hyn1 = py[(i64)(k + 3) * sz];
    }
    __syncthreads();
    tile[0][ty + R][tx + R] = q[R];
    tile[1][ty + R][tx + R] = q[R + 1];
    if (hx) {
      tile[0][ty + R][hx_lx] = hx0;
      tile[1][ty + R][hx_lx] = hx1;
    }
    if (hy) {
      tile[0][hy_ly][tx + R] = hy0;
      tile[1][hy_ly][tx + R] = hy1;
    }
    __syncthreads();
    if (active) {
      T acc0 = T(0), acc1 = T(0);
#pragma unroll
      for (int d = R; d >= 1; d--) {
        const T sx0 = A::add(tile[0][ty + R][tx + R - d], tile[0][ty + R][tx + R + d]);
        const T sx1 = A::add(tile[1][ty + R][tx + R - d], tile[1][ty + R][tx + R + d]);
        const T sy0 = A::add(tile[0][ty + R - d][tx + R], tile[0][ty + R + d][tx + R]);
        const T sy1 = A::add(tile[1][ty + R - d][tx + R], tile[1][ty + R + d][tx + R]);
        const T sz0 = A::add(q[R - d], q[R + d]);
        const T sz1 = A::add(q[R + 1 - d], q[R + 1 + d]);
        const T s0 = A::add(A::add(sx0, sy0), sz0);
        const T s1 = A::add(A::add(sx1, sy1), sz1);
        const T t0 = A::mul(cf.c[d], s0);
        const T t1 = A::mul(cf.c[d], s1);
        acc0 = (d == R) ? t0 : A::add(acc0, t0);
        acc1 = (d == R) ? t1 : A::add(acc1, t1);
      }
      if (HAS_C0) {
        acc0 = A::add(acc0, A::mul(cf.c[0], q[R]));
        acc1 = A::add(acc1, A::mul(cf.c[0], q[R + 1]));
      }
      const i64 o0 = gi + gj * sy + (i64)k * sz;
      if (HAS_B) {
        acc0 = A::add(acc0, b[o0]);
        if (two) acc1 = A::add(acc1, b[o0 + sz]);
      }
      if (MODE != kResidualOnly) {
        out[o0] = acc0;
        if (two) out[o0 + sz] = acc1;
      }
      if (MODE != kSweep) {
        const double r0 = (double)acc0 - (double)q[R];
        rsum = __fma_rn(r0, r0, rsum);
        if (two) {
          const double r1 = (double)acc1 - (double)q[R + 1];
          rsum = __fma_rn(r1, r1, rsum);
        }
      }
    }
#pragma unroll
    for (int m = 0; m < Q - 2; m++) q[m] = q[m + 2];
    q[Q - 2] = qn0;
    q[Q - 1] = qn1;
    hx0 = hxn0;
    hx1 = hxn1;
    hy0 = hyn0;
    hy1 = hyn1;
  }
  __syncthreads();
  *rsum_io = rsum;
}

template <typename T, int R, bool HAS_B, bool HAS_C0, int MODE>
__global__ void __launch_bounds__(TX* TY)
    star2_kernel(const T* __restrict__ u, const T* __restrict__ b, T* __restrict__ out, int nx,
                 int ny, int nz, int NX, int NY, int kchunk, StarCoeffs<T, R> cf,
                 double* __restrict__ partials) {
  __shared__ T tile[2][TY + 2 * R][TX + 2 * R];
  __shared__ double red[TX * TY / 32];
  const int k0 = R + blockIdx.z * kchunk;
  const int k1 = min(k0 + kchunk, nz + R);
  double rsum = 0.0;
  star_tile2<T, R, HAS_B, HAS_C0, MODE>(u, b, out, nx, ny, NX, NY, blockIdx.x, blockIdx.y, k0, k1, cf,
                                         tile, &rsum);
  if (MODE != kSweep) {
    const double t = block_sum_fixed<TX * TY>(rsum, red);
    if (threadIdx.x == 0 && threadIdx.y == 0)
      partials[blockIdx.x + gridDim.x * ((i64)blockIdx.y + (i64)gridDim.y * blockIdx.z)] = t;
  }
}

template <typename T, int R, bool HAS_B, bool HAS_C0, int MODE>
__global__ void __launch_bounds__(TX* TY)
    star_kernel(const T* __restrict__ u, const T* __restrict__ b, T* __restrict__ out, int nx,
                int ny, int nz, int NX, int NY, int kchunk, StarCoeffs<T, R> cf,
                double* __restrict__ partials) {
  __shared__ T tile[TY + 2 * R][TX + 2 * R];
  __shared__ double red[TX * TY / 32];
  const int k0 = R + blockIdx.z * kchunk;
  const int k1 = min(k0 + kchunk, nz + R);
  double rsum = 0.0;
  star_tile<T, R, HAS_B, HAS_C0, MODE>(u, b, out, nx, ny, NX, NY, blockIdx.x, blockIdx.y, k0, k1, cf, TX, TY,
                                        &tile[0][0], &rsum);
  if (MODE != kSweep) {
    const double t = block_sum_fixed<TX * TY>(rsum, red);
    if (threadIdx.x == 0 && threadIdx.y == 0)
      partials[blockIdx.x + gridDim.x * ((i64)blockIdx.y + (i64)gridDim.y * blockIdx.z)] = t;
  }
}

// ---------------------------------------------------------------------------
// Column variant: no shared memory and no barriers.  A warp covers 32
// consecutive i (the 32 - 2R middle lanes compute, the R lanes at each end
// only load the halo columns); the i neighbours come from the adjacent lanes
// by warp shuffle.  Each thread owns SC_TJ consecutive j rows of its column,
// so the j neighbours are its own registers except for R extra rows above and
// below, which it loads too.  The k neighbours come from a ring of
// Q = 2R+1+PF register planes; the k loop is unrolled Q times so the ring
// rotates by renaming, and plane k+R+PF is loaded before plane k is computed.
// Addresses are 32-bit offsets from a per-plane base.  Arithmetic and its
// order are those of star_kernel.
// ---------------------------------------------------------------------------
constexpr int SC_WARPS = 4;
constexpr int SC_TJ = 8;
// planes of prefetch: two for float (measured best at 512^3), one for double
// (its wider registers would cost occupancy)
template <typename T>
struct ColPF {
  static constexpr int value = sizeof(T) == 4 ? 2 : 1;
};

template <typename T, int R, bool HAS_B, bool HAS_C0, int MODE, int TJ, int PF, int WARPS = SC_WARPS>
__global__ void __launch_bounds__(32 * WARPS)
    star_col_kernel(const T* __restrict__ u, const T* __restrict__ b, T* __restrict__ out, int nx,
                    int ny, int nz, int NX, int NY, int kchunk, StarCoeffs<T, R> cf,
                    double* __restrict__ partials) {
  using A = Arith<T>;
  constexpr int Q = 2 * R + 1 + PF;
  constexpr int CW = 32 - 2 * R;  // computing lanes per warp
  __shared__ double red[WARPS];
  const int lane = threadIdx.x, w = threadIdx.y;
  const int gi = blockIdx.x * CW + lane;  // padded i of this lane (lane R <-> interior column)
  const int j0 = R + (blockIdx.y * WARPS + w) * TJ;
  const i64 sz = (i64)NX * NY;
  const int k0 = R + blockIdx.z * kchunk;
  const int k1 = min(k0 + kchunk, nz + R);
  const bool col_ok = gi < NX;
  const bool lane_c = lane >= R && lane < 32 - R && gi < nx + R;
  // row offsets (elements, 32-bit) from this column's top halo row j0-R
  // rows: 0..R-1 top halo, R..R+TJ-1 own, R+TJ..TJ+2R-1 bottom halo
  constexpr int NR = TJ + 2 * R;
  unsigned roff[NR];
  bool rok[NR];
#pragma unroll
  for (int r2 = 0; r2 < NR; r2++) {
    const int j = j0 - R + r2;
    rok[r2] = col_ok && j < NY;
    roff[r2] = (unsigned)r2 * (unsigned)NX;
  }
  bool act[TJ];
#pragma unroll
  for (int t = 0; t < TJ; t++) act[t] = lane_c && j0 + t < ny + R;
  const T* ubase = u + gi + (i64)(j0 - R) * NX;
  T* obase = out ? out + gi + (i64)(j0 - R) * NX : nullptr;
  const T* bbase = b ? b + gi + (i64)(j0 - R) * NX : nullptr;

  T q[Q][TJ];     // own rows, planes k-R .. k+R+PF
  T hq[Q][2 * R];  // halo rows (R above, R below), planes k .. k+PF (same ring indexing)

  auto load_own = [&](int slot, int kk) {
    const T* p = ubase + (i64)kk * sz;
#pragma unroll
    for (int t = 0; t < TJ; t++) q[slot][t] = rok[R + t] ? p[roff[R + t]] : T(0);
  };
  auto load_halo = [&](int slot, int kk) {
    const T* p = ubase + (i64)kk * sz;
#pragma unroll
    for (int h = 0; h < R; h++) {
      hq[slot][h] = rok[h] ? p[roff[h]] : T(0);
      hq[slot][R + h] = rok[R + TJ + h] ? p[roff[R + TJ + h]] : T(0);
    }
  };
#pragma unroll
  for (int m = 0; m < Q - 1; m++) {
    const int kk = k0 - R + m;
    if (kk <= k1 - 1 + R) load_own(m, kk);
  }
#pragma unroll
  for (int m = 0; m < PF; m++)
    if (k0 + m < k1) load_halo(m, k0 + m);
  double rsum = 0.0;

  for (int kb = k0; kb < k1; kb += Q) {
#pragma unroll
    for (int J = 0; J < Q; J++) {
      const int k = kb + J;
      if (k >= k1) break;
      if (k + PF < k1) {
        load_own((J + Q - 1) % Q, k + R + PF);
        load_halo((J + PF) % Q, k + PF);
      }
      const T* qc = q[(J + R) % Q];
      const T* hc = hq[J % Q];
      const i64 ko = (i64)k * sz;
      T* op = MODE != kResidualOnly ? obase + ko : nullptr;
      const T* bp = HAS_B ? bbase + ko : nullptr;
#pragma unroll
      for (int t = 0; t < TJ; t++) {
        const T c = qc[t];
        T acc = T(0);
#pragma unroll
        for (int d = R; d >= 1; d--) {
          const T xm = __shfl_up_sync(0xffffffffu, c, d);
          const T xp = __shfl_down_sync(0xffffffffu, c, d);
          const T ym = t - d >= 0 ? qc[t - d] : hc[t - d + R];
          const T yp = t + d < TJ ? qc[t + d] : hc[R + t + d - TJ];
          const T zm = q[(J + R - d) % Q][t], zp = q[(J + R + d) % Q][t];
          const T s = A::add(A::add(A::add(xm, xp), A::add(ym, yp)), A::add(zm, zp));
          const T tt = A::mul(cf.c[d], s);
          acc = (d == R) ? tt : A::add(acc, tt);
        }
        if (HAS_C0) acc = A::add(acc, A::mul(cf.c[0], c));
        if (act[t]) {
          if (HAS_B) acc = A::add(acc, bp[roff[R + t]]);
          if (MODE != kResidualOnly) op[roff[R + t]] = acc;
          if (MODE != kSweep) {
            const double rho = (double)acc - (double)c;
            rsum = __fma_rn(rho, rho, rsum);
          }
        }
      }
    }
  }
  if (MODE != kSweep) {
    const double t = block_sum_fixed<32 * WARPS>(rsum, red);
    if (lane == 0 && w == 0)
      partials[blockIdx.x + gridDim.x * ((i64)blockIdx.y + (i64)gridDim.y * blockIdx.z)] = t;
  }
}

// ---------------------------------------------------------------------------
// Staged variant: a block owns `rg` interior rows j (whole rows in i) of a
// chunk of planes.  The planes stream through a ring of 2R + 1 + SG_PF
// shared-memory stages: the rg + 2R rows a plane contributes are one
// contiguous span of the grid, fetched as 16-byte asynchronous copies
// (cp.async.cg) of the 16-byte-aligned chunks covering it, SG_PF planes ahead
// of the 2R + 1 in use, and waited for with cp.async.wait_group (a hardware
// wait, no spin loop).  Chunks that would
// reach outside the grid's own bytes (an unaligned first or last element)
// are copied element by element instead, so nothing outside [u, u + count)
// is read.  The bytes in flight live in shared memory, not in registers.
// Every operand of an update comes from shared memory; results are stored
// straight to global memory.  Arithmetic and its order are those of
// star_kernel.
// ---------------------------------------------------------------------------
// One plane in flight beyond the 2R+1 in use, with a ring as deep in rows
// as an SM's shared memory allows (one block per SM), measured fastest at
// 512^3 float: 701 GLUP/s, against 598 with two blocks per SM and 526-572
// with two or three planes in flight.
constexpr int SG_WARPS = 16;
constexpr int SG_PF = 1;

__device__ __forceinline__ void sg_cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void sg_cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename T, int R, bool HAS_B, bool HAS_C0, int MODE>
__global__ void __launch_bounds__(32 * SG_WARPS)
    star_staged_kernel(const T* __restrict__ u, const T* __restrict__ b, T* __restrict__ out, int nx, int ny,
                       int nz, int NX, int NY, int kchunk, int rg, int stage_elems, StarCoeffs<T, R> cf,
                       double* __restrict__ partials) {
  using A = Arith<T>;
  constexpr int S = 2 * R + 1 + SG_PF;
  constexpr int WIN = 2 * R + 1;
  extern __shared__ __align__(16) unsigned char sg_smem[];
  T* const ring = reinterpret_cast<T*>(sg_smem);
  __shared__ double red[SG_WARPS];  // block_sum_fixed reads SG_WARPS slots: fewer warps leave 0.0
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < SG_WARPS) red[tid] = 0.0;
  const int NT = (int)blockDim.x;
  const int j0 = R + (int)blockIdx.y * rg;  // first interior row of the block (padded index)
  const int rows = min(rg, ny + R - j0);
  const int k0 = R + (int)blockIdx.z * kchunk;
  const int k1 = min(k0 + kchunk, nz + R);
  const int pfirst = k0 - R, plast = k1 - 1 + R;  // planes staged
  const i64 psz = (i64)NX * NY;
  const i64 n_el = (i64)(rows + 2 * R) * NX;  // elements a plane contributes
  const uintptr_t gbase = reinterpret_cast<uintptr_t>(u);
  const uintptr_t gend = gbase + (uintptr_t)(psz * (i64)(nz + 2 * R)) * sizeof(T);

  // element offset of plane p's first staged element (row j0 - R, i = 0); in
  // its stage it sits shift(p) elements past the chunk grid's start (the
  // aligned address below it), and shift advances by psz modulo the
  // elements per 16-byte chunk from one plane to the next
  constexpr int EPC = 16 / (int)sizeof(T);
  auto first = [&](int p) -> i64 { return ((i64)p * NY + (j0 - R)) * NX; };
  const int shift0 = (int)(((gbase + (uintptr_t)first(pfirst) * sizeof(T)) & 15u) / sizeof(T));
  const int pstep = (int)(psz & (EPC - 1));
  auto shift_of = [&](int p) -> int { return (shift0 + (p - pfirst) * pstep) & (EPC - 1); };
  const unsigned ring_s = (unsigned)__cvta_generic_to_shared(ring);
  auto issue = [&](int p, int slot) {
    if (p <= plast) {
      const uintptr_t addr = gbase + (uintptr_t)first(p) * sizeof(T);
      const uintptr_t a0 = addr & ~(uintptr_t)15;
      const int nch = (int)((addr - a0 + (uintptr_t)n_el * sizeof(T) + 15) >> 4);
      // chunks [c_lo, c_hi) lie inside the grid's bytes; at most the first and
      // the last reach outside it, and those go element by element
      const int c_lo = a0 < gbase ? 1 : 0;
      const int c_hi = a0 + ((uintptr_t)nch << 4) > gend ? nch - 1 : nch;
      const unsigned dst = ring_s + (unsigned)(slot * stage_elems * (int)sizeof(T));
      const char* src = reinterpret_cast<const char*>(a0);
      for (int c = c_lo + tid; c < c_hi; c += NT) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + (unsigned)c * 16u),
                     "l"(src + (size_t)c * 16)
                     : "memory");
      }
      const int edge = tid == 0 ? (c_lo ? 0 : -1) : (tid == NT - 1 && c_hi < nch && nch - 1 >= c_lo ? nch - 1 : -1);
      if (edge >= 0) {
        T* d = ring + slot * stage_elems + edge * EPC;
        const T* g = reinterpret_cast<const T*>(a0) + edge * EPC;
        for (int e = 0; e < EPC; e++) {
          const uintptr_t sa = reinterpret_cast<uintptr_t>(g + e);
          if (sa >= gbase && sa < gend) d[e] = g[e];
        }
      }
    }
    sg_cp_async_commit();  // one group per plane slot, empty past the last plane
  };

  for (int q = 0; q < S; q++) issue(pfirst + q, q);
  int slot_k = R;  // ring slot of plane k (plane p sits in slot (p - pfirst) mod S)
  double rsum = 0.0;
  const int ntx = (nx + 31) / 32;
  const int nw = (int)(blockDim.x >> 5);
  for (int k = k0; k < k1; k++) {
    sg_cp_async_wait<SG_PF>();  // this thread's copies of planes <= k + R are done
    __syncthreads();            // and everyone's
    // 32-bit element offsets of the planes in the ring (shared-memory
    // addressing): plane k, and the distances to planes k -+ d from it
    const int ok = slot_k * stage_elems + shift_of(k);
    int dm[R], dp[R];
#pragma unroll
    for (int d = 1; d <= R; d++) {
      const int sm = slot_k - d < 0 ? slot_k - d + S : slot_k - d;
      const int sp = slot_k + d >= S ? slot_k + d - S : slot_k + d;
      dm[d - 1] = sm * stage_elems + shift_of(k - d) - ok;
      dp[d - 1] = sp * stage_elems + shift_of(k + d) - ok;
    }
    // a warp takes a 32-wide i segment and walks down the block's rows with
    // the 2R+1 centres around the current row in registers (j neighbours);
    // i neighbours and k neighbours come from the ring
    for (int tx = warp; tx < ntx; tx += nw) {
      const int i = R + tx * 32 + lane;
      if (i < nx + R) {
        int e = ok + R * NX + i;
        i64 go = ((i64)k * NY + j0) * NX + i;
        T w[WIN];
#pragma unroll
        for (int q = 0; q < WIN; q++) w[q] = ring[ok + q * NX + i];
        // unrolled by the window length, so the window rotates by renaming
#pragma unroll WIN
        for (int row = 0; row < rows; row++) {
          const T c = w[R];
          T acc = T(0);
#pragma unroll
          for (int d = R; d >= 1; d--) {
            const T sx = A::add(ring[e - d], ring[e + d]);
            const T sy = A::add(w[R - d], w[R + d]);
            const T sz = A::add(ring[e + dm[d - 1]], ring[e + dp[d - 1]]);
            const T sv = A::add(A::add(sx, sy), sz);
            const T t = A::mul(cf.c[d], sv);
            acc = (d == R) ? t : A::add(acc, t);
          }
          if (HAS_C0) acc = A::add(acc, A::mul(cf.c[0], c));
          if (HAS_B) acc = A::add(acc, b[go]);
          if (MODE != kResidualOnly) out[go] = acc;
          if (MODE != kSweep) {
            const double rho = (double)acc - (double)c;
            rsum = __fma_rn(rho, rho, rsum);
          }
#pragma unroll
          for (int q = 0; q < 2 * R; q++) w[q] = w[q + 1];
          if (row + 1 < rows) w[2 * R] = ring[e + (R + 1) * NX];
          e += NX;
          go += NX;
        }
      }
    }
    __syncthreads();      // plane k - R's stage is free again
    const int s_free = slot_k - R < 0 ? slot_k - R + S : slot_k - R;
    issue(k - R + S, s_free);  // the plane S ahead goes into it
    slot_k = slot_k + 1 == S ? 0 : slot_k + 1;
  }
  sg_cp_async_wait<0>();  // no copy in flight at exit
  if (MODE != kSweep) {
    const double t = block_sum_fixed<32 * SG_WARPS>(rsum, red);
    if (tid == 0) partials[blockIdx.x + gridDim.x * ((i64)blockIdx.y + (i64)gridDim.y * blockIdx.z)] = t;
  }
}

template <typename T>
__global__ void copy_halo_kernel(const T* __restrict__ src, T* __restrict__ dst, int nx, int ny,
                                 int nz, int r) {
  const int NX = nx + 2 * r, NY = ny + 2 * r, NZ = nz + 2 * r;
  const i64 rows = (i64)NY * NZ;
  const int lane = threadIdx.x & 31;
  const i64 warp0 = ((i64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const i64 nwarps = ((i64)gridDim.x * blockDim.x) >> 5;
  for (i64 row = warp0; row < rows; row += nwarps) {
    const int j = (int)(row % NY), k = (int)(row / NY);
    const i64 base = row * NX;
    if (k < r || k >= nz + r || j < r || j >= ny + r) {
      for (int i = lane; i < NX; i += 32) dst[base + i] = src[base + i];
    } else if (lane < 2 * r) {
      const int i = lane < r ? lane : nx + lane;  // lanes r..2r-1 -> nx+r .. nx+2r-1
      dst[base + i] = src[base + i];
    }
  }
}

template <typename T, int R, bool HAS_B, bool HAS_C0>
int launch_star_t(const T* u, const T* b, T* out, const Grid& g, const double* coeffs,
                  SweepMode mode, double* partials, cudaStream_t s, const ZPlan& p) {
  const int variant = p.variant;  // the plan's own: a staged request whose ring does not fit runs the plane kernel
  star_last().variant = variant;
  star_last().chunks = p.chunks;
  StarCoeffs<T, R> cf;
  for (int d = 0; d <= R; d++) cf.c[d] = (T)coeffs[d];
  dim3 grid(p.tiles_x, p.tiles_y, p.chunks);
  const int nx = (int)g.nx, ny = (int)g.ny, nz = (int)g.nz, NX = (int)g.NX(), NY = (int)g.NY();
#define STN_LAUNCH_MODES(KERNEL_EXPR, BLOCK)                                                     \
  switch (mode) {                                                                                \
    case kSweep: KERNEL_EXPR(kSweep)<<<grid, BLOCK, 0, s>>>(u, b, out, nx, ny, nz, NX, NY, p.kchunk, cf, partials); break; \
    case kSweepResidual: KERNEL_EXPR(kSweepResidual)<<<grid, BLOCK, 0, s>>>(u, b, out, nx, ny, nz, NX, NY, p.kchunk, cf, partials); break; \
    default: KERNEL_EXPR(kResidualOnly)<<<grid, BLOCK, 0, s>>>(u, b, out, nx, ny, nz, NX, NY, p.kchunk, cf, partials); break; \
  }
#define STN_SCALAR(M) star_kernel<T, R, HAS_B, HAS_C0, M>
#define STN_COL(M) star_col_kernel<T, R, HAS_B, HAS_C0, M, SC_TJ, ColPF<T>::value>
#define STN_PLANE2(M) star2_kernel<T, R, HAS_B, HAS_C0, M>
  if (variant == kStarStaged) {
    // the staged kernels take their shared-memory ring as dynamic memory
    // per device and mode: the attribute is set (setting it twice is harmless)
    static std::atomic<bool> attr_set[64][3];
    const int m = mode == kSweep ? 0 : (mode == kSweepResidual ? 1 : 2);
    auto kern = m == 0 ? star_staged_kernel<T, R, HAS_B, HAS_C0, kSweep>
                       : (m == 1 ? star_staged_kernel<T, R, HAS_B, HAS_C0, kSweepResidual>
                                 : star_staged_kernel<T, R, HAS_B, HAS_C0, kResidualOnly>);
    int dev = 0;
    STN_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr_set[dev][m].load(std::memory_order_relaxed)) {
      STN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kStagedSmemMax));
      if (dev >= 0 && dev < 64) attr_set[dev][m].store(true, std::memory_order_relaxed);
    }
    // one warp per 32-wide i segment, at most SG_WARPS
    const int nw = (int)std::min<i64>((g.nx + 31) / 32, SG_WARPS);
    kern<<<grid, 32 * nw, p.smem, s>>>(u, b, out, nx, ny, nz, NX, NY, p.kchunk, p.rg, p.stage_elems, cf, partials);
    STN_CUDA_TRY(cudaGetLastError());
    return STN_OK;
  }
  if (variant == kStarColumn) {
    STN_LAUNCH_MODES(STN_COL, dim3(32, SC_WARPS))
  } else if (variant == kStarPlane2) {
    STN_LAUNCH_MODES(STN_PLANE2, dim3(TX, TY))
  } else {
    STN_LAUNCH_MODES(STN_SCALAR, dim3(TX, TY))
  }
#undef STN_SCALAR
#undef STN_COL
#undef STN_PLANE2
#undef STN_LAUNCH_MODES
  STN_CUDA_TRY(cudaGetLastError());
  return STN_OK;
}

}  // namespace

template <typename T>
int launch_star(const T* u, const T* b, T* out, const Grid& g, const double* coeffs,
                SweepMode mode, double* partials, cudaStream_t s, i64 max_partials, i64* nparts) {
  const bool hb = b != nullptr, hc0 = coeffs[0] != 0.0;
  // One plan for the whole launch: the knobs and the tuning cache may change
  // on another thread, so the partial count checked here, the grid launched
  // and the count returned for the reduction all come from this one plan.
  const ZPlan v = plan_star(g, star_variant(g, sizeof(T), u, b, out), sizeof(T));
  if (int rc = check_launch_grid(v.tiles_x, v.tiles_y, v.chunks)) return rc;
  if (mode != kSweep && max_partials >= 0 && v.blocks() > max_partials) {
    set_error("invalid argument: the launch plan needs " + std::to_string(v.blocks()) +
              " partial sums, more than the " + std::to_string(max_partials) + " slots given");
    return STN_EINVAL;
  }
  if (nparts) *nparts = v.blocks();
  if (g.r == 1) {
    if (hb) return hc0 ? launch_star_t<T, 1, true, true>(u, b, out, g, coeffs, mode, partials, s, v)
                       : launch_star_t<T, 1, true, false>(u, b, out, g, coeffs, mode, partials, s, v);
    return hc0 ? launch_star_t<T, 1, false, true>(u, b, out, g, coeffs, mode, partials, s, v)
               : launch_star_t<T, 1, false, false>(u, b, out, g, coeffs, mode, partials, s, v);
  }
  if (hb) return hc0 ? launch_star_t<T, 2, true, true>(u, b, out, g, coeffs, mode, partials, s, v)
                     : launch_star_t<T, 2, true, false>(u, b, out, g, coeffs, mode, partials, s, v);
  return hc0 ? launch_star_t<T, 2, false, true>(u, b, out, g, coeffs, mode, partials, s, v)
             : launch_star_t<T, 2, false, false>(u, b, out, g, coeffs, mode, partials, s, v);
}

template <typename T>
int launch_copy_halo(const T* src, T* dst, const Grid& g, cudaStream_t s) {
  const i64 rows = g.NY() * g.NZ();
  i64 blocks = (rows + 7) / 8;
  if (blocks > 152 * 16) blocks = 152 * 16;
  copy_halo_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(src, dst, (int)g.nx, (int)g.ny, (int)g.nz, g.r);
  STN_CUDA_TRY(cudaGetLastError());
  return STN_OK;
}


}  // namespace stn
