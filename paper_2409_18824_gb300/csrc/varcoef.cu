// Variable-coefficient star operator (radius 1 or 2) for the Poisson solves:
//   (A u)(p) = sum_{d} w_d sum_{q = p +- d e_axis} kappa(p,q) (u(p) - u(q)),
//   kappa(p,q) = (a(p) + a(q)) / 2,
// the Jacobi update u'(p) = (f(p) + N(p)) / D(p), its application and its
// residual f - A u.  arXiv 2409.18824 states only Laplace's equation (Sec. 4);
// this symmetric M-matrix form is the reading used for the variable-
// coefficient workload.  D and N are accumulated d = 1..R, axis x, y, z, minus
// neighbour first, every operation rounded separately (bitwise equal to the
// CPU oracle in double).
//
// Same z-streaming structure as sweep.cu, with two staged fields (u and a):
// register queues along k for both, shared-memory planes with an R halo for
// the in-plane neighbours.
#include <atomic>

#include "arith.cuh"
#include "internal.h"

namespace stn {

namespace {

constexpr int TX = 32;
constexpr int TY = 8;

template <typename T, int R>
struct VarW {
  T w[R + 1];
};

template <typename T, int R>
__device__ __forceinline__ void accum(T& D, T& N, T ap, T aq, T uq, T wd) {
  using A = Arith<T>;
  const T kap = A::mul(T(0.5), A::add(ap, aq));
  const T t = A::mul(wd, kap);
  D = A::add(D, t);
  N = A::add(N, A::mul(t, uq));
}

template <typename T, int R, int MODE>
__global__ void __launch_bounds__(TX* TY)
    var_kernel(const T* __restrict__ u, const T* __restrict__ a, const T* __restrict__ f,
               T* __restrict__ out, int nx, int ny, int nz, int NX, int NY, int kchunk,
               VarW<T, R> wt, double* __restrict__ partials, double* __restrict__ partials_max) {
  using A = Arith<T>;
  __shared__ T tu[TY + 2 * R][TX + 2 * R];
  __shared__ T ta[TY + 2 * R][TX + 2 * R];
  __shared__ double red[TX * TY / 32];
  __shared__ double redm[TX * TY / 32];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int gi = blockIdx.x * TX + tx + R;
  const int gj = blockIdx.y * TY + ty + R;
  const i64 sy = NX, sz = (i64)NX * NY;
  const int k0 = R + blockIdx.z * kchunk;
  const int k1 = min(k0 + kchunk, nz + R);
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
  const i64 oc = gi + gj * sy, ox = hx_i + gj * sy, oy = gi + (i64)hy_j * sy;
  const bool ld_c = inx && iny;

  T qu[2 * R + 1], qa[2 * R + 1];
#pragma unroll
  for (int m = 0; m < 2 * R + 1; m++) {
    const i64 o = oc + (i64)(k0 - R + m) * sz;
    qu[m] = ld_c ? u[o] : T(0);
    qa[m] = ld_c ? a[o] : T(0);
  }
  T hxu = hx_ok ? u[ox + (i64)k0 * sz] : T(0), hxa = hx_ok ? a[ox + (i64)k0 * sz] : T(0);
  T hyu = hy_ok ? u[oy + (i64)k0 * sz] : T(0), hya = hy_ok ? a[oy + (i64)k0 * sz] : T(0);
  double rsum = 0.0, rmax = 0.0;

  for (int k = k0; k < k1; k++) {
    const bool more = k + 1 < k1;
    T qun = T(0), qan = T(0), hxun = T(0), hxan = T(0), hyun = T(0), hyan = T(0);
    if (more) {
      if (ld_c) {
        qun = u[oc + (i64)(k + 1 + R) * sz];
        qan = a[oc + (i64)(k + 1 + R) * sz];
      }
      if (hx_ok) {
        hxun = u[ox + (i64)(k + 1) * sz];
        hxan = a[ox + (i64)(k + 1) * sz];
      }
      if (hy_ok) {
        hyun = u[oy + (i64)(k + 1) * sz];
        hyan = a[oy + (i64)(k + 1) * sz];
      }
    }
    __syncthreads();
    tu[ty + R][tx + R] = qu[R];
    ta[ty + R][tx + R] = qa[R];
    if (hx) {
      tu[ty + R][hx_lx] = hxu;
      ta[ty + R][hx_lx] = hxa;
    }
    if (hy) {
      tu[hy_ly][tx + R] = hyu;
      ta[hy_ly][tx + R] = hya;
    }
    __syncthreads();
    if (active) {
      const T ap = qa[R], up = qu[R];
      T D = T(0), N = T(0);
#pragma unroll
      for (int d = 1; d <= R; d++) {
        const T wd = wt.w[d];
        accum<T, R>(D, N, ap, ta[ty + R][tx + R - d], tu[ty + R][tx + R - d], wd);
        accum<T, R>(D, N, ap, ta[ty + R][tx + R + d], tu[ty + R][tx + R + d], wd);
        accum<T, R>(D, N, ap, ta[ty + R - d][tx + R], tu[ty + R - d][tx + R], wd);
        accum<T, R>(D, N, ap, ta[ty + R + d][tx + R], tu[ty + R + d][tx + R], wd);
        accum<T, R>(D, N, ap, qa[R - d], qu[R - d], wd);
        accum<T, R>(D, N, ap, qa[R + d], qu[R + d], wd);
      }
      const i64 o = oc + (i64)k * sz;
      if (MODE == kVarSweep) {
        out[o] = A::div(A::add(f[o], N), D);
      } else if (MODE == kVarApply) {
        out[o] = A::add(A::mul(D, up), -N);
      } else {
        const T au = A::add(A::mul(D, up), -N);
        const double rho = (double)A::add(f[o], -au);
        rsum = __fma_rn(rho, rho, rsum);
        if (MODE == kVarRefine) {
          out[o] = (T)rho;
          rmax = fmax(rmax, fabs(rho));
        }
      }
    }
#pragma unroll
    for (int m = 0; m < 2 * R; m++) {
      qu[m] = qu[m + 1];
      qa[m] = qa[m + 1];
    }
    qu[2 * R] = qun;
    qa[2 * R] = qan;
    hxu = hxun;
    hxa = hxan;
    hyu = hyun;
    hya = hyan;
  }
  if (MODE == kVarResidual || MODE == kVarRefine) {
    const int lane = (ty * TX + tx) & 31, warp = (ty * TX + tx) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
      rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    }
    if (lane == 0) {
      red[warp] = rsum;
      redm[warp] = rmax;
    }
    __syncthreads();
    if (tx == 0 && ty == 0) {
      double t = 0.0, m = 0.0;
      for (int w = 0; w < TX * TY / 32; w++) {
        t += red[w];
        m = fmax(m, redm[w]);
      }
      const i64 bid = blockIdx.x + gridDim.x * ((i64)blockIdx.y + (i64)gridDim.y * blockIdx.z);
      partials[bid] = t;
      if (MODE == kVarRefine) partials_max[bid] = m;
    }
  }
}

// ---------------------------------------------------------------------------
// Column variant (default): no shared memory, no barriers.  As in the star
// column kernel, a warp covers 32 consecutive i (the 32 - 2R middle lanes
// compute), each thread owns TJ consecutive j rows plus R halo rows above and
// below, and k comes from register rings (planes k-R..k+R and one plane of
// prefetch; the loop is unrolled by the ring length so the rings rotate by
// renaming).
//
// Face coefficients are computed once per face: t = hw_d * (a(p) + a(q)),
// hw_d = w_d / 2.  That is bitwise the oracle's w_d * (0.5 * (a(p)+a(q))),
// because halving a normal number is exact, so both are one rounding of the
// same real product, and addition commutes, so a face has one value seen from
// either side.  A lane's minus x-face is its left neighbour's plus x-face (one
// shuffle), and a j-face between two rows of the same thread serves both.  D
// and N are then accumulated in the oracle's order (d = 1..R; axis x, y, z;
// minus before plus), each operation rounded separately.
// ---------------------------------------------------------------------------
constexpr int VC_WARPS = 2;  // measured: 2 warps of 4 rows beat 4 warps (register-limited occupancy)
template <typename T>
struct VarColTJ {
  static constexpr int value = sizeof(T) == 4 ? 4 : 2;
};

template <typename T, int R, int MODE, int TJ>
__global__ void __launch_bounds__(32 * VC_WARPS)
    var_col_kernel(const T* __restrict__ u, const T* __restrict__ a, const T* __restrict__ f,
                   T* __restrict__ out, int nx, int ny, int nz, int NX, int NY, int kchunk,
                   VarW<T, R> hw, double* __restrict__ partials, double* __restrict__ partials_max) {
  using A = Arith<T>;
  constexpr int Q = 2 * R + 2;   // ring: planes k-R .. k+R and the prefetched k+R+1
  constexpr int CW = 32 - 2 * R;  // computing lanes per warp
  constexpr int NR = TJ + 2 * R;  // rows of a thread: R top halo, TJ own, R bottom halo
  constexpr bool NEED_F = MODE != kVarApply;
  __shared__ double red[VC_WARPS], redm[VC_WARPS];
  const int lane = threadIdx.x, w = threadIdx.y;
  const int gi = blockIdx.x * CW + lane;
  const int j0 = R + (blockIdx.y * VC_WARPS + w) * TJ;
  const i64 sz = (i64)NX * NY;
  const int k0 = R + blockIdx.z * kchunk;
  const int k1 = min(k0 + kchunk, nz + R);
  const bool col_ok = gi < NX;
  const bool lane_c = lane >= R && lane < 32 - R && gi < nx + R;
  unsigned roff[NR];
  bool rok[NR];
#pragma unroll
  for (int r2 = 0; r2 < NR; r2++) {
    rok[r2] = col_ok && j0 - R + r2 < NY;
    roff[r2] = (unsigned)r2 * (unsigned)NX;
  }
  bool act[TJ];
#pragma unroll
  for (int t = 0; t < TJ; t++) act[t] = lane_c && j0 + t < ny + R;
  const i64 base = gi + (i64)(j0 - R) * NX;
  const T* ub = u + base;
  const T* ab = a + base;

  T qu[Q][TJ], qa[Q][TJ];      // own rows, planes by ring slot
  T hu[2][2 * R], ha[2][2 * R];  // halo rows (R top, R bottom) at planes k, k+1
  T fq[2][TJ];                   // f of own rows at planes k, k+1

  auto load_own = [&](int slot, int kk) {
    const i64 po = (i64)kk * sz;
#pragma unroll
    for (int t = 0; t < TJ; t++) {
      qu[slot][t] = rok[R + t] ? ub[po + roff[R + t]] : T(0);
      qa[slot][t] = rok[R + t] ? ab[po + roff[R + t]] : T(0);
    }
  };
  auto load_halo = [&](int hs, int kk) {
    const i64 po = (i64)kk * sz;
#pragma unroll
    for (int h = 0; h < R; h++) {
      hu[hs][h] = rok[h] ? ub[po + roff[h]] : T(0);
      ha[hs][h] = rok[h] ? ab[po + roff[h]] : T(0);
      hu[hs][R + h] = rok[R + TJ + h] ? ub[po + roff[R + TJ + h]] : T(0);
      ha[hs][R + h] = rok[R + TJ + h] ? ab[po + roff[R + TJ + h]] : T(0);
    }
  };
  auto load_f = [&](int fs, int kk) {
    if (NEED_F) {
      const T* fb = f + base + (i64)kk * sz;
#pragma unroll
      for (int t = 0; t < TJ; t++) fq[fs][t] = rok[R + t] ? fb[roff[R + t]] : T(0);
    }
  };
#pragma unroll
  for (int m = 0; m < Q - 1; m++) {
    const int kk = k0 - R + m;
    if (kk <= k1 - 1 + R) load_own(m, kk);
  }
  if (k0 < k1) {
    load_halo(0, k0);
    load_f(0, k0);
  }
  double rsum = 0.0, rmax = 0.0;

  for (int kb = k0; kb < k1; kb += Q) {
#pragma unroll
    for (int J = 0; J < Q; J++) {
      const int k = kb + J;
      if (k >= k1) break;
      if (k + 1 < k1) {
        load_own((J + Q - 1) % Q, k + R + 1);
        load_halo((J + 1) & 1, k + 1);
        load_f((J + 1) & 1, k + 1);
      }
      const T* cu = qu[(J + R) % Q];
      const T* ca = qa[(J + R) % Q];
      const int hs = J & 1;
      // the thread's column of a and u at plane k, rows -R .. TJ+R-1
      T colA[NR], colU[NR];
#pragma unroll
      for (int r2 = 0; r2 < NR; r2++) {
        if (r2 < R) {
          colA[r2] = ha[hs][r2];
          colU[r2] = hu[hs][r2];
        } else if (r2 < R + TJ) {
          colA[r2] = ca[r2 - R];
          colU[r2] = cu[r2 - R];
        } else {
          colA[r2] = ha[hs][r2 - TJ];
          colU[r2] = hu[hs][r2 - TJ];
        }
      }
      T D[TJ], N[TJ];
#pragma unroll
      for (int t = 0; t < TJ; t++) {
        D[t] = T(0);
        N[t] = T(0);
      }
#pragma unroll
      for (int d = 1; d <= R; d++) {
        const T h = hw.w[d];
        // j-faces (r, r+d) for r = -d .. TJ-1, stored at [r + d]
        T ty[TJ + R];
#pragma unroll
        for (int r = -d; r < TJ; r++) ty[r + d] = A::mul(h, A::add(colA[R + r], colA[R + r + d]));
#pragma unroll
        for (int t = 0; t < TJ; t++) {
          const T c_a = ca[t];
          const T txp = A::mul(h, A::add(c_a, __shfl_down_sync(0xffffffffu, c_a, d)));
          const T txm = __shfl_up_sync(0xffffffffu, txp, d);
          const T uxm = __shfl_up_sync(0xffffffffu, cu[t], d);
          const T uxp = __shfl_down_sync(0xffffffffu, cu[t], d);
          const T tzm = A::mul(h, A::add(c_a, qa[(J + R - d) % Q][t]));
          const T tzp = A::mul(h, A::add(c_a, qa[(J + R + d) % Q][t]));
          D[t] = A::add(D[t], txm);
          N[t] = A::add(N[t], A::mul(txm, uxm));
          D[t] = A::add(D[t], txp);
          N[t] = A::add(N[t], A::mul(txp, uxp));
          D[t] = A::add(D[t], ty[t]);
          N[t] = A::add(N[t], A::mul(ty[t], colU[R + t - d]));
          D[t] = A::add(D[t], ty[t + d]);
          N[t] = A::add(N[t], A::mul(ty[t + d], colU[R + t + d]));
          D[t] = A::add(D[t], tzm);
          N[t] = A::add(N[t], A::mul(tzm, qu[(J + R - d) % Q][t]));
          D[t] = A::add(D[t], tzp);
          N[t] = A::add(N[t], A::mul(tzp, qu[(J + R + d) % Q][t]));
        }
      }
      const i64 po = (i64)k * sz;
#pragma unroll
      for (int t = 0; t < TJ; t++) {
        if (!act[t]) continue;
        const i64 o = base + po + roff[R + t];
        if (MODE == kVarSweep) {
          out[o] = A::div(A::add(fq[hs][t], N[t]), D[t]);
        } else if (MODE == kVarApply) {
          out[o] = A::add(A::mul(D[t], cu[t]), -N[t]);
        } else {
          const T au = A::add(A::mul(D[t], cu[t]), -N[t]);
          const double rho = (double)A::add(fq[hs][t], -au);
          rsum = __fma_rn(rho, rho, rsum);
          if (MODE == kVarRefine) {
            out[o] = (T)rho;
            rmax = fmax(rmax, fabs(rho));
          }
        }
      }
    }
  }
  if (MODE == kVarResidual || MODE == kVarRefine) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
      rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    }
    if (lane == 0) {
      red[w] = rsum;
      redm[w] = rmax;
    }
    __syncthreads();
    if (lane == 0 && w == 0) {
      double t = 0.0, m = 0.0;
      for (int q = 0; q < VC_WARPS; q++) {
        t += red[q];
        m = fmax(m, redm[q]);
      }
      const i64 bid = blockIdx.x + gridDim.x * ((i64)blockIdx.y + (i64)gridDim.y * blockIdx.z);
      partials[bid] = t;
      if (MODE == kVarRefine) partials_max[bid] = m;
    }
  }
}

template <typename T, int R, int TJ>
int launch_var_col_t(const T* u, const T* a, const T* f, T* out, const Grid& g, const double* w,
                     VarMode mode, double* partials, double* partials_max, cudaStream_t s) {
  const ZPlan p = plan_var(g, sizeof(T));
  if (int rc = check_launch_grid(p.tiles_x, p.tiles_y, p.chunks)) return rc;
  VarW<T, R> hw;
  for (int d = 0; d <= R; d++) hw.w[d] = (T)(0.5 * w[d]);  // exact: halving
  dim3 grid(p.tiles_x, p.tiles_y, p.chunks), block(32, VC_WARPS);
  const int nx = (int)g.nx, ny = (int)g.ny, nz = (int)g.nz, NX = (int)g.NX(), NY = (int)g.NY();
#define STN_VARC_LAUNCH(M)                                                                       \
  var_col_kernel<T, R, M, TJ><<<grid, block, 0, s>>>(u, a, f, out, nx, ny, nz, NX, NY, p.kchunk, \
                                                     hw, partials, partials_max)
  switch (mode) {
    case kVarSweep: STN_VARC_LAUNCH(kVarSweep); break;
    case kVarApply: STN_VARC_LAUNCH(kVarApply); break;
    case kVarResidual: STN_VARC_LAUNCH(kVarResidual); break;
    default: STN_VARC_LAUNCH(kVarRefine); break;
  }
#undef STN_VARC_LAUNCH
  STN_CUDA_TRY(cudaGetLastError());
  return STN_OK;
}

template <typename T, int R>
int launch_var_t(const T* u, const T* a, const T* f, T* out, const Grid& g, const double* w,
                 VarMode mode, double* partials, double* partials_max, cudaStream_t s) {
  const ZPlan p = plan_star(g, kStarScalar, 8);
  if (int rc = check_launch_grid(p.tiles_x, p.tiles_y, p.chunks)) return rc;
  VarW<T, R> wt;
  for (int d = 0; d <= R; d++) wt.w[d] = (T)w[d];
  dim3 grid(p.tiles_x, p.tiles_y, p.chunks), block(TX, TY);
  const int nx = (int)g.nx, ny = (int)g.ny, nz = (int)g.nz, NX = (int)g.NX(), NY = (int)g.NY();
#define STN_VAR_LAUNCH(M) \
  var_kernel<T, R, M><<<grid, block, 0, s>>>(u, a, f, out, nx, ny, nz, NX, NY, p.kchunk, wt, partials, partials_max)
  switch (mode) {
    case kVarSweep: STN_VAR_LAUNCH(kVarSweep); break;
    case kVarApply: STN_VAR_LAUNCH(kVarApply); break;
    case kVarResidual: STN_VAR_LAUNCH(kVarResidual); break;
    default: STN_VAR_LAUNCH(kVarRefine); break;
  }
#undef STN_VAR_LAUNCH
  STN_CUDA_TRY(cudaGetLastError());
  return STN_OK;
}

}  // namespace

// -1 automatic (TMA-staged for aligned radius-2 float sweeps, else column),
// 0 plane, 1 column, 2 TMA-staged where it applies (column elsewhere)
static std::atomic<int> g_var_variant{-1};

int tune_set_var_variant(int v) {
  if (v < -1 || v > 2) return STN_EINVAL;
  g_var_variant = v;
  return STN_OK;
}
int tune_get_var_variant() { return g_var_variant; }

static std::atomic<int> g_var_chunks{0};  // k chunks of the TMA-staged sweep (0 = planned)
int tune_set_var_chunks(int v) {
  if (v < 0 || v > 65535) return STN_EINVAL;
  g_var_chunks = v;
  return STN_OK;
}
int tune_get_var_chunks() { return g_var_chunks.load(); }

static bool var_use_column(const Grid& g, size_t esize) {
  // 32-bit row offsets: TJ + 2R rows of NX elements
  const int tj = esize == 4 ? VarColTJ<float>::value : VarColTJ<double>::value;
  if ((i64)(tj + 2 * g.r) * g.NX() >= ((i64)1 << 31)) return false;
  return g_var_variant.load() != 0;
}

// The TMA-staged kernel takes float sweeps of radius 2 on grids whose rows
// are a multiple of 16 bytes, unless a knob asks for the plane or column
// kernel.
// Automatically only on grids with at least four waves of its 64 x 16-column,
// 16-plane blocks: on fewer (96 x 96 x 48: 36 blocks) the column kernel's
// finer grid is faster.
static bool var_use_tma(const Grid& g, size_t esize, const void* u, const void* a, const void* f,
                        const void* out) {
  const int v = g_var_variant.load();
  if (v != -1 && v != 2) return false;
  if (!var_tma_applicable(g, esize, u, a, f, out)) return false;
  if (v == 2) return true;
  const i64 blocks = ((g.nx + 63) / 64) * ((g.ny + 15) / 16) * ((g.nz + 15) / 16);
  return blocks >= 4 * 2 * (i64)device_sms();
}

ZPlan plan_var(const Grid& g, size_t esize) {
  if (!var_use_column(g, esize)) return plan_star(g, kStarScalar, 8);
  ZPlan p;
  const int tj = esize == 4 ? VarColTJ<float>::value : VarColTJ<double>::value;
  p.tiles_x = (int)((g.nx + (32 - 2 * g.r) - 1) / (32 - 2 * g.r));
  p.tiles_y = (int)((g.ny + VC_WARPS * tj - 1) / (VC_WARPS * tj));
  const i64 tiles = (i64)p.tiles_x * p.tiles_y;
  // enough blocks for every SM several times over; chunks of >= 8 planes,
  // at most 32768 blocks
  i64 chunks = (152 * 8 + tiles - 1) / tiles;
  const i64 c16 = (g.nz + 15) / 16;
  if (c16 > chunks) chunks = c16;
  const i64 cap = 32768 / (tiles > 0 ? tiles : 1);
  if (chunks > cap) chunks = cap;
  const i64 max_chunks = (g.nz + 7) / 8;
  if (chunks > max_chunks) chunks = max_chunks;
  if (chunks < 1) chunks = 1;
  p.kchunk = (int)((g.nz + chunks - 1) / chunks);
  p.chunks = (int)((g.nz + p.kchunk - 1) / p.kchunk);
  return p;
}

LaunchPlan var_launch_plan(const Grid& g, size_t esize) {
  LaunchPlan q;
  if (var_use_tma(g, esize, nullptr, nullptr, nullptr, nullptr)) {
    const ZPlan p = plan_var_tma(g);
    q.variant = 2;
    q.grid_x = p.tiles_x;
    q.grid_y = p.tiles_y;
    q.grid_z = p.chunks;
    q.kchunk = p.kchunk;
    q.block_threads = 288;  // 8 consumer warps and the producer warp
    q.tile_w = 64;
    q.tile_h = p.rg;
    q.smem = p.smem;
    return q;
  }
  const ZPlan p = plan_var(g, esize);
  q.grid_x = p.tiles_x;
  q.grid_y = p.tiles_y;
  q.grid_z = p.chunks;
  q.kchunk = p.kchunk;
  if (var_use_column(g, esize)) {
    const int tj = esize == 4 ? VarColTJ<float>::value : VarColTJ<double>::value;
    q.variant = 1;
    q.block_threads = 32 * VC_WARPS;
    q.tile_w = 32 - 2 * g.r;
    q.tile_h = VC_WARPS * tj;
  } else {
    q.variant = 0;
    q.block_threads = TX * TY;
    q.tile_w = TX;
    q.tile_h = TY;
  }
  return q;
}

template <typename T>
int launch_var(const T* u, const T* a, const T* f, T* out, const Grid& g, const double* w,
               VarMode mode, double* partials, double* partials_max, cudaStream_t s) {
  constexpr int TJ = VarColTJ<T>::value;
  if constexpr (sizeof(T) == 4) {
    if (mode == kVarSweep && var_use_tma(g, sizeof(T), u, a, f, out))
      return launch_var_tma(u, a, f, out, g, w, s);
  }
  if (var_use_column(g, sizeof(T))) {
    if (g.r == 1) return launch_var_col_t<T, 1, TJ>(u, a, f, out, g, w, mode, partials, partials_max, s);
    return launch_var_col_t<T, 2, TJ>(u, a, f, out, g, w, mode, partials, partials_max, s);
  }
  if (g.r == 1) return launch_var_t<T, 1>(u, a, f, out, g, w, mode, partials, partials_max, s);
  return launch_var_t<T, 2>(u, a, f, out, g, w, mode, partials, partials_max, s);
}

template int launch_var<double>(const double*, const double*, const double*, double*, const Grid&,
                                const double*, VarMode, double*, double*, cudaStream_t);
template int launch_var<float>(const float*, const float*, const float*, float*, const Grid&,
                               const double*, VarMode, double*, double*, cudaStream_t);

}  // namespace stn
