// Multi-field advection: a synthetic stand-in for the paper's pw-advection
// and tra-adv workloads (arXiv 2409.18824 Sec. 4: fields carried by a wind on
// 2048 x 1024 x 1024 and 1024 x 512 x 512 grids; the paper gives no
// formulas).  Second-order centred flux-form advection of a field q by the
// velocity (u, v, w) on a halo-1 grid; per axis a with velocity V,
//     F-(p) = (V(p-e)+V(p)) * (q(p-e)+q(p)),  F+(p) = (V(p)+V(p+e)) * (q(p)+q(p+e)),
//     T_a = c_a * (F- - F+),                   s = (T_x + T_y) + T_z,
// each operation rounded separately in this order (bitwise the CPU oracle).
//
// A face flux is the same number seen from either side, so it is computed
// once: lane l's F-x is lane l-1's F+x (one shuffle), a thread's F-y is the
// F+y of its row above, and F-z is the F+z the thread computed one plane
// earlier.  Layout as the star column kernel: a warp covers 32 consecutive
// padded columns (the 30 middle lanes produce output), a thread owns TJ rows
// (plus the rows above and below for the j faces), and planes stream in k
// through a three-plane register ring (planes k and k+1 in use, k+2 loading),
// unrolled by three so the ring rotates by renaming.
//
// Self mode (pw-like): the velocity components advect themselves, q_m = the
// m-th velocity component, so only u, v, w are read.
#include "arith.cuh"
#include "internal.h"

namespace stn {

namespace {

constexpr int ADV_WARPS = 4;

template <typename T>
struct AdvPtrs {
  const T* q[3];
  T* s[3];
};

template <typename T>
struct AdvTJ {
  static constexpr int value = sizeof(T) == 4 ? 4 : 2;
};

template <typename T, int NQ, bool SELF, int TJ>
__global__ void __launch_bounds__(32 * ADV_WARPS)
    advect_kernel(const T* __restrict__ u, const T* __restrict__ v, const T* __restrict__ w,
                  AdvPtrs<T> io, int nx, int ny, int nz, int NX, int NY, int kchunk, T cx, T cy, T cz) {
  using A = Arith<T>;
  constexpr int NF = SELF ? 3 : 3 + NQ;  // distinct fields read
  constexpr int NR = TJ + 2;             // rows: above, TJ own, below
  const int lane = threadIdx.x, wp = threadIdx.y;
  const int gi = (int)blockIdx.x * 30 + lane;  // padded column (lane 1 <-> first interior column)
  const int j0 = 1 + ((int)blockIdx.y * ADV_WARPS + wp) * TJ;
  const i64 sz = (i64)NX * NY;
  const int k0 = 1 + (int)blockIdx.z * kchunk;
  const int k1 = min(k0 + kchunk, nz + 1);
  const bool col_ok = gi < NX;
  const bool lane_c = lane >= 1 && lane <= 30 && gi <= nx;
  unsigned roff[NR];
  bool rok[NR];
#pragma unroll
  for (int r = 0; r < NR; r++) {
    rok[r] = col_ok && j0 - 1 + r < NY;
    roff[r] = (unsigned)r * (unsigned)NX;
  }
  bool act[TJ];
#pragma unroll
  for (int t = 0; t < TJ; t++) act[t] = lane_c && j0 + t <= ny;
  const i64 base = gi + (i64)(j0 - 1) * NX;
  const T* fld[NF];
  fld[0] = u;
  fld[1] = v;
  fld[2] = w;
  if (!SELF) {
#pragma unroll
    for (int m = 0; m < NQ; m++) fld[3 + m] = io.q[m];
  }
  constexpr int QF0 = SELF ? 0 : 3;  // field index of q_0

  T P[3][NF][NR];  // plane ring: slot, field, row
  auto load = [&](int slot, int kk) {
    const i64 po = base + (i64)kk * sz;
#pragma unroll
    for (int f = 0; f < NF; f++)
#pragma unroll
      for (int r = 0; r < NR; r++) P[slot][f][r] = rok[r] ? fld[f][po + roff[r]] : T(0);
  };
  // F-z of plane k0: F+z of plane k0-1
  T fzm[NQ][TJ];
  {
    load(0, k0 - 1);
    load(1, k0);
#pragma unroll
    for (int m = 0; m < NQ; m++)
#pragma unroll
      for (int t = 0; t < TJ; t++)
        fzm[m][t] = A::mul(A::add(P[0][2][t + 1], P[1][2][t + 1]),
                           A::add(P[0][QF0 + m][t + 1], P[1][QF0 + m][t + 1]));
  }
  // ring: plane k in slot (J+1)%3, k+1 in (J+2)%3, k+2 loads into J%3
  if (k0 < k1) load(2, k0 + 1);

  for (int kb = k0; kb < k1; kb += 3) {
#pragma unroll
    for (int J = 0; J < 3; J++) {
      const int k = kb + J;
      if (k >= k1) break;
      const int sc = (J + 1) % 3, sn = (J + 2) % 3;
      if (k + 2 <= k1) load(J % 3, k + 2);
      const i64 po = base + (i64)k * sz;
#pragma unroll
      for (int m = 0; m < NQ; m++) {
        const T* Q = P[sc][QF0 + m];
        // j faces: F+y of rows -1 .. TJ-1 (row r and r+1), at [r + 1]
        T fy[TJ + 1];
#pragma unroll
        for (int r = 0; r <= TJ; r++)
          fy[r] = A::mul(A::add(P[sc][1][r], P[sc][1][r + 1]), A::add(Q[r], Q[r + 1]));
#pragma unroll
        for (int t = 0; t < TJ; t++) {
          const T uc = P[sc][0][t + 1], qc = Q[t + 1];
          const T fxp = A::mul(A::add(uc, __shfl_down_sync(0xffffffffu, uc, 1)),
                               A::add(qc, __shfl_down_sync(0xffffffffu, qc, 1)));
          const T fxm = __shfl_up_sync(0xffffffffu, fxp, 1);
          const T fzp = A::mul(A::add(P[sc][2][t + 1], P[sn][2][t + 1]), A::add(qc, P[sn][QF0 + m][t + 1]));
          const T tx = A::mul(cx, A::add(fxm, -fxp));
          const T ty = A::mul(cy, A::add(fy[t], -fy[t + 1]));
          const T tz = A::mul(cz, A::add(fzm[m][t], -fzp));
          fzm[m][t] = fzp;
          if (act[t]) io.s[m][po + roff[t + 1]] = A::add(A::add(tx, ty), tz);
        }
      }
    }
  }
}

template <typename T, int NQ, bool SELF>
int launch_advect_t(const T* u, const T* v, const T* w, const AdvPtrs<T>& io, const Grid& g,
                    const double* c, cudaStream_t s) {
  constexpr int TJ = AdvTJ<T>::value;
  const int tiles_x = (int)((g.nx + 29) / 30);
  const int tiles_y = (int)((g.ny + ADV_WARPS * TJ - 1) / (ADV_WARPS * TJ));
  // chunks of 64 planes: many blocks, each long enough to amortise its first planes
  const int kchunk = (int)std::min<i64>(g.nz, 64);
  const int chunks = (int)((g.nz + kchunk - 1) / kchunk);
  if (int rc = check_launch_grid(tiles_x, tiles_y, chunks)) return rc;
  advect_kernel<T, NQ, SELF, TJ><<<dim3(tiles_x, tiles_y, chunks), dim3(32, ADV_WARPS), 0, s>>>(
      u, v, w, io, (int)g.nx, (int)g.ny, (int)g.nz, (int)g.NX(), (int)g.NY(), kchunk, (T)c[0], (T)c[1],
      (T)c[2]);
  STN_CUDA_TRY(cudaGetLastError());
  return STN_OK;
}

}  // namespace

// q == nullptr: self mode (the tendencies of u, v, w into s[0..2]).  Otherwise
// nq in 1..3 fields per call.
template <typename T>
int launch_advect(const T* u, const T* v, const T* w, const T* const* q, int nq, T* const* s,
                  const Grid& g, const double* c, cudaStream_t st) {
  AdvPtrs<T> io = {};
  for (int m = 0; m < 3; m++) {
    io.q[m] = q && m < nq ? q[m] : nullptr;
    io.s[m] = m < (q ? nq : 3) ? s[m] : nullptr;
  }
  if (!q) return launch_advect_t<T, 3, true>(u, v, w, io, g, c, st);
  switch (nq) {
    case 1: return launch_advect_t<T, 1, false>(u, v, w, io, g, c, st);
    case 2: return launch_advect_t<T, 2, false>(u, v, w, io, g, c, st);
    default: return launch_advect_t<T, 3, false>(u, v, w, io, g, c, st);
  }
}

template int launch_advect<double>(const double*, const double*, const double*, const double* const*, int,
                                   double* const*, const Grid&, const double*, cudaStream_t);
template int launch_advect<float>(const float*, const float*, const float*, const float* const*, int,
                                  float* const*, const Grid&, const double*, cudaStream_t);

}  // namespace stn
