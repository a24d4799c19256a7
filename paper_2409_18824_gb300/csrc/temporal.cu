// Temporally blocked star-stencil sweeps: TL Jacobi sweeps per pass over HBM.
//
// The paper's benchmark repeats the Jacobi sweep a fixed number of times
// (arXiv 2409.18824 Sec. 4); this kernel fuses TL consecutive sweeps so that
// each grid value is read from and written to HBM once per TL sweeps instead
// of once per sweep.  The result is bitwise the result of TL separate sweeps:
// every level is computed with the canonical operation order of star.cuh,
// and Dirichlet-halo cells keep their value at every level.
//
// Scheme (overlapped tiling in i/j, wavefront in k):
//   * a block owns an output tile of TWO x THO interior columns and a chunk of
//     k planes.  Level t (t = 0 input, t = TL output) is needed on the tile
//     grown by R*(TL-t) on each side, so level t is W_t x H_t with
//     W_t = TWO + 2R(TL-t), H_t = THO + 2R(TL-t).
//   * for each level t < TL a ring of 2R+1 planes of W_t x H_t values lives in
//     shared memory.  Step p loads input plane p into ring 0 (its loads were
//     issued during the previous step), then computes level t plane p - tR for
//     t = 1..TL from ring t-1; level TL goes straight to global memory.
//   * every neighbour offset inside a level plane is a compile-time constant
//     (+-d, +-d*W_{t-1}); each thread's cell offsets are computed once.
// Cells outside the global array are never read by a cell that matters (a
// cell's inputs lie within distance R, and the halo is R wide), so they are
// left unwritten.
#include "arith.cuh"
#include "internal.h"

namespace stn {

namespace {

constexpr int TB_THREADS = 256;

template <int R, int TL, int TWO, int THO>
struct TBGeom {
  static constexpr int W(int t) { return TWO + 2 * R * (TL - t); }
  static constexpr int H(int t) { return THO + 2 * R * (TL - t); }
  static constexpr int A(int t) { return W(t) * H(t); }
  static constexpr int NS(int t) { return (A(t) + TB_THREADS - 1) / TB_THREADS; }
  static constexpr int RING = 2 * R + 1;
  // offset (elements) of level t's ring in shared memory
  static constexpr int OFF(int t) { return t == 0 ? 0 : OFF(t - 1) + RING * A(t - 1); }
  static constexpr int SMEM_ELEMS = OFF(TL);
};

template <typename T, int R>
struct TBCoeffs {
  T c[R + 1];
};

// Computes level t (1 <= t <= TL) plane q of the block.  `src` is level t-1's
// plane q in shared memory, `srcm/srcp` its planes q-d / q+d (d = 1..R, given
// as plane pointers), `dst` level t's plane (shared) or nullptr for the last
// level, which goes to global `out` at plane offset `og`.
template <typename T, int R, int TL, int TWO, int THO, int t, bool HAS_C0>
__device__ __forceinline__ void tb_level(const T* const* ring_prev, T* dst, T* __restrict__ out,
                                         i64 og, bool halo_plane, int ox, int oy, int gx0,
                                         int gy0, int nx, int ny, int NX, const TBCoeffs<T, R>& cf) {
  using G = TBGeom<R, TL, TWO, THO>;
  using A = Arith<T>;
  constexpr int Wp = G::W(t - 1);
  constexpr int Wt = G::W(t);
  constexpr int At = G::A(t);
  const T* cen = ring_prev[R];  // plane q of level t-1
#pragma unroll
  for (int m = 0; m < G::NS(t); m++) {
    const int c = threadIdx.x + TB_THREADS * m;
    if (At % TB_THREADS != 0 && c >= At) break;
    const int y = c / Wt, x = c - y * Wt;
    // global padded coordinates of this cell
    const int gx = gx0 - R * (TL - t) + x, gy = gy0 - R * (TL - t) + y;
    const int sp = (y + R) * Wp + (x + R);  // same cell in level t-1 coordinates
    const T u0 = cen[sp];
    T v;
    const bool interior = !halo_plane && gx >= R && gx < nx + R && gy >= R && gy < ny + R;
    if (interior) {
      T acc = T(0);
#pragma unroll
      for (int d = R; d >= 1; d--) {
        const T sx = A::add(cen[sp - d], cen[sp + d]);
        const T sy = A::add(cen[sp - d * Wp], cen[sp + d * Wp]);
        const T sz = A::add(ring_prev[R - d][sp], ring_prev[R + d][sp]);
        const T s = A::add(A::add(sx, sy), sz);
        const T tt = A::mul(cf.c[d], s);
        acc = (d == R) ? tt : A::add(acc, tt);
      }
      if (HAS_C0) acc = A::add(acc, A::mul(cf.c[0], u0));
      v = acc;
    } else {
      v = u0;  // Dirichlet halo: constant through every level
    }
    if (t < TL) {
      dst[c] = v;
    } else if (interior) {
      out[og + gx + (i64)gy * NX] = v;
    }
  }
}

template <typename T, int R, int TL, int TWO, int THO, int t, bool HAS_C0>
struct TBLevels {
  // runs level t for step p, then the higher levels
  static __device__ __forceinline__ void run(T* sm, T* __restrict__ out, int p, int k0, int k1,
                                             int NZ, int nz, int nx, int ny, int NX, i64 sz,
                                             int gx0, int gy0, const TBCoeffs<T, R>& cf) {
    using G = TBGeom<R, TL, TWO, THO>;
    const int q = p - t * R;
    const int lo = max(k0 - (TL - t) * R, 0), hi = min(k1 + (TL - t) * R, NZ);
    if (q >= lo && q < hi) {
      const T* planes[2 * R + 1];
#pragma unroll
      for (int d = -R; d <= R; d++) {
        const int qq = q + d;
        const int slot = ((qq % G::RING) + G::RING) % G::RING;
        planes[d + R] = sm + G::OFF(t - 1) + slot * G::A(t - 1);
      }
      const bool halo_plane = q < R || q >= nz + R;
      T* dst = nullptr;
      if constexpr (t < TL) dst = sm + G::OFF(t) + (q % G::RING) * G::A(t);
      tb_level<T, R, TL, TWO, THO, t, HAS_C0>(planes, dst, out, (i64)q * sz, halo_plane, 0, 0, gx0,
                                             gy0, nx, ny, NX, cf);
    }
    if constexpr (t < TL) {
      __syncthreads();
      TBLevels<T, R, TL, TWO, THO, t + 1, HAS_C0>::run(sm, out, p, k0, k1, NZ, nz, nx, ny, NX, sz,
                                                      gx0, gy0, cf);
    }
  }
};

template <typename T, int R, int TL, int TWO, int THO, bool HAS_C0>
__global__ void __launch_bounds__(TB_THREADS)
    tb_kernel(const T* __restrict__ u, T* __restrict__ out, int nx, int ny, int nz, int NX, int NY,
              int kchunk, TBCoeffs<T, R> cf) {
  using G = TBGeom<R, TL, TWO, THO>;
  extern __shared__ __align__(16) unsigned char tb_smem_raw[];
  T* sm = reinterpret_cast<T*>(tb_smem_raw);
  const int NZ = nz + 2 * R;
  const i64 sz = (i64)NX * NY;
  const int gx0 = R + blockIdx.x * TWO;  // padded coordinates of the output tile origin
  const int gy0 = R + blockIdx.y * THO;
  const int k0 = R + blockIdx.z * kchunk;
  const int k1 = min(k0 + kchunk, nz + R);
  const int p0 = max(k0 - TL * R, 0);
  const int pend = min(k1 + TL * R, NZ);  // input planes [p0, pend)
  const int plast = k1 - 1 + TL * R;      // last step (computes level TL plane k1-1)

  // this thread's input cells of the level-0 region: in-plane global offsets
  constexpr int NS0 = G::NS(0);
  constexpr int A0 = G::A(0);
  constexpr int W0 = G::W(0);
  int goff[NS0];
  bool gok[NS0];
#pragma unroll
  for (int m = 0; m < NS0; m++) {
    const int c = threadIdx.x + TB_THREADS * m;
    const int y = c / W0, x = c - y * W0;
    const int gx = gx0 - R * TL + x, gy = gy0 - R * TL + y;
    gok[m] = c < A0 && gx >= 0 && gx < NX && gy >= 0 && gy < NY;
    goff[m] = gok[m] ? gx + gy * NX : 0;
  }
  T nxt[NS0];
  auto load = [&](int p) {
    const T* pl = u + (i64)p * sz;
#pragma unroll
    for (int m = 0; m < NS0; m++) nxt[m] = gok[m] ? pl[goff[m]] : T(0);
  };
  if (p0 < pend) load(p0);
  for (int p = p0; p <= plast; p++) {
    if (p < pend) {
      T* r0 = sm + G::OFF(0) + (p % G::RING) * A0;
#pragma unroll
      for (int m = 0; m < NS0; m++) {
        const int c = threadIdx.x + TB_THREADS * m;
        if (A0 % TB_THREADS == 0 || c < A0) r0[c] = nxt[m];
      }
      if (p + 1 < pend) load(p + 1);
    }
    __syncthreads();
    TBLevels<T, R, TL, TWO, THO, 1, HAS_C0>::run(sm, out, p, k0, k1, NZ, nz, nx, ny, NX, sz, gx0, gy0,
                                                 cf);
  }
}

constexpr int TB_TWO = 62;
constexpr int TB_THO = 16;

template <typename T, int R, int TL, bool HAS_C0>
int launch_tb_t(const T* u, T* out, const Grid& g, const double* coeffs, cudaStream_t s) {
  using G = TBGeom<R, TL, TB_TWO, TB_THO>;
  TBCoeffs<T, R> cf;
  for (int d = 0; d <= R; d++) cf.c[d] = (T)coeffs[d];
  const size_t smem = (size_t)G::SMEM_ELEMS * sizeof(T);
  auto kern = tb_kernel<T, R, TL, TB_TWO, TB_THO, HAS_C0>;
  STN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int resident = 0;
  STN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, kern, TB_THREADS, smem));
  if (resident < 1) {
    set_error("temporal-blocking kernel does not fit on an SM");
    return STN_ECUDA;
  }
  const ZPlan p = plan_temporal(g, TL, resident);
  if (int rc = check_launch_grid(p.tiles_x, p.tiles_y, p.chunks)) return rc;
  kern<<<dim3(p.tiles_x, p.tiles_y, p.chunks), TB_THREADS, smem, s>>>(
      u, out, (int)g.nx, (int)g.ny, (int)g.nz, (int)g.NX(), (int)g.NY(), p.kchunk, cf);
  STN_CUDA_TRY(cudaGetLastError());
  return STN_OK;
}

template <typename T, int R, bool HAS_C0>
int launch_tb_r(const T* u, T* out, const Grid& g, const double* coeffs, int depth, cudaStream_t s) {
  switch (depth) {
    case 2: return launch_tb_t<T, R, 2, HAS_C0>(u, out, g, coeffs, s);
    case 3: return launch_tb_t<T, R, 3, HAS_C0>(u, out, g, coeffs, s);
    default:
      if constexpr (sizeof(T) == 8 && R == 2) return launch_tb_t<T, R, 3, HAS_C0>(u, out, g, coeffs, s);
      else return launch_tb_t<T, R, 4, HAS_C0>(u, out, g, coeffs, s);
  }
}

}  // namespace

int temporal_depth_supported(int depth, size_t esize, int radius) {
  if (depth < 2) return 1;
  if (depth > 4) depth = 4;
  if (esize == 8 && radius == 2 && depth > 3) depth = 3;
  return depth;
}

ZPlan plan_temporal(const Grid& g, int depth, int resident) {
  ZPlan p;
  p.tiles_x = (int)((g.nx + TB_TWO - 1) / TB_TWO);
  p.tiles_y = (int)((g.ny + TB_THO - 1) / TB_THO);
  const i64 tiles = (i64)p.tiles_x * p.tiles_y;
  // one full wave of resident blocks
  const i64 want = 152 * (i64)resident;
  i64 chunks = (want + tiles - 1) / tiles;
  // keep chunks long against the TL*R planes of warm-up each one re-reads
  const i64 min_len = 16 * depth;
  i64 max_chunks = g.nz / min_len;
  if (max_chunks < 1) max_chunks = 1;
  if (chunks > max_chunks) chunks = max_chunks;
  if (chunks < 1) chunks = 1;
  p.kchunk = (int)((g.nz + chunks - 1) / chunks);
  p.chunks = (int)((g.nz + p.kchunk - 1) / p.kchunk);
  return p;
}

template <typename T>
int launch_temporal(const T* u, T* out, const Grid& g, const double* coeffs, int depth,
                    cudaStream_t s) {
  const bool hc0 = coeffs[0] != 0.0;
  if (g.r == 1)
    return hc0 ? launch_tb_r<T, 1, true>(u, out, g, coeffs, depth, s)
               : launch_tb_r<T, 1, false>(u, out, g, coeffs, depth, s);
  return hc0 ? launch_tb_r<T, 2, true>(u, out, g, coeffs, depth, s)
             : launch_tb_r<T, 2, false>(u, out, g, coeffs, depth, s);
}

template int launch_temporal<double>(const double*, double*, const Grid&, const double*, int,
                                     cudaStream_t);
template int launch_temporal<float>(const float*, float*, const Grid&, const double*, int,
                                    cudaStream_t);

}  // namespace stn
