// Two-dimensional star-stencil Jacobi sweeps: the paper's own jacobi
// benchmark (arXiv 2409.18824 Sec. 4: a Jacobi iteration for Laplace's
// equation on one 1024 x 1024 grid, 100000 iterations), written with the
// 2-D form of the canonical operation order of star.cuh:
//     S_d = (u[i-d]+u[i+d]) + (u[j-d]+u[j+d]);  acc = c_r S_r;
//     acc = acc + c_d S_d (d = r-1..1);  + c0 u if c0 != 0;  + b if given.
//
// Two paths:
//  * resident.  A 1024^2 double grid is 8 MB, well inside the 152 SMs' 34 MB
//    of shared memory.  One cooperative launch runs one CTA per SM; CTA b owns
//    a band of rows and keeps two copies of it (the current and the next
//    iterate, each with R halo rows above and below) in shared memory for
//    every sweep of the launch, so HBM is read and written once per launch.
//    Per sweep a CTA computes its inner rows (which need no neighbour data)
//    while the neighbours' boundary rows of the previous sweep travel through
//    L2 -- each warp waits for the neighbours' counters (acquire poll,
//    bounded) half way through and loads its columns of those rows into
//    registers -- then computes its R top and R bottom rows, storing them
//    both to shared memory and to a global exchange slot, and publishes its
//    counter (release store).  Two barriers per sweep.
//  * per-sweep.  For grids that do not fit: a grid-stride kernel, one point
//    per thread, ping-ponging through HBM; it also computes the residual.
#include "arith.cuh"
#include "star.cuh"

namespace stn {

namespace {

template <typename T, int R>
struct Co2 {
  T c[R + 1];
};

// The canonical 2-D update of the point at `p` (row stride NX).
template <typename T, int R, bool HAS_C0>
__device__ __forceinline__ T point2d(const T* p, int NX, const Co2<T, R>& cf) {
  using A = Arith<T>;
  T acc = T(0);
#pragma unroll
  for (int d = R; d >= 1; d--) {
    const T sx = A::add(p[-d], p[d]);
    const T sy = A::add(p[-d * NX], p[d * NX]);
    const T t = A::mul(cf.c[d], A::add(sx, sy));
    acc = (d == R) ? t : A::add(acc, t);
  }
  if (HAS_C0) acc = A::add(acc, A::mul(cf.c[0], p[0]));
  return acc;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_i32(const int* p) { return *(const volatile int*)p; }

// Waits until *flag >= target.  Gives up when *status is set by another CTA,
// or after `limit` clock cycles, in which case it sets *status = 1.
__device__ bool wait_flag(const unsigned long long* flag, unsigned long long target, int* status,
                          long long limit) {
  const long long t0 = clock64();
  for (;;) {
    if (ld_acquire_u64(flag) >= target) return true;
    if (ld_volatile_i32(status) != 0) return false;
    if (clock64() - t0 > limit) {
      atomicExch(status, 1);
      return false;
    }
    __nanosleep(32);
  }
}

// ---- shared-memory band layout ----
// A band buffer holds rows of the padded grid with row stride NS elements;
// padded column c of buffer row L is at L*NS + P + c.  P and NS are chosen so
// that every row's interior (column R) starts on a 16-byte boundary, which
// lets the halo rows arrive by bulk copy.

// Buffer rows [L0, L1), interior columns: nxt = S(cur).  Narrow rows: the
// threads walk the rows x columns rectangle in row-major order without
// division, so that no thread idles.
template <typename T, int R, bool HAS_C0>
__device__ __forceinline__ void band_rows(const T* cur, T* nxt, int NS, int P, int nx, int L0, int L1,
                                          const Co2<T, R>& cf) {
  if (L1 <= L0) return;
  if (nx >= (int)blockDim.x) {  // rows at least a block wide: plain row loop
#pragma unroll 2
    for (int l = L0; l < L1; l++)
      for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const int o = l * NS + P + R + i;
        nxt[o] = point2d<T, R, HAS_C0>(cur + o, NS, cf);
      }
    return;
  }
  int l = L0 + (int)threadIdx.x / nx;
  int i = (int)threadIdx.x % nx;
  while (l < L1) {
    const int o = l * NS + P + R + i;
    nxt[o] = point2d<T, R, HAS_C0>(cur + o, NS, cf);
    i += blockDim.x;
    while (i >= nx) {
      i -= nx;
      l++;
    }
  }
}

// Boundary rows [L0, L1) of the next iterate, as band_rows, each value also
// stored to this band's exchange slots: own rows [0, R) to `xtop`, own rows
// [nb - R, nb) to `xbot` (either may be NULL).
template <typename T, int R, bool HAS_C0>
__device__ __forceinline__ void edge_rows(const T* cur, T* nxt, int NS, int P, int nx, int L0, int L1,
                                          int nb, T* xtop, T* xbot, const Co2<T, R>& cf) {
  if (L1 <= L0) return;
  int l = L0 + (int)threadIdx.x / nx;
  int i = (int)threadIdx.x % nx;
  while (l < L1) {
    const int o = l * NS + P + R + i;
    const T v = point2d<T, R, HAS_C0>(cur + o, NS, cf);
    nxt[o] = v;
    const int own = l - R;
    if (xtop && own < R) xtop[own * nx + i] = v;
    if (xbot && own >= nb - R) xbot[(own - (nb - R)) * nx + i] = v;
    i += blockDim.x;
    while (i >= nx) {
      i -= nx;
      l++;
    }
  }
}

// ---- mbarrier and bulk-copy helpers (inline PTX) ----
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* m, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* m, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* m, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(m)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait for the completion of the mbarrier phase of parity `parity`.
__device__ __forceinline__ bool mbar_wait(unsigned long long* m, unsigned parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(m, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* m) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(m))
      : "memory");
}

// Most interior columns one thread covers in a band row when the halo rows
// arrive through registers: that path requires nx <= kJ2Cols * blockDim.x.
constexpr int kJ2Cols = 4;

// One sweep of a band (iterate s in `cur` -> iterate s+1 in `nxt`):
//   1. first half of the inner rows (they read only the band's own rows);
//   2. the neighbours' boundary rows of iterate s (exchange slots of parity
//      s-1, counter s) are fetched: with TMA, thread 0 alone waits for the
//      counters and issues bulk copies into cur's halo rows, completing on an
//      mbarrier, so only its warp pauses; without (rows not a multiple of 16
//      bytes), every warp waits and loads its columns into registers;
//   3. second half of the inner rows while the rows travel;
//   4. barrier; the halo rows are in place (mbarrier wait, or register
//      stores before the barrier);
//   5. boundary rows of iterate s+1, written to nxt and to this band's
//      exchange slots of parity s; barrier; thread 0 publishes counter s+1.
// A band rewrites a slot of parity s only in sweep s+2, after both
// neighbours have published s+1 -- which they do after reading the slot.
template <typename T, int R, bool HAS_C0, bool TMA>
__global__ void __launch_bounds__(1024, 1)
    j2d_resident_kernel(const T* src, T* dst, int nx, int ny, int NX, int NS, int P, int nbmax,
                        int sweeps, Co2<T, R> cf, T* __restrict__ xchg,
                        unsigned long long* __restrict__ flags, int* __restrict__ status,
                        long long spin_limit, int withhold_last) {
  extern __shared__ __align__(128) unsigned char j2_smem[];
  __shared__ __align__(8) unsigned long long s_mbar;
  __shared__ int s_abort;
  const int nblk = gridDim.x, b = blockIdx.x;
  const int jb = (int)(((long long)b * ny) / nblk);
  const int nb = (int)(((long long)(b + 1) * ny) / nblk) - jb;  // own rows (>= R unless nblk == 1)
  const int LR = nb + 2 * R;
  T* buf0 = reinterpret_cast<T*>(j2_smem);
  T* buf1 = buf0 + (size_t)(nbmax + 2 * R) * NS;
  if (threadIdx.x == 0) {
    s_abort = ld_volatile_i32(status);
    if (TMA) {
      mbar_init(&s_mbar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
  }
  __syncthreads();
  if (s_abort) return;  // an earlier launch of this call timed out

  // both copies <- padded rows [jb, jb + LR) of src, full width
  for (int L = 0; L < LR; L++)
    for (int c = threadIdx.x; c < NX; c += blockDim.x) {
      const T v = src[(size_t)(jb + L) * NX + c];
      buf0[L * NS + P + c] = v;
      buf1[L * NS + P + c] = v;
    }
  __syncthreads();

  const bool up = b > 0, down = b + 1 < nblk;
  const size_t slot = (size_t)R * nx;  // one side's rows in an exchange slot
  const bool publish = !(withhold_last && b == nblk - 1);
  const bool has_inner = nb > 2 * R;
  const int mid = has_inner ? 2 * R + (nb - 2 * R) / 2 : 2 * R;
  const int lane = threadIdx.x & 31;
  unsigned phase = 0;
  for (int s = 0; s < sweeps; s++) {
    T* cur = (s & 1) ? buf1 : buf0;
    T* nxt = (s & 1) ? buf0 : buf1;
    if (has_inner) band_rows<T, R, HAS_C0>(cur, nxt, NS, P, nx, 2 * R, mid, cf);
    const T* xp = xchg + (size_t)((s - 1) & 1) * nblk * 2 * slot;
    const T* from_up = up ? xp + (size_t)(2 * (b - 1) + 1) * slot : xp;  // band b-1's bottom rows
    const T* from_dn = down ? xp + (size_t)(2 * (b + 1)) * slot : xp;    // band b+1's top rows
    T hv[TMA ? 1 : 2 * R * kJ2Cols];
    bool ok = true;
    if (s > 0) {
      if (TMA) {
        if (threadIdx.x == 0) {
          if (up) ok = wait_flag(flags + b - 1, (unsigned long long)s, status, spin_limit);
          if (ok && down) ok = wait_flag(flags + b + 1, (unsigned long long)s, status, spin_limit);
          if (ok) {
            // the rows were written by other SMs' ordinary stores: order them
            // before this thread's bulk (async-proxy) reads, and this CTA's
            // earlier reads of the halo rows before the bulk writes
            asm volatile("fence.proxy.async.global;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const unsigned bytes = (unsigned)(nx * sizeof(T));
            mbar_arrive_expect_tx(&s_mbar, (unsigned)((up ? R : 0) + (down ? R : 0)) * bytes);
#pragma unroll
            for (int r = 0; r < R; r++) {
              if (up) bulk_g2s(cur + r * NS + P + R, from_up + (size_t)r * nx, bytes, &s_mbar);
              if (down) bulk_g2s(cur + (R + nb + r) * NS + P + R, from_dn + (size_t)r * nx, bytes, &s_mbar);
            }
          } else {
            mbar_arrive_expect_tx(&s_mbar, 0);  // completes the phase: nobody waits on it
            s_abort = 1;
          }
        }
      } else {
        if (lane == 0) {
          if (up) ok = wait_flag(flags + b - 1, (unsigned long long)s, status, spin_limit);
          if (ok && down) ok = wait_flag(flags + b + 1, (unsigned long long)s, status, spin_limit);
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        __syncwarp();
        if (ok) {
#pragma unroll
          for (int k = 0; k < kJ2Cols; k++) {
            const int i = (int)threadIdx.x + k * (int)blockDim.x;
#pragma unroll
            for (int r = 0; r < R; r++) {
              hv[r * kJ2Cols + k] = (up && i < nx) ? __ldcg(from_up + r * nx + i) : T(0);
              hv[(R + r) * kJ2Cols + k] = (down && i < nx) ? __ldcg(from_dn + r * nx + i) : T(0);
            }
          }
        } else {
          s_abort = 1;
        }
      }
    }
    if (has_inner) band_rows<T, R, HAS_C0>(cur, nxt, NS, P, nx, mid, nb, cf);
    if (!TMA && s > 0 && ok) {
#pragma unroll
      for (int k = 0; k < kJ2Cols; k++) {
        const int i = (int)threadIdx.x + k * (int)blockDim.x;
        if (i < nx) {
#pragma unroll
          for (int r = 0; r < R; r++) {
            if (up) cur[r * NS + P + R + i] = hv[r * kJ2Cols + k];
            if (down) cur[(R + nb + r) * NS + P + R + i] = hv[(R + r) * kJ2Cols + k];
          }
        }
      }
    }
    __syncthreads();
    if (s_abort) return;
    if (TMA && s > 0) {
      const bool arrived = mbar_wait(&s_mbar, phase & 1, spin_limit) ||
                           mbar_wait(&s_mbar, phase & 1, spin_limit);  // once more before leaving
      phase++;
      if (!arrived) {
        atomicExch(status, 1);
        return;
      }
    }
    T* xs = xchg + (size_t)(s & 1) * nblk * 2 * slot;
    T* xtop = up ? xs + (size_t)(2 * b) * slot : nullptr;
    T* xbot = down ? xs + (size_t)(2 * b + 1) * slot : nullptr;
    if (has_inner) {
      edge_rows<T, R, HAS_C0>(cur, nxt, NS, P, nx, R, 2 * R, nb, xtop, xbot, cf);
      edge_rows<T, R, HAS_C0>(cur, nxt, NS, P, nx, nb, nb + R, nb, xtop, xbot, cf);
    } else {
      edge_rows<T, R, HAS_C0>(cur, nxt, NS, P, nx, R, R + nb, nb, xtop, xbot, cf);
    }
    __syncthreads();
    if (threadIdx.x == 0 && publish && (up || down)) {
      __threadfence();
      st_release_u64(flags + b, (unsigned long long)(s + 1));
    }
  }
  // The neighbours read this band's rows of src at their start; in place
  // (src == dst) they must be past it before the rows are overwritten: wait
  // for their last counter.
  if (up || down) {
    if (threadIdx.x == 0) {
      bool ok = true;
      if (up) ok = wait_flag(flags + b - 1, (unsigned long long)sweeps, status, spin_limit);
      if (ok && down) ok = wait_flag(flags + b + 1, (unsigned long long)sweeps, status, spin_limit);
      s_abort = ok ? 0 : 1;
    }
    __syncthreads();
    if (s_abort) return;
  }
  // own rows (and the grid's top / bottom halo rows for the end bands) -> dst
  const T* fin = (sweeps & 1) ? buf1 : buf0;
  const int L0 = b == 0 ? 0 : R, L1 = down ? R + nb : LR;
  for (int L = L0; L < L1; L++)
    for (int c = threadIdx.x; c < NX; c += blockDim.x) dst[(size_t)(jb + L) * NX + c] = fin[L * NS + P + c];
}

// Per-sweep / residual kernel: 32 x 8 tiles, grid-stride over tiles; in
// residual modes one partial per block (fixed order: a block's tiles in
// sequence, then block_sum_fixed).
template <typename T, int R, bool HAS_B, bool HAS_C0, int MODE>
__global__ void __launch_bounds__(256)
    j2d_kernel(const T* u, const T* b, T* out, int nx, int ny, int NX, int tiles_x, i64 ntiles,
               Co2<T, R> cf, double* __restrict__ partials) {
  using A = Arith<T>;
  __shared__ double red[8];
  double rsum = 0.0;
  for (i64 t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const i64 ty = t / tiles_x;
    const int tx = (int)(t - ty * tiles_x);
    const int i = tx * 32 + (int)threadIdx.x + R;
    const i64 j = ty * 8 + threadIdx.y + R;
    if (i < nx + R && j < ny + R) {
      const i64 o = j * NX + i;
      T acc = point2d<T, R, HAS_C0>(u + o, NX, cf);
      if (HAS_B) acc = A::add(acc, b[o]);
      if (MODE != kResidualOnly) out[o] = acc;
      if (MODE != kSweep) {
        const double rho = (double)acc - (double)u[o];
        rsum = __fma_rn(rho, rho, rsum);
      }
    }
  }
  if (MODE != kSweep) {
    const double t = block_sum_fixed<256>(rsum, red);
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[blockIdx.x] = t;
  }
}

template <typename T, int R, bool HAS_B, bool HAS_C0>
int launch_j2d_t(const T* u, const T* b, T* out, const Grid2& g, const double* coeffs, SweepMode mode,
                 double* partials, cudaStream_t s) {
  Co2<T, R> cf;
  for (int d = 0; d <= R; d++) cf.c[d] = (T)coeffs[d];
  const int tiles_x = (int)((g.nx + 31) / 32);
  const i64 ntiles = (i64)tiles_x * ((g.ny + 7) / 8);
  const unsigned blocks = (unsigned)(ntiles < kJ2dBlocks ? ntiles : kJ2dBlocks);
  const int nx = (int)g.nx, ny = (int)g.ny, NX = (int)g.NX();
  const dim3 blk(32, 8);
  switch (mode) {
    case kSweep:
      j2d_kernel<T, R, HAS_B, HAS_C0, kSweep><<<blocks, blk, 0, s>>>(u, b, out, nx, ny, NX, tiles_x, ntiles, cf, partials);
      break;
    case kSweepResidual:
      j2d_kernel<T, R, HAS_B, HAS_C0, kSweepResidual><<<blocks, blk, 0, s>>>(u, b, out, nx, ny, NX, tiles_x, ntiles, cf, partials);
      break;
    default:
      j2d_kernel<T, R, HAS_B, HAS_C0, kResidualOnly><<<blocks, blk, 0, s>>>(u, b, out, nx, ny, NX, tiles_x, ntiles, cf, partials);
      break;
  }
  STN_CUDA_TRY(cudaGetLastError());
  return STN_OK;
}

template <typename T, int R>
int launch_j2d_r(const T* u, const T* b, T* out, const Grid2& g, const double* coeffs, SweepMode mode,
                 double* partials, cudaStream_t s) {
  const bool hc0 = coeffs[0] != 0.0;
  if (b)
    return hc0 ? launch_j2d_t<T, R, true, true>(u, b, out, g, coeffs, mode, partials, s)
               : launch_j2d_t<T, R, true, false>(u, b, out, g, coeffs, mode, partials, s);
  return hc0 ? launch_j2d_t<T, R, false, true>(u, b, out, g, coeffs, mode, partials, s)
             : launch_j2d_t<T, R, false, false>(u, b, out, g, coeffs, mode, partials, s);
}

// ---- knobs ----
int g_resident2d = -1;          // -1 automatic, 0 never, 1 whenever it fits
i64 g_chunk2d = 32768;          // sweeps per resident launch
int g_withhold2d = 0;           // fault injection: last band never publishes
int g_tma2d = 1;                // halo rows by bulk copy when rows are 16-byte multiples
int g_ctas2d = 1;               // resident bands (CTAs) per SM
constexpr double kWait2dSeconds = 2.0;

template <typename T, int R, bool HAS_C0, bool TMA>
int launch_resident_t(const T* src, T* dst, const Grid2& g, const double* coeffs, const Plan2d& p,
                      int sweeps, unsigned char* scratch, cudaStream_t s) {
  Co2<T, R> cf;
  for (int d = 0; d <= R; d++) cf.c[d] = (T)coeffs[d];
  auto kern = j2d_resident_kernel<T, R, HAS_C0, TMA>;
  STN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
  unsigned long long* flags = reinterpret_cast<unsigned long long*>(scratch);
  int* status = reinterpret_cast<int*>(scratch + 8 * (size_t)p.nblk);
  T* xchg = reinterpret_cast<T*>(scratch + p.xchg_off);
  STN_CUDA_TRY(cudaMemsetAsync(flags, 0, 8 * (size_t)p.nblk, s));
  int nx = (int)g.nx, ny = (int)g.ny, NX = (int)g.NX(), NS = p.ns, P = p.pad, nbmax = p.nbmax;
  int withhold = g_withhold2d;
  long long limit = (long long)(kWait2dSeconds * 2.07e9);
  void* args[] = {(void*)&src, (void*)&dst, &nx,    &ny,    &NX,    &NS,     &P,     &nbmax,
                  &sweeps,     &cf,         &xchg,  &flags, &status, &limit, &withhold};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)kern, dim3(p.nblk), dim3(p.threads), args,
                                              p.smem, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchCooperativeKernel(j2d_resident_kernel)");
  return STN_OK;
}

template <typename T, int R, bool HAS_C0>
int launch_resident_c(const T* src, T* dst, const Grid2& g, const double* coeffs, const Plan2d& p,
                      int sweeps, unsigned char* scratch, cudaStream_t s) {
  return p.tma ? launch_resident_t<T, R, HAS_C0, true>(src, dst, g, coeffs, p, sweeps, scratch, s)
               : launch_resident_t<T, R, HAS_C0, false>(src, dst, g, coeffs, p, sweeps, scratch, s);
}

template <typename T>
int launch_resident(const T* src, T* dst, const Grid2& g, const double* coeffs, const Plan2d& p,
                    int sweeps, unsigned char* scratch, cudaStream_t s) {
  const bool hc0 = coeffs[0] != 0.0;
  if (g.r == 1)
    return hc0 ? launch_resident_c<T, 1, true>(src, dst, g, coeffs, p, sweeps, scratch, s)
               : launch_resident_c<T, 1, false>(src, dst, g, coeffs, p, sweeps, scratch, s);
  return hc0 ? launch_resident_c<T, 2, true>(src, dst, g, coeffs, p, sweeps, scratch, s)
             : launch_resident_c<T, 2, false>(src, dst, g, coeffs, p, sweeps, scratch, s);
}

}  // namespace

Plan2d plan_resident2d(const Grid2& g, size_t esize) {
  Plan2d p;
  int dev = 0, sms = 0, optin = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    // no device (planning only): GB300's SMs and shared memory
    sms = 152;
    optin = 227 * 1024;
    per_sm = 228 * 1024;
  }
  // `ctas` bands per SM (the knob), fewer when their shared memory does not fit
  for (int ctas = g_ctas2d; ctas >= 1; ctas--) {
    i64 nblk = g.ny / g.r;  // every band owns at least R rows
    if (nblk > (i64)sms * ctas) nblk = (i64)sms * ctas;
    if (nblk < 1) nblk = 1;
    p.nblk = (int)nblk;
    p.nbmax = (int)((g.ny + nblk - 1) / nblk);
    const i64 rows = (i64)p.nbmax + 2 * g.r;
    // row layout: interior of every row 16-byte aligned (see the kernel)
    const i64 per16 = 16 / (i64)esize;
    p.pad = (int)((per16 - g.r % per16) % per16);
    p.ns = (int)((p.pad + g.NX() + per16 - 1) / per16 * per16);
    p.tma = (g.nx * (i64)esize) % 16 == 0 && g_tma2d != 0;
    const i64 smem = 2 * rows * p.ns * (i64)esize;
    i64 thr = (i64)p.nbmax * g.nx;
    thr = (thr + 31) / 32 * 32;
    const i64 thr_max = 1024 / ctas / 32 * 32;  // the SM's threads shared by its bands, whole warps
    p.threads = (int)(thr > thr_max ? thr_max : thr);
    p.smem = (size_t)smem;
    p.xchg_off = ((size_t)8 * p.nblk + 8 + 255) / 256 * 256;
    p.scratch = p.xchg_off + (size_t)2 * p.nblk * 2 * g.r * g.nx * esize;
    // leave room for the kernel's static shared memory
    p.ok = smem + 1024 <= optin && rows * p.ns < ((i64)1 << 31) &&
           (p.tma || g.nx <= kJ2Cols * (i64)p.threads);
    if (!p.ok || ctas == 1 || (smem + 2048) * ctas <= per_sm) return p;
  }
  return p;
}

bool use_resident2d(const Plan2d& p) { return p.ok && g_resident2d != 0; }

LaunchPlan sweep2d_launch_plan(const Grid2& g, size_t esize) {
  const Plan2d p = plan_resident2d(g, esize);
  LaunchPlan q;
  q.grid_y = q.grid_z = 1;
  if (use_resident2d(p)) {
    // one cooperative launch: band b owns rows [b ny / nblk, (b+1) ny / nblk)
    q.variant = 1;
    q.grid_x = p.nblk;
    q.block_threads = p.threads;
    q.tile_w = (int)g.nx;
    q.tile_h = p.nbmax;
    q.kchunk = 1;
    q.smem = (int)p.smem;
    q.row_stride = p.ns;
    q.row_pad = p.pad;
    q.bulk_copy = p.tma ? 1 : 0;
    q.scratch = (i64)p.scratch;
    q.xchg_off = (i64)p.xchg_off;
  } else {
    // one launch per sweep, a grid-stride loop over 32 x 8 tiles
    q.variant = 0;
    q.grid_x = (int)star2d_blocks(g);
    q.block_threads = 256;
    q.tile_w = 32;
    q.tile_h = 8;
    q.kchunk = 1;
  }
  return q;
}

template <typename T>
int launch_star2d(const T* u, const T* b, T* out, const Grid2& g, const double* coeffs,
                  SweepMode mode, double* partials, cudaStream_t s) {
  return g.r == 1 ? launch_j2d_r<T, 1>(u, b, out, g, coeffs, mode, partials, s)
                  : launch_j2d_r<T, 2>(u, b, out, g, coeffs, mode, partials, s);
}

i64 star2d_blocks(const Grid2& g) {
  const i64 ntiles = ((g.nx + 31) / 32) * ((g.ny + 7) / 8);
  return ntiles < kJ2dBlocks ? ntiles : kJ2dBlocks;
}

template <typename T>
int sweep2d_run(const T* in, T* out, const Grid2& g, const double* coeffs, i64 iters,
                unsigned char* scratch, const Plan2d& p, bool resident, T* pingpong,
                cudaStream_t s) {
  const size_t bytes = (size_t)g.count() * sizeof(T);
  if (resident) {
    int* status = reinterpret_cast<int*>(scratch + 8 * (size_t)p.nblk);
    STN_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
    const T* src = in;
    for (i64 done = 0; done < iters;) {
      i64 n = iters - done;
      if (n > g_chunk2d) n = g_chunk2d;
      if (int rc = launch_resident<T>(src, out, g, coeffs, p, (int)n, scratch, s)) return rc;
      src = out;  // later launches run in place (see the kernel's exchange order)
      done += n;
    }
    int host_status = 0;
    STN_CUDA_TRY(cudaMemcpyAsync(&host_status, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    STN_CUDA_TRY(cudaStreamSynchronize(s));
    if (host_status != 0) {
      set_error("2-D sweep: a device-side wait for a neighbouring band ran out");
      return STN_ETIMEOUT;
    }
    return STN_OK;
  }
  // per-sweep path: out and `pingpong` alternate; both start as copies of in
  STN_CUDA_TRY(cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, s));
  if (pingpong != in) STN_CUDA_TRY(cudaMemcpyAsync(pingpong, in, bytes, cudaMemcpyDeviceToDevice, s));
  const T* cur = in;
  T* nxt = out;
  for (i64 it = 0; it < iters; it++) {
    if (int rc = launch_star2d<T>(cur, nullptr, nxt, g, coeffs, kSweep, nullptr, s)) return rc;
    cur = nxt;
    nxt = (nxt == out) ? pingpong : out;
  }
  if (cur != out) STN_CUDA_TRY(cudaMemcpyAsync(out, cur, bytes, cudaMemcpyDeviceToDevice, s));
  STN_CUDA_TRY(cudaStreamSynchronize(s));
  return STN_OK;
}

template int launch_star2d<double>(const double*, const double*, double*, const Grid2&, const double*,
                                   SweepMode, double*, cudaStream_t);
template int launch_star2d<float>(const float*, const float*, float*, const Grid2&, const double*,
                                  SweepMode, double*, cudaStream_t);
template int sweep2d_run<double>(const double*, double*, const Grid2&, const double*, i64,
                                 unsigned char*, const Plan2d&, bool, double*, cudaStream_t);
template int sweep2d_run<float>(const float*, float*, const Grid2&, const double*, i64,
                                unsigned char*, const Plan2d&, bool, float*, cudaStream_t);

int tune_set_resident2d(int v) {
  if (v < -1 || v > 1) return STN_EINVAL;
  g_resident2d = v;
  return STN_OK;
}
int tune_get_resident2d() { return g_resident2d; }
int tune_set_chunk2d(i64 v) {
  if (v < 1 || v > ((i64)1 << 30)) return STN_EINVAL;
  g_chunk2d = v;
  return STN_OK;
}
i64 tune_get_chunk2d() { return g_chunk2d; }
int tune_set_withhold2d(int v) {
  if (v < 0 || v > 1) return STN_EINVAL;
  g_withhold2d = v;
  return STN_OK;
}
int tune_get_withhold2d() { return g_withhold2d; }
int tune_set_tma2d(int v) {
  if (v < 0 || v > 1) return STN_EINVAL;
  g_tma2d = v;
  return STN_OK;
}
int tune_get_tma2d() { return g_tma2d; }
int tune_set_ctas2d(int v) {
  if (v < 1 || v > 4) return STN_EINVAL;
  g_ctas2d = v;
  return STN_OK;
}
int tune_get_ctas2d() { return g_ctas2d; }

}  // namespace stn
