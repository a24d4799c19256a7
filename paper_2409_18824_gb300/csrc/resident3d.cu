// Many sweeps of a small 3-D grid in one cooperative launch.
//
// A sweep of a grid that stays in L2 (64^3 doubles: 2.3 MB) computes in a
// few microseconds, about as long as a kernel launch and its pipeline
// drain, so per-sweep launches leave the GPU idle most of the time.  Here
// every thread of a single cooperative launch owns up to RS_PMAX interior
// points (their offsets computed once), and each sweep it issues all of its
// points' neighbour loads at once (plain loads, after the barrier's acquire),
// computes
// the canonical update of the Jacobi sweep (arXiv 2409.18824 Sec. 4; the
// order of include/stencil.h, every operation rounded separately, so the
// iterates are bitwise those of the per-sweep kernels) and stores it.
// Sweeps are separated by a grid-wide barrier: one arrival counter that only
// grows (barrier g completes when it reaches nblocks * g) and a generation
// word released by the last arrival; waits are bounded (about two seconds),
// after which the launch records a timeout in its status word and every
// block stops.  The launch is cooperative, so all its blocks are resident
// together and the barrier cannot wait for a block that never runs.
// Optionally the last sweep also sums rho^2 = (new - old)^2 per block in a
// fixed order (one partial per block) for the residual norm.
#include <atomic>

#include "arith.cuh"
#include "internal.h"

namespace stn {

// knobs: resident sweeps on (1) or off (0); withhold (host-side fault
// injection): the last block of the next launches skips its barrier
// arrivals
static std::atomic<int> g_resident3d{1};
static std::atomic<int> g_withhold3d{0};

namespace {

constexpr int RS_THREADS = 512;
constexpr int RS_PMAX = 8;
// points whose loads are issued together: as many as two blocks of
// RS_THREADS per SM leave registers for (64 per thread)
template <typename T, int R>
struct RsBatch {
  static constexpr int value = sizeof(T) == 8 ? (R == 1 ? 2 : 1) : (R == 1 ? 4 : 2);
};
constexpr unsigned long long RS_WAIT_NS = 2000000000ull;

template <typename T, int R>
struct RsCoeffs {
  T c[R + 1];
};

__device__ __forceinline__ unsigned long long rs_timer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier number `target` (1, 2, ...): bar[0] counts arrivals,
// bar[1] holds the last completed barrier.  False when the wait ran out or
// another block reported a failure.
// The block barrier orders the block's stores before thread 0's arrival,
// which releases them at gpu scope (atom.add.release); the last arrival
// acquires every other block's release (atom.acq_rel) and publishes the
// barrier with a release store; the others acquire it by polling
// (ld.acquire), and the block barrier orders the block's next loads after
// that acquire.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned target, int* status, int* stop_sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(prev) : "l"(bar) : "memory");
    if (prev + 1 == gridDim.x * target) {
      st_release(&bar[1], target);
    } else if (ld_acquire(&bar[1]) < target) {
      const unsigned long long t0 = rs_timer();
      while (ld_acquire(&bar[1]) < target) {
        if (*(volatile int*)status != 0 || rs_timer() - t0 > RS_WAIT_NS) {
          atomicCAS(status, 0, kResidentTimeout);
          *stop_sh = 1;
          break;
        }
      }
    }
  }
  __syncthreads();
  return *(volatile int*)stop_sh == 0;
}

// Loads of the grids: plain, L1-cached loads.  Each sweep's reads start after
// the grid barrier, whose gpu-scope acquire (ld.acquire.gpu, then the block
// barrier) orders them after every block's stores of the previous sweep, so
// the memory model guarantees they see those stores; within a sweep nothing
// read is written.  L1 then serves the neighbour loads of a point that its
// neighbours already brought in.
template <typename T>
__device__ __forceinline__ T ldcg(const T* p) {
  return *p;
}

template <typename T, int R, bool HAS_B, bool HAS_C0>
__global__ void __launch_bounds__(RS_THREADS, 2)
    star_resident_kernel(T* a, T* b2, const T* rhs, int nx, int ny, int nz, int NX, int NY, RsCoeffs<T, R> cf,
                         long long sweeps, int resid_last, double* partials, unsigned* bar, int* status,
                         int withhold) {
  using A = Arith<T>;
  __shared__ double red[RS_THREADS / 32];
  __shared__ int stop_sh;
  if (threadIdx.x == 0) stop_sh = 0;
  const int gthreads = gridDim.x * blockDim.x;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int npts = nx * ny * nz;
  int off[RS_PMAX];
#pragma unroll
  for (int m = 0; m < RS_PMAX; m++) {
    const int q = gtid + m * gthreads;
    off[m] = -1;
    if (q < npts) {
      const int i = q % nx, rw = q / nx, j = rw % ny, k = rw / ny;
      off[m] = (i + R) + NX * ((j + R) + NY * (k + R));
    }
  }
  const int sy = NX, sz = NX * NY;
  __syncthreads();
  for (long long s = 0; s < sweeps; s++) {
    const T* src = (s & 1) ? b2 : a;
    T* dst = (s & 1) ? a : b2;
    const bool resid = resid_last && s == sweeps - 1;
    double rsum = 0.0;
    // points in batches: every load of a batch is issued before its first
    // store (the compiler may not move a load above a store to the other
    // buffer, which it cannot prove distinct), so a batch costs one L2 latency
    constexpr int NB = 1 + 6 * R + (HAS_B ? 1 : 0);  // values one point reads
    constexpr int RS_BATCH = RsBatch<T, R>::value;
#pragma unroll
    for (int m0 = 0; m0 < RS_PMAX; m0 += RS_BATCH) {
      if (off[m0] < 0) break;  // points are numbered in order: none left
      T v[RS_BATCH][NB];
#pragma unroll
      for (int bq = 0; bq < RS_BATCH; bq++) {
        const int o = off[m0 + bq];
        if (o >= 0) {
          const T* p = src + o;
          v[bq][0] = ldcg(p);
#pragma unroll
          for (int d = 1; d <= R; d++) {
            v[bq][6 * d - 5] = ldcg(p - d);
            v[bq][6 * d - 4] = ldcg(p + d);
            v[bq][6 * d - 3] = ldcg(p - d * sy);
            v[bq][6 * d - 2] = ldcg(p + d * sy);
            v[bq][6 * d - 1] = ldcg(p - d * sz);
            v[bq][6 * d] = ldcg(p + d * sz);
          }
          if (HAS_B) v[bq][NB - 1] = ldcg(rhs + o);
        }
      }
#pragma unroll
      for (int bq = 0; bq < RS_BATCH; bq++) {
        const int o = off[m0 + bq];
        if (o >= 0) {
          const T c = v[bq][0];
          T acc = T(0);
#pragma unroll
          for (int d = R; d >= 1; d--) {
            const T sx = A::add(v[bq][6 * d - 5], v[bq][6 * d - 4]);
            const T syy = A::add(v[bq][6 * d - 3], v[bq][6 * d - 2]);
            const T szz = A::add(v[bq][6 * d - 1], v[bq][6 * d]);
            const T t = A::mul(cf.c[d], A::add(A::add(sx, syy), szz));
            acc = (d == R) ? t : A::add(acc, t);
          }
          if (HAS_C0) acc = A::add(acc, A::mul(cf.c[0], c));
          if (HAS_B) acc = A::add(acc, v[bq][NB - 1]);
          __stcg(dst + o, acc);
          if (resid) {
            const double rho = (double)acc - (double)c;
            rsum = __fma_rn(rho, rho, rsum);
          }
        }
      }
    }
    if (resid) {
      // fixed-order block sum: warp shuffles, then warp 0 over the warps
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
      if (lane == 0) red[warp] = rsum;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < RS_THREADS / 32; w++) t += red[w];
        partials[blockIdx.x] = t;
      }
    }
    // host-side fault injection: the last block leaves before its first
    // arrival, so every other block's bounded wait runs out
    if (withhold && blockIdx.x == gridDim.x - 1) return;
    if (s + 1 < sweeps && !grid_barrier(bar, (unsigned)(s + 1), status, &stop_sh)) return;
  }
}

template <typename T, int R, bool HAS_B, bool HAS_C0>
int rs_blocks_per_sm() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    (void)cudaGetLastError();
    return 2;
  }
  const int known = cache[dev].load(std::memory_order_relaxed);
  if (known > 0) return known;
  int v = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, star_resident_kernel<T, R, HAS_B, HAS_C0>, RS_THREADS, 0) !=
          cudaSuccess ||
      v < 1) {
    (void)cudaGetLastError();
    return 2;  // no device (planning only)
  }
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

template <typename T, int R, bool HAS_B, bool HAS_C0>
int launch_t(T* a, T* b2, const T* rhs, const Grid& g, const double* coeffs, i64 sweeps, bool resid_last,
             double* partials, i64* nparts, unsigned* bar, int* status, cudaStream_t s) {
  const i64 npts = g.interior();
  const i64 cap_blocks = (i64)device_sms() * rs_blocks_per_sm<T, R, HAS_B, HAS_C0>();
  const i64 nb = resident3d_blocks(g);
  if (nb > cap_blocks || npts > nb * RS_THREADS * RS_PMAX) {
    set_error("grid too large for the resident sweep");
    return STN_EINVAL;
  }
  RsCoeffs<T, R> cf;
  for (int d = 0; d <= R; d++) cf.c[d] = (T)coeffs[d];
  int nx = (int)g.nx, ny = (int)g.ny, nz = (int)g.nz, NX = (int)g.NX(), NY = (int)g.NY();
  long long sw = sweeps;
  int rl = resid_last ? 1 : 0;
  int wh = g_withhold3d.load() ? 1 : 0;
  STN_CUDA_TRY(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
  void* args[] = {&a, &b2, &rhs, &nx, &ny, &nz, &NX, &NY, &cf, &sw, &rl, &partials, &bar, &status, &wh};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nb);
  cfg.blockDim = dim3(RS_THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  STN_CUDA_TRY(cudaLaunchKernelExC(&cfg, (const void*)star_resident_kernel<T, R, HAS_B, HAS_C0>, args));
  if (nparts) *nparts = nb;
  return STN_OK;
}

}  // namespace

int tune_set_withhold3d(int v) {
  if (v < 0 || v > 1) return STN_EINVAL;
  g_withhold3d = v;
  return STN_OK;
}
int tune_get_withhold3d() { return g_withhold3d.load(); }
int tune_set_resident3d(int v) {
  if (v < 0 || v > 1) return STN_EINVAL;
  g_resident3d = v;
  return STN_OK;
}
int tune_get_resident3d() { return g_resident3d.load(); }

// Grids of at most 2^18 interior points (64^3).  Measured per sweep (GB300,
// microseconds, resident / per-sweep kernels in device-repeated graphs):
// 32^3 double 3.48 / 4.80, float 2.90 / 3.96; 64^3 double 6.63 / 6.56, float
// 4.30 / 4.05 (the 64^3 FP64 configuration of 100 sweeps and a norm: 0.705 /
// 0.753 ms per step); 96^3 double 16.0 / 13.8, float 8.86 / 4.43.  A grid
// barrier costs about 2.5 us of round trips to L2, so beyond these sizes the
// per-sweep kernels, which read each value once through shared memory, win.
constexpr i64 kResidentMaxPoints = (i64)1 << 18;

bool resident3d_applicable(const Grid& g, size_t esize) {
  if (!g_resident3d.load()) return false;
  (void)esize;
  // also: every point one of at most RS_PMAX per thread of two blocks of
  // RS_THREADS per SM (the kernels are bounded to 64 registers: two fit),
  // and 32-bit offsets
  const i64 cap = (i64)device_sms() * 2 * RS_THREADS * RS_PMAX;
  return g.interior() <= kResidentMaxPoints && g.interior() <= cap && g.count() < ((i64)1 << 31);
}

// At most two blocks per SM, so that a grid barrier has few arrivals, unless
// the grid needs more to keep to RS_PMAX points per thread.
i64 resident3d_blocks(const Grid& g) {
  const i64 npts = g.interior();
  i64 nb = (npts + RS_THREADS - 1) / RS_THREADS;
  const i64 two = (i64)device_sms() * 2;
  if (nb > two) nb = two;
  const i64 need = (npts + (i64)RS_THREADS * RS_PMAX - 1) / ((i64)RS_THREADS * RS_PMAX);
  return nb > need ? nb : need;
}

template <typename T>
int launch_star_resident(T* a, T* b2, const T* rhs, const Grid& g, const double* coeffs, i64 sweeps,
                         bool resid_last, double* partials, i64* nparts, unsigned* bar, int* status,
                         cudaStream_t s) {
  const bool hb = rhs != nullptr, hc0 = coeffs[0] != 0.0;
#define STN_RS(RR, HB, HC)                                                                                   \
  return launch_t<T, RR, HB, HC>(a, b2, rhs, g, coeffs, sweeps, resid_last, partials, nparts, bar, status, s)
  if (g.r == 1) {
    if (hb) {
      if (hc0) STN_RS(1, true, true);
      STN_RS(1, true, false);
    }
    if (hc0) STN_RS(1, false, true);
    STN_RS(1, false, false);
  }
  if (hb) {
    if (hc0) STN_RS(2, true, true);
    STN_RS(2, true, false);
  }
  if (hc0) STN_RS(2, false, true);
  STN_RS(2, false, false);
#undef STN_RS
}

template int launch_star_resident<double>(double*, double*, const double*, const Grid&, const double*, i64, bool,
                                          double*, i64*, unsigned*, int*, cudaStream_t);
template int launch_star_resident<float>(float*, float*, const float*, const Grid&, const double*, i64, bool,
                                         double*, i64*, unsigned*, int*, cudaStream_t);

}  // namespace stn
