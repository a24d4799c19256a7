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
//    Per sweep a CTA computes its R top and R bottom rows first, copies them
//    to a global exchange slot and publishes a counter (release store), then
//    computes its inner rows while those rows travel through L2, and finally
//    waits (acquire poll, bounded) for the neighbours' counters and copies
//    their boundary rows into its halo rows.  Exchange slots alternate with
//    the sweep parity: a CTA can only overwrite a slot two sweeps later, after
//    both neighbours have published the sweep in between, i.e. after they
//    have read it.
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

// Buffer rows [L0, L1) of a band (buffer row L = padded grid row jb + L),
// interior columns: nxt = S(cur).  Threads walk the rows x columns rectangle
// in row-major order without division.
template <typename T, int R, bool HAS_C0>
__device__ __forceinline__ void band_rows(const T* cur, T* nxt, int NX, int nx, int L0, int L1,
                                          const Co2<T, R>& cf) {
  if (L1 <= L0) return;
  int l = L0 + (int)threadIdx.x / nx;
  int i = (int)threadIdx.x % nx;
  while (l < L1) {
    const int o = l * NX + i + R;
    nxt[o] = point2d<T, R, HAS_C0>(cur + o, NX, cf);
    i += blockDim.x;
    while (i >= nx) {
      i -= nx;
      l++;
    }
  }
}

// Copies `rows` rows of `nx` interior values between shared memory (row
// stride NX, starting at column R) and a packed global slot.
template <typename T, int R, bool TO_GLOBAL>
__device__ __forceinline__ void copy_rows(T* sm, T* gl, int NX, int nx, int rows) {
  const int n = rows * nx;
  int l = (int)threadIdx.x / nx;
  int i = (int)threadIdx.x % nx;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    if (TO_GLOBAL)
      gl[c] = sm[l * NX + i + R];
    else
      sm[l * NX + i + R] = __ldcg(gl + c);
    i += blockDim.x;
    while (i >= nx) {
      i -= nx;
      l++;
    }
  }
}

template <typename T, int R, bool HAS_C0>
__global__ void __launch_bounds__(1024, 1)
    j2d_resident_kernel(const T* src, T* dst, int nx, int ny, int NX, int nbmax, int sweeps,
                        Co2<T, R> cf, T* __restrict__ xchg, unsigned long long* __restrict__ flags,
                        int* __restrict__ status, long long spin_limit, int withhold_last) {
  extern __shared__ __align__(16) unsigned char j2_smem[];
  __shared__ int s_abort;
  const int nblk = gridDim.x, b = blockIdx.x;
  const int jb = (int)(((long long)b * ny) / nblk);
  const int nb = (int)(((long long)(b + 1) * ny) / nblk) - jb;  // own rows (>= R)
  const int LR = nb + 2 * R;
  T* buf0 = reinterpret_cast<T*>(j2_smem);
  T* buf1 = buf0 + (size_t)(nbmax + 2 * R) * NX;
  if (threadIdx.x == 0) s_abort = ld_volatile_i32(status);
  __syncthreads();
  if (s_abort) return;  // an earlier launch of this call timed out

  // both copies <- padded rows [jb, jb + LR) of src, full width
  for (int c = threadIdx.x; c < LR * NX; c += blockDim.x) {
    const T v = src[(size_t)jb * NX + c];
    buf0[c] = v;
    buf1[c] = v;
  }
  __syncthreads();

  const bool up = b > 0, down = b + 1 < nblk;
  const size_t slot = (size_t)R * nx;  // one side's rows in an exchange slot
  const bool publish = !(withhold_last && b == nblk - 1);
  for (int s = 0; s < sweeps; s++) {
    const T* cur = (s & 1) ? buf1 : buf0;
    T* nxt = (s & 1) ? buf0 : buf1;
    T* xs = xchg + (size_t)(s & 1) * nblk * 2 * slot;  // this sweep's exchange slots
    // boundary rows first: own rows [0, R) and [nb - R, nb) = buffer rows
    // [R, 2R) and [nb, nb + R) (all own rows when the band is that thin)
    if (nb <= 2 * R) {
      band_rows<T, R, HAS_C0>(cur, nxt, NX, nx, R, R + nb, cf);
    } else {
      band_rows<T, R, HAS_C0>(cur, nxt, NX, nx, R, 2 * R, cf);
      band_rows<T, R, HAS_C0>(cur, nxt, NX, nx, nb, nb + R, cf);
    }
    __syncthreads();
    if (up) copy_rows<T, R, true>(nxt + R * NX, xs + (size_t)(2 * b) * slot, NX, nx, R);
    if (down) copy_rows<T, R, true>(nxt + nb * NX, xs + (size_t)(2 * b + 1) * slot, NX, nx, R);
    __syncthreads();
    if (threadIdx.x == 0 && publish && (up || down)) {
      __threadfence();
      st_release_u64(flags + b, (unsigned long long)(s + 1));
    }
    // inner rows while the boundary rows travel
    if (nb > 2 * R) band_rows<T, R, HAS_C0>(cur, nxt, NX, nx, 2 * R, nb, cf);
    // neighbours' boundary rows -> this band's halo rows of the next iterate
    if (threadIdx.x == 0) {
      bool ok = true;
      if (up) ok = wait_flag(flags + b - 1, (unsigned long long)(s + 1), status, spin_limit);
      if (ok && down) ok = wait_flag(flags + b + 1, (unsigned long long)(s + 1), status, spin_limit);
      s_abort = ok ? 0 : 1;
    }
    __syncthreads();
    if (s_abort) return;
    if (up) copy_rows<T, R, false>(nxt, xs + (size_t)(2 * (b - 1) + 1) * slot, NX, nx, R);
    if (down) copy_rows<T, R, false>(nxt + (R + nb) * NX, xs + (size_t)(2 * (b + 1)) * slot, NX, nx, R);
    __syncthreads();
  }
  // own rows (and the grid's top / bottom halo rows for the end bands) -> dst
  const T* fin = (sweeps & 1) ? buf1 : buf0;
  const int L0 = b == 0 ? 0 : R, L1 = down ? R + nb : LR;
  for (int c = L0 * NX + threadIdx.x; c < L1 * NX; c += blockDim.x) dst[(size_t)jb * NX + c] = fin[c];
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
constexpr double kWait2dSeconds = 2.0;

template <typename T, int R, bool HAS_C0>
int launch_resident_t(const T* src, T* dst, const Grid2& g, const double* coeffs, const Plan2d& p,
                      int sweeps, unsigned char* scratch, cudaStream_t s) {
  Co2<T, R> cf;
  for (int d = 0; d <= R; d++) cf.c[d] = (T)coeffs[d];
  auto kern = j2d_resident_kernel<T, R, HAS_C0>;
  STN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
  unsigned long long* flags = reinterpret_cast<unsigned long long*>(scratch);
  int* status = reinterpret_cast<int*>(scratch + 8 * (size_t)p.nblk);
  T* xchg = reinterpret_cast<T*>(scratch + p.xchg_off);
  STN_CUDA_TRY(cudaMemsetAsync(flags, 0, 8 * (size_t)p.nblk, s));
  int nx = (int)g.nx, ny = (int)g.ny, NX = (int)g.NX(), nbmax = p.nbmax;
  int withhold = g_withhold2d;
  long long limit = (long long)(kWait2dSeconds * 2.07e9);
  void* args[] = {(void*)&src, (void*)&dst, &nx,    &ny,    &NX,    &nbmax,   &sweeps,
                  &cf,         &xchg,       &flags, &status, &limit, &withhold};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)kern, dim3(p.nblk), dim3(p.threads), args,
                                              p.smem, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchCooperativeKernel(j2d_resident_kernel)");
  return STN_OK;
}

template <typename T>
int launch_resident(const T* src, T* dst, const Grid2& g, const double* coeffs, const Plan2d& p,
                    int sweeps, unsigned char* scratch, cudaStream_t s) {
  const bool hc0 = coeffs[0] != 0.0;
  if (g.r == 1)
    return hc0 ? launch_resident_t<T, 1, true>(src, dst, g, coeffs, p, sweeps, scratch, s)
               : launch_resident_t<T, 1, false>(src, dst, g, coeffs, p, sweeps, scratch, s);
  return hc0 ? launch_resident_t<T, 2, true>(src, dst, g, coeffs, p, sweeps, scratch, s)
             : launch_resident_t<T, 2, false>(src, dst, g, coeffs, p, sweeps, scratch, s);
}

}  // namespace

Plan2d plan_resident2d(const Grid2& g, size_t esize) {
  Plan2d p;
  int dev = 0, sms = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return p;  // ok = false
  }
  i64 nblk = g.ny / g.r;  // every band owns at least R rows
  if (nblk > sms) nblk = sms;
  if (nblk < 1) nblk = 1;
  p.nblk = (int)nblk;
  p.nbmax = (int)((g.ny + nblk - 1) / nblk);
  const i64 rows = (i64)p.nbmax + 2 * g.r;
  const i64 smem = 2 * rows * g.NX() * (i64)esize;
  i64 thr = (i64)p.nbmax * g.nx;
  thr = (thr + 31) / 32 * 32;
  p.threads = (int)(thr > 1024 ? 1024 : thr);
  p.smem = (size_t)smem;
  p.xchg_off = ((size_t)8 * p.nblk + 8 + 255) / 256 * 256;
  p.scratch = p.xchg_off + (size_t)2 * p.nblk * 2 * g.r * g.nx * esize;
  // leave room for the kernel's static shared memory
  p.ok = smem + 1024 <= optin && rows * g.NX() < ((i64)1 << 31);
  return p;
}

bool use_resident2d(const Plan2d& p) { return p.ok && g_resident2d != 0; }

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

}  // namespace stn
