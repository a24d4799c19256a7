// Deterministic second stage of the residual reductions (arXiv 2409.18824
// Sec. 5.3 / Listing 8: a sum initialised to zero with an add combiner).
// Per-block partials written by the sweep kernels are added here by a single
// block in a fixed order (strided per-thread sums, then a fixed tree), so the
// result depends only on the number of partials, never on timing.
#include <math.h>

#include "internal.h"

namespace stn {

namespace {

constexpr int FT = 1024;

__device__ __forceinline__ double tree_sum_1024(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = red[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;
}

__device__ __forceinline__ double tree_max_1024(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = red[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
  }
  return t;
}

// dst[0] = sum, dst[1] = sqrt(sum); if scale_src: dst[2] = dst[1] / scale
// (scale = *scale_src, or 1 when it is 0) and dst[3] = (dst[2] <= tol).
__global__ void __launch_bounds__(FT) finalize_kernel(const double* __restrict__ partials, i64 n,
                                                      double* __restrict__ dst,
                                                      const double* __restrict__ scale_src,
                                                      double tol) {
  __shared__ double red[32];
  double v = 0.0;
  for (i64 i = threadIdx.x; i < n; i += FT) v += partials[i];
  const double t = tree_sum_1024(v, red);
  if (threadIdx.x == 0) {
    dst[0] = t;
    const double nrm = sqrt(t);
    dst[1] = nrm;
    if (scale_src) {
      double sc = *scale_src;
      if (!(sc > 0.0)) sc = 1.0;
      dst[2] = nrm / sc;
      dst[3] = (nrm / sc <= tol) ? 1.0 : 0.0;
    }
  }
}

// Device-side convergence decision of the graph-driven solve: the same
// fixed-order sum as finalize_kernel (so the same bits as the host-driven
// loop), then iteration bookkeeping and the while-node condition.
// dst[0] sum, [1] norm, [2] rel, [3] converged, [5] sweeps done (as double).
__global__ void __launch_bounds__(FT) decide_kernel(const double* __restrict__ partials, i64 n,
                                                    double* __restrict__ dst, double tol, i64 group,
                                                    i64 max_full, cudaGraphConditionalHandle h) {
  __shared__ double red[32];
  double v = 0.0;
  for (i64 i = threadIdx.x; i < n; i += FT) v += partials[i];
  const double t = tree_sum_1024(v, red);
  if (threadIdx.x == 0) {
    dst[0] = t;
    const double nrm = sqrt(t);
    dst[1] = nrm;
    double sc = dst[9];
    if (!(sc > 0.0)) sc = 1.0;
    const double rel = nrm / sc;
    dst[2] = rel;
    const bool conv = rel <= tol;
    dst[3] = conv ? 1.0 : 0.0;
    const i64 it = (i64)dst[5] + group;
    dst[5] = (double)it;
    cudaGraphSetConditional(h, (!conv && it + group <= max_full) ? 1u : 0u);
  }
}

// Loop counter of a device-repeated graph body: one more repetition done;
// the while node runs again while fewer than n are done.
__global__ void count_kernel(unsigned long long* __restrict__ ctr, unsigned long long n,
                             cudaGraphConditionalHandle h) {
  const unsigned long long v = *ctr + 1;
  *ctr = v;
  cudaGraphSetConditional(h, v < n ? 1u : 0u);
}

__global__ void __launch_bounds__(FT) max_finalize_kernel(const double* __restrict__ partials,
                                                          i64 n, double* __restrict__ dst) {
  __shared__ double red[32];
  double v = 0.0;
  for (i64 i = threadIdx.x; i < n; i += FT) v = fmax(v, partials[i]);
  const double t = tree_max_1024(v, red);
  if (threadIdx.x == 0) dst[0] = t;
}

template <typename T>
__global__ void __launch_bounds__(256) interior_sumsq_kernel(const T* __restrict__ x, int nx, int ny,
                                                             int nz, int r,
                                                             double* __restrict__ partials) {
  // one block per (j, k) row group: grid-stride over interior rows, fixed order
  __shared__ double red[8];
  const i64 NX = nx + 2 * r, NY = ny + 2 * r;
  const i64 rows = (i64)ny * nz;
  double v = 0.0;
  for (i64 row = blockIdx.x; row < rows; row += gridDim.x) {
    const i64 j = row % ny + r, k = row / ny + r;
    const T* p = x + r + NX * (j + NY * k);
    for (int i = threadIdx.x; i < nx; i += 256) {
      const double e = (double)p[i];
      v = __fma_rn(e, e, v);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; w++) t += red[w];
    partials[blockIdx.x] = t;
  }
}

}  // namespace

int launch_finalize(const double* partials, i64 n, double* dst, const double* scale_src, double tol,
                    cudaStream_t s) {
  finalize_kernel<<<1, FT, 0, s>>>(partials, n, dst, scale_src, tol);
  STN_CUDA_TRY(cudaGetLastError());
  return STN_OK;
}

int launch_decide(const double* partials, i64 n, double* dst, double tol, i64 group, i64 max_full,
                  cudaGraphConditionalHandle h, cudaStream_t s) {
  decide_kernel<<<1, FT, 0, s>>>(partials, n, dst, tol, group, max_full, h);
  STN_CUDA_TRY(cudaGetLastError());
  return STN_OK;
}

int launch_count(unsigned long long* ctr, i64 n, cudaGraphConditionalHandle h, cudaStream_t s) {
  count_kernel<<<1, 1, 0, s>>>(ctr, (unsigned long long)n, h);
  STN_CUDA_TRY(cudaGetLastError());
  return STN_OK;
}

int launch_max_finalize(const double* partials, i64 n, double* dst, cudaStream_t s) {
  max_finalize_kernel<<<1, FT, 0, s>>>(partials, n, dst);
  STN_CUDA_TRY(cudaGetLastError());
  return STN_OK;
}

template <typename T>
int launch_interior_sumsq(const T* x, const Grid& g, double* partials, i64* nparts, cudaStream_t s) {
  i64 rows = g.ny * g.nz;
  i64 blocks = rows < 152 * 8 ? rows : 152 * 8;
  interior_sumsq_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(x, (int)g.nx, (int)g.ny, (int)g.nz, g.r,
                                                           partials);
  STN_CUDA_TRY(cudaGetLastError());
  *nparts = blocks;
  return STN_OK;
}

template int launch_interior_sumsq<double>(const double*, const Grid&, double*, i64*, cudaStream_t);
template int launch_interior_sumsq<float>(const float*, const Grid&, double*, i64*, cudaStream_t);

}  // namespace stn
