// Element-wise steps of the mixed-precision iterative refinement (double
// residual and update around float Jacobi sweeps).  Not in arXiv 2409.18824;
// the double work is confined to these kernels and the residual reduction.
#include "internal.h"

namespace stn {

namespace {

// Visits every interior point of a padded grid: grid-stride over rows.
template <typename F>
__device__ __forceinline__ void for_interior(int nx, int ny, int nz, int r, F&& f) {
  const i64 NX = nx + 2 * r, NY = ny + 2 * r;
  const i64 rows = (i64)ny * nz;
  for (i64 row = blockIdx.x; row < rows; row += gridDim.x) {
    const i64 j = row % ny + r, k = row / ny + r;
    const i64 base = r + NX * (j + NY * k);
    for (int i = threadIdx.x; i < nx; i += blockDim.x) f(base + i);
  }
}

__global__ void scale_kernel(const double* __restrict__ rho, float* __restrict__ r32, int nx, int ny,
                             int nz, int r, const double* __restrict__ smax) {
  const double s = *smax;
  for_interior(nx, ny, nz, r, [&](i64 p) { r32[p] = __double2float_rn(__ddiv_rn(rho[p], s)); });
}

__global__ void update_kernel(double* __restrict__ u, const float* __restrict__ e, int nx, int ny,
                              int nz, int r, const double* __restrict__ smax) {
  const double s = *smax;
  for_interior(nx, ny, nz, r, [&](i64 p) { u[p] = __dadd_rn(u[p], __dmul_rn(s, (double)e[p])); });
}

// Block maxima of |t - u| over the interior (the refinement's scale s), one
// partial per block in a fixed order.
__global__ void __launch_bounds__(256) diff_max_kernel(const double* __restrict__ t, const double* __restrict__ u,
                                                       int nx, int ny, int nz, int r,
                                                       double* __restrict__ partials) {
  __shared__ double red[8];
  double m = 0.0;
  for_interior(nx, ny, nz, r, [&](i64 p) { m = fmax(m, fabs(__dsub_rn(t[p], u[p]))); });
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) red[warp] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < 8; w++) v = fmax(v, red[w]);
    partials[blockIdx.x] = v;
  }
}

// r32 = float((t - u) / s): the refinement's scaled residual, rho = t - u
// formed in double exactly as the oracle forms it.
__global__ void scale_diff_kernel(const double* __restrict__ t, const double* __restrict__ u,
                                  float* __restrict__ r32, int nx, int ny, int nz, int r,
                                  const double* __restrict__ smax) {
  const double s = *smax;
  for_interior(nx, ny, nz, r,
               [&](i64 p) { r32[p] = __double2float_rn(__ddiv_rn(__dsub_rn(t[p], u[p]), s)); });
}

template <typename T, typename U>
__global__ void convert_kernel(const T* __restrict__ src, U* __restrict__ dst, i64 n) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    dst[i] = (U)src[i];
}

unsigned rows_blocks(const Grid& g) {
  i64 rows = g.ny * g.nz;
  return (unsigned)(rows < 152 * 16 ? rows : 152 * 16);
}

}  // namespace

int launch_refine_scale(const double* rho, float* r32, const Grid& g, const double* smax,
                        cudaStream_t s) {
  scale_kernel<<<rows_blocks(g), 256, 0, s>>>(rho, r32, (int)g.nx, (int)g.ny, (int)g.nz, g.r, smax);
  STN_CUDA_TRY(cudaGetLastError());
  return STN_OK;
}

int launch_refine_update(double* u, const float* e, const Grid& g, const double* smax,
                         cudaStream_t s) {
  update_kernel<<<rows_blocks(g), 256, 0, s>>>(u, e, (int)g.nx, (int)g.ny, (int)g.nz, g.r, smax);
  STN_CUDA_TRY(cudaGetLastError());
  return STN_OK;
}

int launch_diff_max(const double* t, const double* u, const Grid& g, double* partials, i64* nparts,
                    cudaStream_t s) {
  const unsigned blocks = rows_blocks(g);
  diff_max_kernel<<<blocks, 256, 0, s>>>(t, u, (int)g.nx, (int)g.ny, (int)g.nz, g.r, partials);
  STN_CUDA_TRY(cudaGetLastError());
  *nparts = blocks;
  return STN_OK;
}

int launch_refine_scale_diff(const double* t, const double* u, float* r32, const Grid& g, const double* smax,
                             cudaStream_t s) {
  scale_diff_kernel<<<rows_blocks(g), 256, 0, s>>>(t, u, r32, (int)g.nx, (int)g.ny, (int)g.nz, g.r, smax);
  STN_CUDA_TRY(cudaGetLastError());
  return STN_OK;
}

template <typename T, typename U>
int launch_convert(const T* src, U* dst, i64 n, cudaStream_t s) {
  i64 blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  convert_kernel<T, U><<<(unsigned)blocks, 256, 0, s>>>(src, dst, n);
  STN_CUDA_TRY(cudaGetLastError());
  return STN_OK;
}

template int launch_convert<double, float>(const double*, float*, i64, cudaStream_t);
template int launch_convert<float, double>(const float*, double*, i64, cudaStream_t);

}  // namespace stn
