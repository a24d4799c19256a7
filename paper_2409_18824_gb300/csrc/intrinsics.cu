// The Fortran `sum` and `dotproduct` intrinsics on a GPU-resident array
// (arXiv 2409.18824 Sec. 5.4, Table 3: the sum of a 32768 x 32768 double
// array and the dot product of two 134-million-element double vectors; both
// are the linalg.reduce of Sec. 5.3 / Listing 8 -- zero initial value, add
// combiner).
//
// Both stream through HBM once (8 or 16 bytes per element).  The dot
// product is bound by HBM.  The sum is not: it needs one double add per
// 8 bytes, and GB300 issues only 2 double FMAs per clock per SM (adds as FMAs
// with a unit factor; plain adds run at 1.7), which caps a 2^30-element sum
// at ~1.8 ms against ~1.3 ms of HBM time.  The design is about bytes in flight: a fixed grid of 4 blocks of
// 256 threads per SM; per step a block reads a tile of 256 x U 16-byte
// vectors (U = 8 for sum, 4 per operand for dot: 128 bytes in flight per
// thread, ~128 KB per SM) with streaming (evict-first) loads and keeps U
// independent accumulators per thread.  Block b takes tiles b, b + G, ...;
// the leftover vectors go round the grid one per thread, an odd last element
// to the last block.  Each block reduces its threads in a fixed order into
// one partial and the partials are added in index order (reduce.cu), so the
// result depends only on n and the operands' 16-byte alignment.
#include "arith.cuh"
#include "star.cuh"

namespace stn {

namespace {

constexpr int kRedThreads = 256;

// The sum: one tile of prefetch per thread (the next tile's loads are issued
// before the current tile's adds), so the FP64 pipe, which bounds the sum,
// keeps working while loads are in flight.
__global__ void __launch_bounds__(kRedThreads)
    sum_kernel(const double* __restrict__ x, i64 n, int head, double* __restrict__ partials) {
  constexpr int U = 4;
  using A = Arith<double>;
  __shared__ double red[kRedThreads / 32];
  double acc[2 * U];
#pragma unroll
  for (int u = 0; u < 2 * U; u++) acc[u] = 0.0;
  if (head && blockIdx.x == 0 && threadIdx.x == 0) acc[0] = x[0];
  const double* xa = x + head;  // 16-byte aligned from here
  const i64 m = n - head;
  const double2* x2 = reinterpret_cast<const double2*>(xa);
  const i64 n2 = m >> 1;
  constexpr i64 tile = (i64)kRedThreads * U;
  const i64 ntiles = n2 / tile;
  double2 a[U];
  i64 t = blockIdx.x;
  if (t < ntiles) {
#pragma unroll
    for (int u = 0; u < U; u++) a[u] = __ldcs(x2 + t * tile + threadIdx.x + u * kRedThreads);
  }
  for (; t < ntiles; t += gridDim.x) {
    const i64 tn = t + gridDim.x;
    double2 nxt[U];
    if (tn < ntiles) {
#pragma unroll
      for (int u = 0; u < U; u++) nxt[u] = __ldcs(x2 + tn * tile + threadIdx.x + u * kRedThreads);
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      acc[2 * u] = A::add(acc[2 * u], a[u].x);
      acc[2 * u + 1] = A::add(acc[2 * u + 1], a[u].y);
    }
#pragma unroll
    for (int u = 0; u < U; u++) a[u] = nxt[u];
  }
  for (i64 k = ntiles * tile + (i64)blockIdx.x * kRedThreads + threadIdx.x; k < n2;
       k += (i64)gridDim.x * kRedThreads) {
    const double2 v = __ldcs(x2 + k);
    acc[0] = A::add(A::add(acc[0], v.x), v.y);
  }
  if ((m & 1) && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) acc[0] = A::add(acc[0], xa[m - 1]);
  double v = acc[0];
#pragma unroll
  for (int u = 1; u < 2 * U; u++) v = A::add(v, acc[u]);
  const double tot = block_sum_fixed<kRedThreads>(v, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// The dot product (HBM-bound): U tiles of both operands per step.
template <bool DOT>
__global__ void __launch_bounds__(kRedThreads)
    vec_reduce_kernel(const double* __restrict__ x, const double* __restrict__ y, i64 n, int head,
                      double* __restrict__ partials) {
  constexpr int U = DOT ? 4 : 8;
  __shared__ double red[kRedThreads / 32];
  double acc[U];
#pragma unroll
  for (int u = 0; u < U; u++) acc[u] = 0.0;
  if (head && blockIdx.x == 0 && threadIdx.x == 0) acc[0] = DOT ? x[0] * y[0] : x[0];
  const double* xa = x + head;  // 16-byte aligned from here
  const double* ya = DOT ? y + head : nullptr;
  const i64 m = n - head;
  const double2* x2 = reinterpret_cast<const double2*>(xa);
  const double2* y2 = reinterpret_cast<const double2*>(ya);
  const i64 n2 = m >> 1;
  constexpr i64 tile = (i64)kRedThreads * U;
  const i64 ntiles = n2 / tile;
  for (i64 t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const i64 base = t * tile + threadIdx.x;
    double2 a[U], b[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      a[u] = __ldcs(x2 + base + u * kRedThreads);
      if (DOT) b[u] = __ldcs(y2 + base + u * kRedThreads);
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      if (DOT) {
        acc[u] = __fma_rn(a[u].x, b[u].x, acc[u]);
        acc[u] = __fma_rn(a[u].y, b[u].y, acc[u]);
      } else {
        acc[u] = Arith<double>::add(Arith<double>::add(acc[u], a[u].x), a[u].y);
      }
    }
  }
  for (i64 k = ntiles * tile + (i64)blockIdx.x * kRedThreads + threadIdx.x; k < n2;
       k += (i64)gridDim.x * kRedThreads) {
    const double2 a = __ldcs(x2 + k);
    if (DOT) {
      const double2 b = __ldcs(y2 + k);
      acc[0] = __fma_rn(a.y, b.y, __fma_rn(a.x, b.x, acc[0]));
    } else {
      acc[0] = Arith<double>::add(Arith<double>::add(acc[0], a.x), a.y);
    }
  }
  if ((m & 1) && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
    acc[0] = DOT ? __fma_rn(xa[m - 1], ya[m - 1], acc[0]) : __dadd_rn(acc[0], xa[m - 1]);
  double v = acc[0];
#pragma unroll
  for (int u = 1; u < U; u++) v = __dadd_rn(v, acc[u]);
  const double tot = block_sum_fixed<kRedThreads>(v, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// Operands whose 16-byte phases differ (dot only): scalar loads.
__global__ void __launch_bounds__(kRedThreads)
    dot_scalar_kernel(const double* __restrict__ x, const double* __restrict__ y, i64 n,
                      double* __restrict__ partials) {
  constexpr int U = 4;
  __shared__ double red[kRedThreads / 32];
  double acc[U] = {0.0, 0.0, 0.0, 0.0};
  constexpr i64 tile = (i64)kRedThreads * U;
  const i64 ntiles = n / tile;
  for (i64 t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const i64 base = t * tile + threadIdx.x;
#pragma unroll
    for (int u = 0; u < U; u++)
      acc[u] = __fma_rn(__ldcs(x + base + u * kRedThreads), __ldcs(y + base + u * kRedThreads), acc[u]);
  }
  for (i64 k = ntiles * tile + (i64)blockIdx.x * kRedThreads + threadIdx.x; k < n;
       k += (i64)gridDim.x * kRedThreads)
    acc[0] = __fma_rn(__ldcs(x + k), __ldcs(y + k), acc[0]);
  const double v = __dadd_rn(__dadd_rn(acc[0], acc[1]), __dadd_rn(acc[2], acc[3]));
  const double tot = block_sum_fixed<kRedThreads>(v, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

}  // namespace

i64 vec_reduce_blocks(i64 n) {
  // 4 blocks per SM for large arrays; fewer (a function of n only) for small
  const i64 full = 152 * 4;
  const i64 want = (n + 2 * kRedThreads * 8 - 1) / (2 * kRedThreads * 8);
  return want < 1 ? 1 : (want > full ? full : want);
}

int launch_vec_reduce(const double* x, const double* y, i64 n, double* partials, cudaStream_t s) {
  const i64 blocks = vec_reduce_blocks(n);
  const uintptr_t px = (uintptr_t)x, py = (uintptr_t)y;
  if (!y) {
    const int head = (px & 15) ? 1 : 0;
    sum_kernel<<<(unsigned)blocks, kRedThreads, 0, s>>>(x, n, n > 0 ? head : 0, partials);
  } else if ((px & 15) == (py & 15)) {
    const int head = (px & 15) ? 1 : 0;
    vec_reduce_kernel<true><<<(unsigned)blocks, kRedThreads, 0, s>>>(x, y, n, n > 0 ? head : 0, partials);
  } else {
    dot_scalar_kernel<<<(unsigned)blocks, kRedThreads, 0, s>>>(x, y, n, partials);
  }
  STN_CUDA_TRY(cudaGetLastError());
  return STN_OK;
}

}  // namespace stn
