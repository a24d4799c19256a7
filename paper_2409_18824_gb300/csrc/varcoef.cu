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

template <typename T, int R>
int launch_var_t(const T* u, const T* a, const T* f, T* out, const Grid& g, const double* w,
                 VarMode mode, double* partials, double* partials_max, cudaStream_t s) {
  const ZPlan p = plan_var(g);
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

ZPlan plan_var(const Grid& g) { return plan_star(g, kStarScalar, 8); }

template <typename T>
int launch_var(const T* u, const T* a, const T* f, T* out, const Grid& g, const double* w,
               VarMode mode, double* partials, double* partials_max, cudaStream_t s) {
  if (g.r == 1) return launch_var_t<T, 1>(u, a, f, out, g, w, mode, partials, partials_max, s);
  return launch_var_t<T, 2>(u, a, f, out, g, w, mode, partials, partials_max, s);
}

template int launch_var<double>(const double*, const double*, const double*, double*, const Grid&,
                                const double*, VarMode, double*, double*, cudaStream_t);
template int launch_var<float>(const float*, const float*, const float*, float*, const Grid&,
                               const double*, VarMode, double*, double*, cudaStream_t);

}  // namespace stn
