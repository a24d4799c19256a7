// Opt-in double sweep evaluated in double-word (float pair) arithmetic.
//
// GB300 issues two double operations per clock per SM, so the canonical
// 7-point double update (6 double operations) cannot exceed about 105 GLUP/s
// whatever the memory system does.  This variant computes the same update,
// out = c1 * (((u(i-1)+u(i+1)) + (u(j-1)+u(j+1))) + (u(k-1)+u(k+1))), with
// every value held as an unevaluated sum hi + lo of two floats (about 48
// significant bits) on the FP32 pipe:
//   * a double is split with integer operations: hi = its top 24 significant
//     bits (truncated), lo = the remaining 29 bits rounded to a float (an
//     integer-to-float conversion scaled by an exact power of two), then
//     renormalised (Fast2Sum); |x - (hi + lo)| <= 2^-47 |x|;
//   * sums use the accurate double-word addition (two TwoSums and two
//     Fast2Sums; relative error <= 3 * 2^-48 + O(2^-72), Joldes, Muller and
//     Popescu, "Tight and rigorous error bounds for basic building blocks of
//     double-word arithmetic", 2017); the product with c1 (itself split into
//     a float pair) uses the FMA-based double-word product (relative error
//     <= 5 * 2^-48);
//   * the result hi + lo is formed in double by one exact addition of the two
//     floats' double images (built with integer operations), the only double
//     instruction of an update.
// It is not the canonical order and not bitwise the oracle; its error per
// sweep is bounded by about 40 * 2^-48 of the neighbourhood's largest value.
// Points whose values fall outside the float range that the split handles
// (nonzero magnitudes below 2^-74 or at or above 2^127) take the canonical
// double update instead.  Opt-in (knob fp64_double_word = 1): radius 1, no
// source term, c0 = 0 -- the 7-point Laplace Jacobi sweep.
#include <atomic>

#include "arith.cuh"
#include "internal.h"

namespace stn {

namespace {

constexpr int DW_TX = 32, DW_TY = 8;

struct dw {
  float h, l;
};

// Split of a double into a float pair; false when the value is outside the
// handled range (the caller then uses the double path for the point).
__device__ __forceinline__ bool split(double x, dw& r) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned e = (unsigned)(b >> 52) & 0x7FFu;
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const unsigned sign = (unsigned)(b >> 63) << 31;
  if (e == 0 && m == 0) {
    r.h = __uint_as_float(sign);
    r.l = 0.0f;
    return true;
  }
  // float exponent of hi: e - 1023 + 127 in [1, 254]; lo's scale 2^(e-1075)
  // must stay a normal float: e - 1075 + 127 >= 1, i.e. e >= 949
  if (e < 949u || e > 1150u) return false;
  const unsigned hbits = sign | ((e - 896u) << 23) | (unsigned)(m >> 29);
  const unsigned rem = (unsigned)(m & 0x1FFFFFFFull);           // the 29 bits below hi
  const float scale = __uint_as_float((e - 1075u + 127u) << 23);  // 2^(e - 1075), exact
  const float lo = __fmul_rn(__uint2float_rn(rem), scale);       // rem rounded to 24 bits, scaled exactly
  const float h = __uint_as_float(hbits), l = __uint_as_float(__float_as_uint(lo) | sign);
  // |l| < ulp(h): renormalise so that |lo| <= ulp(hi) / 2 (exact)
  r.h = __fadd_rn(h, l);
  r.l = __fsub_rn(l, __fsub_rn(r.h, h));
  return true;
}

// The double image of a float, built with integer operations (exact).
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned E = (u >> 23) & 0xFFu;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  if (E == 0) return __longlong_as_double((long long)sign);  // zero (subnormal floats do not occur here)
  const unsigned long long bits =
      sign | ((unsigned long long)(E + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  t = __fsub_rn(b, __fsub_rn(s, a));
}

// accurate double-word + double-word
__device__ __forceinline__ dw add(dw x, dw y) {
  float sh, sl, th, tl, vh, vl;
  two_sum(x.h, y.h, sh, sl);
  two_sum(x.l, y.l, th, tl);
  const float c = __fadd_rn(sl, th);
  fast_two_sum(sh, c, vh, vl);
  const float w = __fadd_rn(tl, vl);
  dw z;
  fast_two_sum(vh, w, z.h, z.l);
  return z;
}

// double-word x double-word with FMA
__device__ __forceinline__ dw mul(dw x, dw y) {
  const float ch = __fmul_rn(x.h, y.h);
  const float cl1 = __fmaf_rn(x.h, y.h, -ch);
  const float tl0 = __fmul_rn(x.l, y.l);
  const float tl1 = __fmaf_rn(x.h, y.l, tl0);
  const float cl2 = __fmaf_rn(x.l, y.h, tl1);
  const float cl3 = __fadd_rn(cl1, cl2);
  dw z;
  fast_two_sum(ch, cl3, z.h, z.l);
  return z;
}

// The plane kernel's structure (32 x 8 tile of columns, k streamed, register
// queue of the column's planes k-1..k+1, in-plane neighbours from a shared
// plane with a one-cell halo), with every value a float pair.
__global__ void __launch_bounds__(DW_TX* DW_TY)
    star_dw_kernel(const double* __restrict__ u, double* __restrict__ out, int nx, int ny, int nz, int NX, int NY,
                   int kchunk, dw c1, double c1d) {
  using A = Arith<double>;
  __shared__ float2 tile[DW_TY + 2][DW_TX + 2];
  __shared__ unsigned char bad[DW_TY + 2][DW_TX + 2];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int gi = blockIdx.x * DW_TX + tx + 1, gj = blockIdx.y * DW_TY + ty + 1;
  const i64 sy = NX, sz = (i64)NX * NY;
  const int k0 = 1 + blockIdx.z * kchunk;
  const int k1 = min(k0 + kchunk, nz + 1);
  const bool inx = gi < NX, iny = gj < NY;
  const bool active = gi < nx + 1 && gj < ny + 1;
  const bool hx = tx == 0 || tx == DW_TX - 1;
  const int hx_i = tx == 0 ? gi - 1 : gi + 1, hx_lx = tx == 0 ? 0 : DW_TX + 1;
  const bool hx_ok = hx && hx_i < NX && iny;
  const bool hy = ty == 0 || ty == DW_TY - 1;
  const int hy_j = ty == 0 ? gj - 1 : gj + 1, hy_ly = ty == 0 ? 0 : DW_TY + 1;
  const bool hy_ok = hy && hy_j < NY && inx;
  const double* pc = u + gi + gj * sy;
  const double* px = u + hx_i + gj * sy;
  const double* py = u + gi + (i64)hy_j * sy;
  const bool ld_c = inx && iny;
  // column queue: doubles (for the fallback) and their splits
  double q[3];
  dw cq[3];
  bool okq[3];
#pragma unroll
  for (int m = 0; m < 3; m++) {
    q[m] = ld_c ? pc[(i64)(k0 - 1 + m) * sz] : 0.0;
    okq[m] = split(q[m], cq[m]);
  }
  double hxv = hx_ok ? px[(i64)k0 * sz] : 0.0, hyv = hy_ok ? py[(i64)k0 * sz] : 0.0;
  for (int k = k0; k < k1; k++) {
    const bool more = k + 1 < k1;
    double qn = 0.0, hxn = 0.0, hyn = 0.0;
    if (more) {
      if (ld_c) qn = pc[(i64)(k + 2) * sz];
      if (hx_ok) hxn = px[(i64)(k + 1) * sz];
      if (hy_ok) hyn = py[(i64)(k + 1) * sz];
    }
    const dw cm = cq[0], cc = cq[1], cp = cq[2];
    const bool okm = okq[0], okc = okq[1], okp = okq[2];
    __syncthreads();
    tile[ty + 1][tx + 1] = make_float2(cc.h, cc.l);
    bad[ty + 1][tx + 1] = okc ? 0 : 1;
    if (hx) {
      dw v;
      const bool ok = split(hxv, v);
      tile[ty + 1][hx_lx] = make_float2(v.h, v.l);
      bad[ty + 1][hx_lx] = ok ? 0 : 1;
    }
    if (hy) {
      dw v;
      const bool ok = split(hyv, v);
      tile[hy_ly][tx + 1] = make_float2(v.h, v.l);
      bad[hy_ly][tx + 1] = ok ? 0 : 1;
    }
    __syncthreads();
    if (active) {
      const bool any_bad = !okm || !okp || bad[ty + 1][tx] || bad[ty + 1][tx + 2] || bad[ty][tx + 1] ||
                           bad[ty + 2][tx + 1];
      double res;
      if (!any_bad) {
        const float2 xm = tile[ty + 1][tx], xp = tile[ty + 1][tx + 2];
        const float2 ym = tile[ty][tx + 1], yp = tile[ty + 2][tx + 1];
        const dw sx = add(dw{xm.x, xm.y}, dw{xp.x, xp.y});
        const dw syy = add(dw{ym.x, ym.y}, dw{yp.x, yp.y});
        const dw szz = add(cm, cp);
        const dw s = add(add(sx, syy), szz);
        const dw r = mul(c1, s);
        res = __dadd_rn(widen(r.h), widen(r.l));
      } else {
        // outside the split's range: the canonical double update
        const double* p = u + gi + gj * sy + (i64)k * sz;
        const double s = A::add(A::add(A::add(p[-1], p[1]), A::add(p[-sy], p[sy])), A::add(q[0], q[2]));
        res = A::mul(c1d, s);
      }
      out[gi + gj * sy + (i64)k * sz] = res;
    }
    q[0] = q[1];
    q[1] = q[2];
    q[2] = qn;
    cq[0] = cq[1];
    cq[1] = cq[2];
    okq[0] = okq[1];
    okq[1] = okq[2];
    okq[2] = split(qn, cq[2]);
    hxv = hxn;
    hyv = hyn;
  }
}

}  // namespace

static std::atomic<int> g_double_word{0};
int tune_set_double_word(int v) {
  if (v < 0 || v > 1) return STN_EINVAL;
  g_double_word = v;
  return STN_OK;
}
int tune_get_double_word() { return g_double_word.load(); }

bool dw_applicable(const Grid& g, const double* coeffs, const void* b) {
  return g.r == 1 && b == nullptr && coeffs[0] == 0.0 && (i64)(DW_TY + 2) * g.NX() < ((i64)1 << 40);
}

int launch_star_dw(const double* u, double* out, const Grid& g, const double* coeffs, cudaStream_t s) {
  const int tiles_x = (int)((g.nx + DW_TX - 1) / DW_TX), tiles_y = (int)((g.ny + DW_TY - 1) / DW_TY);
  // about eight waves of 8 resident blocks per SM, chunks of at least 8 planes
  const i64 tiles = (i64)tiles_x * tiles_y;
  i64 chunks = (8 * 8 * (i64)device_sms() + tiles - 1) / tiles;
  const i64 maxc = (g.nz + 7) / 8;
  if (chunks > maxc) chunks = maxc;
  if (chunks < 1) chunks = 1;
  const int kchunk = (int)((g.nz + chunks - 1) / chunks);
  const int nchunks = (int)((g.nz + kchunk - 1) / kchunk);
  if (int rc = check_launch_grid(tiles_x, tiles_y, nchunks)) return rc;
  const double c = coeffs[1];
  dw c1;
  c1.h = (float)c;
  c1.l = (float)(c - (double)c1.h);
  star_dw_kernel<<<dim3(tiles_x, tiles_y, nchunks), dim3(DW_TX, DW_TY), 0, s>>>(
      u, out, (int)g.nx, (int)g.ny, (int)g.nz, (int)g.NX(), (int)g.NY(), kchunk, c1, c);
  STN_CUDA_TRY(cudaGetLastError());
  return STN_OK;
}

}  // namespace stn
