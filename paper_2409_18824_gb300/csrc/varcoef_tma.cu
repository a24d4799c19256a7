// Variable-coefficient float sweep, radius 2, with TMA-staged halo tiles.
//
// The same Jacobi update as varcoef.cu (the symmetric operator
//   (A u)(p) = sum_d w_d sum_{q = p +- d e_axis} kappa(p,q) (u(p) - u(q)),
// kappa = (a(p) + a(q)) / 2, u'(p) = (f(p) + N(p)) / D(p); the paper states
// only Laplace's equation, Sec. 4, and this operator is the reading used for
// the variable-coefficient workload), computed in the same order, operation
// by operation, so its results are bitwise those of the column kernel and of
// the CPU oracle.
//
// Layout of the work:
//   * a block owns a tile of VT_TW x VT_TH interior (i, j) columns and streams
//     a chunk of k planes through a ring of VT_S shared-memory stages;
//   * a producer warp (one lane) issues, per plane, three tiled bulk tensor
//     copies (cp.async.bulk.tensor.3d) of the tile plus its radius-2 halo, of
//     u, a and f, completing on the stage's "full" mbarrier; consumer warps
//     wait on it themselves and each releases the stage with one arrive on
//     its "empty" mbarrier, which the producer waits on before refilling it,
//     so no block-wide barrier separates the planes.  The tensor maps
//     describe the padded Fortran grid directly (rows of NX elements), which
//     needs NX * 4 bytes to be a multiple of 16; the box starts R columns
//     left of the tile, i.e. at a multiple of 64 elements, so every copy
//     starts on a 16-byte boundary.  Halo cells past the grid's end read as
//     zero and are never used for a stored point;
//   * a thread computes 2 consecutive i of 2 consecutive j (8-byte shared
//     loads; interior column pairs start at even padded indices when R = 2).
//     The k neighbours of its four points come from a register queue of
//     planes k-2 .. k+2 of u and a, filled from the stage of plane k+2 as it
//     arrives; the in-plane neighbours come from the stage of plane k.  The
//     loop is unrolled by the queue length, so the queue rotates by renaming;
//   * x and y faces are computed once per face for the thread's points (a
//     face between two of its points serves both); z faces per point.
//   * f is read from the stage; the result is stored with plain 8-byte global
//     stores.
// Every wait on an mbarrier is bounded: after about two seconds (or once
// another thread of the block gave up) the thread records kVarTmaTimeout in a
// status word the host reads and stops; the producer then waits (again
// bounded) for its copies in flight and the block returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <mutex>

#include "arith.cuh"
#include "internal.h"

namespace stn {

namespace {

constexpr int VT_R = 2;
constexpr int VT_TW = 64;   // interior columns per block (32 lanes x 2)
constexpr int VT_TH = 16;   // interior rows per block (8 consumer warps x 2)
constexpr int VT_CWARPS = 8;                       // consumer warps
constexpr int VT_THREADS = 32 * (VT_CWARPS + 1);   // plus one producer warp
constexpr int VT_S = 6;     // ring stages
constexpr int VT_Q = 2 * VT_R + 1;          // register queue: planes k-2 .. k+2
constexpr int VT_PW = VT_TW + 2 * VT_R;     // box width (68 floats = 272 bytes)
constexpr int VT_PH = VT_TH + 2 * VT_R;     // box height
constexpr int VT_BOX = VT_PW * VT_PH;       // floats one copy writes
constexpr int VT_FIELD = (VT_BOX + 31) & ~31;  // a field's box, rounded to 128 bytes
constexpr int VT_STAGE = 3 * VT_FIELD;      // u, a, f
constexpr int VT_SMEM = VT_S * VT_STAGE * 4;
constexpr int VT_SMEM_ALLOC = VT_SMEM + 128;  // slack to start the ring on a 128-byte boundary
constexpr unsigned VT_TX_BYTES = 3u * VT_BOX * 4u;  // bytes each stage's full barrier expects
constexpr unsigned long long VT_WAIT_NS = 2000000000ull;
constexpr int kVarTmaTimeout = 1;

__device__ int g_var_tma_status;  // 0, or kVarTmaTimeout once a wait ran out

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for one phase of the barrier; false when it ran out, or when
// another thread of the block has given up (*abort set).
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, const volatile int* abort) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (!mbar_try(bar, parity))
    if (*abort || gtimer() - t0 > VT_WAIT_NS) return false;
  return true;
}

__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }

// One tiled bulk tensor copy of a (VT_PW x VT_PH x 1) box at (x, y, z) into
// shared memory at dst, completing on the mbarrier at bar.
__device__ __forceinline__ void tma_load(unsigned dst, const CUtensorMap* map, int x, int y, int z, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

struct VtW {
  float h1, h2;  // w_d / 2 (exact halving)
};

// Stage s holds plane p = pfirst + s + VT_S * use: boxes of u, a and f.
// full[s] completes when the copies of a plane have landed (the producer
// arrives once with the expected bytes); empty[s] completes when every
// consumer warp has read the plane for the last time (one arrive per warp),
// after which the producer refills the stage.  Phase parity of use n is n & 1.
__global__ void __launch_bounds__(VT_THREADS, 2)
    var_tma_kernel(const __grid_constant__ CUtensorMap tmu, const __grid_constant__ CUtensorMap tma,
                   const __grid_constant__ CUtensorMap tmf, float* __restrict__ out, int nx, int ny, int nz,
                   int NX, int NY, int kchunk, VtW hw) {
  using A = Arith<float>;
  constexpr int R = VT_R;
  extern __shared__ __align__(16) unsigned char vt_dyn[];
  __shared__ __align__(8) unsigned long long full[VT_S], empty[VT_S];
  __shared__ int abort_flag;
  // the ring starts on a 128-byte boundary (the launch adds 128 bytes of slack)
  float* const vt_ring = reinterpret_cast<float*>(
      vt_dyn + ((128u - ((unsigned)__cvta_generic_to_shared(vt_dyn) & 127u)) & 127u));
  const int tid = threadIdx.x, lx = tid & 31, wid = tid >> 5;
  const int tx0 = blockIdx.x * VT_TW, ty0 = blockIdx.y * VT_TH;  // tile origin (interior offsets)
  const int k0 = R + blockIdx.z * kchunk;
  const int k1 = min(k0 + kchunk, nz + R);
  const int pfirst = k0 - R, plast = k1 - 1 + R;
  const unsigned ring_s = (unsigned)__cvta_generic_to_shared(vt_ring);
  const unsigned full_s = (unsigned)__cvta_generic_to_shared(full);
  const unsigned empty_s = (unsigned)__cvta_generic_to_shared(empty);
  if (tid == 0) {
    for (int s = 0; s < VT_S; s++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full_s + 8u * s) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(empty_s + 8u * s), "r"(VT_CWARPS) : "memory");
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  const volatile int* abortp = &abort_flag;
  auto give_up = [&]() {
    abort_flag = 1;
    atomicExch(&g_var_tma_status, kVarTmaTimeout);
  };

  if (wid == VT_CWARPS) {
    // ---- producer warp: one lane issues every plane's copies in order ------
    if (lx == 0) {
      int p = pfirst;
      for (; p <= plast; p++) {
        const int s = (p - pfirst) % VT_S, use = (p - pfirst) / VT_S;
        if (use > 0 && !mbar_wait(empty_s + 8u * s, (unsigned)((use - 1) & 1), abortp)) {
          give_up();
          break;
        }
        const unsigned bar = full_s + 8u * s;
        const unsigned dst = ring_s + (unsigned)(s * VT_STAGE * 4);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(VT_TX_BYTES)
                     : "memory");
        tma_load(dst, &tmu, tx0, ty0, p, bar);
        tma_load(dst + VT_FIELD * 4u, &tma, tx0, ty0, p, bar);
        tma_load(dst + 2u * VT_FIELD * 4u, &tmf, tx0, ty0, p, bar);
      }
      // leave no copy in flight: wait (bounded) for the last VT_S planes issued
      for (int q = max(pfirst, p - VT_S); q < p; q++) {
        const int s = (q - pfirst) % VT_S;
        (void)mbar_wait(full_s + 8u * s, (unsigned)(((q - pfirst) / VT_S) & 1), abortp);
      }
    }
    return;
  }

  // ---- consumer warps ---------------------------------------------------------
  const int ly = wid;
  const int c = 2 * lx + R, rr = 2 * ly + R;  // box column / row of the thread's first point
  const int gi = tx0 + c, gj = ty0 + rr;
  const bool col0 = gi < nx + R, col1 = gi + 1 < nx + R;
  const bool row0 = gj < ny + R, row1 = gj + 1 < ny + R;
  const i64 psz = (i64)NX * NY;
  float* ob = out + (i64)gj * NX + gi;

  auto stage_u = [&](int p) -> const float* { return vt_ring + ((p - pfirst) % VT_S) * VT_STAGE; };
  // every lane waits; the answer is the warp's (all lanes go on or none)
  auto wait_full = [&](int p) -> bool {
    const int s = (p - pfirst) % VT_S;
    const bool ok = mbar_wait(full_s + 8u * s, (unsigned)(((p - pfirst) / VT_S) & 1), abortp);
    return __all_sync(0xffffffffu, ok);
  };
  auto release = [&](int p) {  // this warp has read plane p for the last time
    __syncwarp();
    if (lx == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(empty_s + 8u * ((p - pfirst) % VT_S)) : "memory");
  };

  // queue: planes by slot (p - pfirst) % VT_Q, rows 0 / 1, columns in .x / .y
  float2 qu[VT_Q][2], qa[VT_Q][2];
  auto fill = [&](int slot, int p) {
    const float* su = stage_u(p);
    const float* sa = su + VT_FIELD;
#pragma unroll
    for (int t = 0; t < 2; t++) {
      qu[slot][t] = ld2(su + (rr + t) * VT_PW + c);
      qa[slot][t] = ld2(sa + (rr + t) * VT_PW + c);
    }
  };

  // prologue: planes k0 - 2 .. k0 + 1 into the queue (k0 - 2 and k0 - 1 are
  // not read again)
  bool stop = false;
#pragma unroll
  for (int m = 0; m < 2 * R; m++) {
    if (!stop && !wait_full(pfirst + m)) {
      give_up();
      stop = true;
    }
    if (!stop) fill(m, pfirst + m);
  }
  if (!stop) {
    release(pfirst);
    release(pfirst + 1);
  }

  for (int kb = k0; kb < k1 && !stop; kb += VT_Q) {
#pragma unroll
    for (int J = 0; J < VT_Q; J++) {
      const int k = kb + J;
      if (k >= k1) break;
      if (!wait_full(k + R)) {
        give_up();
        stop = true;
        break;
      }
      // slots of planes k + d: (k - pfirst + d) % VT_Q = (J + R + d) % VT_Q,
      // since k - pfirst = (kb - k0) + J + R and kb - k0 is a multiple of VT_Q
      fill((J + 2 * R) % VT_Q, k + R);
      const float* su = stage_u(k);
      const float* sa = su + VT_FIELD;
      const float* sf = sa + VT_FIELD;
      // in-plane values: X[t][0..5] = columns c-2 .. c+3 of own row t,
      // Y[q][0..5] = rows rr-2 .. rr+3 of own column q
      float XU[2][6], XA[2][6], YU[2][6], YA[2][6];
      float2 fq[2];
#pragma unroll
      for (int t = 0; t < 2; t++) {
        const float2 l = ld2(su + (rr + t) * VT_PW + c - 2), r = ld2(su + (rr + t) * VT_PW + c + 2);
        const float2 la = ld2(sa + (rr + t) * VT_PW + c - 2), ra = ld2(sa + (rr + t) * VT_PW + c + 2);
        fq[t] = ld2(sf + (rr + t) * VT_PW + c);
        const float2 cu = qu[(J + R) % VT_Q][t], ca = qa[(J + R) % VT_Q][t];
        XU[t][0] = l.x; XU[t][1] = l.y; XU[t][2] = cu.x; XU[t][3] = cu.y; XU[t][4] = r.x; XU[t][5] = r.y;
        XA[t][0] = la.x; XA[t][1] = la.y; XA[t][2] = ca.x; XA[t][3] = ca.y; XA[t][4] = ra.x; XA[t][5] = ra.y;
      }
      {
        const int rows[4] = {rr - 2, rr - 1, rr + 2, rr + 3};
        const int at[4] = {0, 1, 4, 5};
#pragma unroll
        for (int m = 0; m < 4; m++) {
          const float2 vu = ld2(su + rows[m] * VT_PW + c), va = ld2(sa + rows[m] * VT_PW + c);
          YU[0][at[m]] = vu.x; YU[1][at[m]] = vu.y;
          YA[0][at[m]] = va.x; YA[1][at[m]] = va.y;
        }
#pragma unroll
        for (int q = 0; q < 2; q++) {
          YU[q][2] = XU[0][2 + q]; YU[q][3] = XU[1][2 + q];
          YA[q][2] = XA[0][2 + q]; YA[q][3] = XA[1][2 + q];
        }
      }
      release(k);  // plane k's stage is no longer read by this warp
      // faces along a line of six values v[0..5] (own points at 2, 3):
      // F1[m] = face (m+1, m+2) for d = 1, m = 0..2; F2[m] = face (m, m+2) for d = 2, m = 0..3
      float FX1[2][3], FX2[2][4], FY1[2][3], FY2[2][4];
#pragma unroll
      for (int t = 0; t < 2; t++) {
#pragma unroll
        for (int m = 0; m < 3; m++) FX1[t][m] = A::mul(hw.h1, A::add(XA[t][m + 1], XA[t][m + 2]));
#pragma unroll
        for (int m = 0; m < 4; m++) FX2[t][m] = A::mul(hw.h2, A::add(XA[t][m], XA[t][m + 2]));
      }
#pragma unroll
      for (int q = 0; q < 2; q++) {
#pragma unroll
        for (int m = 0; m < 3; m++) FY1[q][m] = A::mul(hw.h1, A::add(YA[q][m + 1], YA[q][m + 2]));
#pragma unroll
        for (int m = 0; m < 4; m++) FY2[q][m] = A::mul(hw.h2, A::add(YA[q][m], YA[q][m + 2]));
      }
      float res[2][2];
#pragma unroll
      for (int t = 0; t < 2; t++) {
#pragma unroll
        for (int q = 0; q < 2; q++) {
          // point (column q, row t): position 2+q in its row's line, 2+t in its column's line
          const float ap = XA[t][2 + q];
          float D = 0.f, N = 0.f;
#pragma unroll
          for (int d = 1; d <= R; d++) {
            const float h = d == 1 ? hw.h1 : hw.h2;
            // x: minus face (2+q-d, 2+q), plus face (2+q, 2+q+d)
            const float txm = d == 1 ? FX1[t][q] : FX2[t][q];
            const float txp = d == 1 ? FX1[t][q + 1] : FX2[t][q + 2];
            const float tym = d == 1 ? FY1[q][t] : FY2[q][t];
            const float typ = d == 1 ? FY1[q][t + 1] : FY2[q][t + 2];
            const float2 am = qa[(J + R - d) % VT_Q][t], apl = qa[(J + R + d) % VT_Q][t];
            const float2 um = qu[(J + R - d) % VT_Q][t], upl = qu[(J + R + d) % VT_Q][t];
            // z faces per point (carrying plus faces to the next planes costs
            // registers that halve the blocks per SM)
            const float tzm = A::mul(h, A::add(ap, q == 0 ? am.x : am.y));
            const float tzp = A::mul(h, A::add(ap, q == 0 ? apl.x : apl.y));
            D = A::add(D, txm);
            N = A::add(N, A::mul(txm, XU[t][2 + q - d]));
            D = A::add(D, txp);
            N = A::add(N, A::mul(txp, XU[t][2 + q + d]));
            D = A::add(D, tym);
            N = A::add(N, A::mul(tym, YU[q][2 + t - d]));
            D = A::add(D, typ);
            N = A::add(N, A::mul(typ, YU[q][2 + t + d]));
            D = A::add(D, tzm);
            N = A::add(N, A::mul(tzm, q == 0 ? um.x : um.y));
            D = A::add(D, tzp);
            N = A::add(N, A::mul(tzp, q == 0 ? upl.x : upl.y));
          }
          const float fv = q == 0 ? fq[t].x : fq[t].y;
          res[t][q] = A::div(A::add(fv, N), D);
        }
      }
      const i64 po = (i64)k * psz;
#pragma unroll
      for (int t = 0; t < 2; t++) {
        const bool rowok = t == 0 ? row0 : row1;
        if (rowok && col1)
          *reinterpret_cast<float2*>(ob + po + t * NX) = make_float2(res[t][0], res[t][1]);
        else if (rowok && col0)
          ob[po + t * NX] = res[t][0];
      }
    }
  }
}

// ---- host side ------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      (void)cudaGetLastError();
  });
  return fn;
}

int encode(CUtensorMap* m, const float* base, const Grid& g) {
  auto fn = encoder();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return STN_ECUDA;
  }
  const cuuint64_t dims[3] = {(cuuint64_t)g.NX(), (cuuint64_t)g.NY(), (cuuint64_t)g.NZ()};
  const cuuint64_t strides[2] = {(cuuint64_t)g.NX() * 4, (cuuint64_t)(g.NX() * g.NY()) * 4};
  const cuuint32_t box[3] = {VT_PW, VT_PH, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return STN_ECUDA;
  }
  return STN_OK;
}

int vt_resident() {
  static std::atomic<int> cache{0};
  const int known = cache.load(std::memory_order_relaxed);
  if (known > 0) return known;
  int v = 0;
  cudaError_t e = cudaFuncSetAttribute(var_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, VT_SMEM_ALLOC);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, var_tma_kernel, VT_THREADS, VT_SMEM_ALLOC);
  if (e != cudaSuccess || v < 1) {
    (void)cudaGetLastError();
    return 2;  // no device (planning only): the design point
  }
  cache.store(v, std::memory_order_relaxed);
  return v;
}

}  // namespace

bool var_tma_applicable(const Grid& g, size_t esize, const void* u, const void* a, const void* f,
                        const void* out) {
  if (esize != 4 || g.r != VT_R) return false;
  if ((g.NX() * 4) % 16 != 0) return false;  // tensor-map row pitch: a multiple of 16 bytes
  if (g.NX() > ((i64)1 << 31) || g.NY() > ((i64)1 << 31) || g.NZ() > ((i64)1 << 31)) return false;
  if ((i64)g.NX() * g.NY() * 4 >= ((i64)1 << 40)) return false;  // plane stride limit of a tensor map
  auto al = [](const void* p, uintptr_t m) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & (m - 1)) == 0; };
  return al(u, 16) && al(a, 16) && al(f, 16) && al(out, 8);
}

ZPlan plan_var_tma(const Grid& g) {
  ZPlan p;
  p.variant = 2;
  p.tiles_x = (int)((g.nx + VT_TW - 1) / VT_TW);
  p.tiles_y = (int)((g.ny + VT_TH - 1) / VT_TH);
  const i64 tiles = (i64)p.tiles_x * p.tiles_y;
  const i64 slots = (i64)device_sms() * vt_resident();
  // about twelve waves of blocks, chunks of at least 16 planes (a knob may set
  // the chunk count).  Measured at 768 x 768 x 384 (576 tiles, 304 slots),
  // GLUP/s for 2 / 3 / 4 / 6 / 8 / 12 / 16 / 24 chunks: 290 / 291 / 292 / 301 /
  // 301 / 300 / 296 / 286
  i64 chunks = (12 * slots + tiles / 2) / tiles;
  if (const int kc = tune_get_var_chunks(); kc > 0) chunks = kc;
  const i64 max_chunks = (g.nz + 15) / 16;
  if (chunks > max_chunks) chunks = max_chunks;
  if (chunks < 1) chunks = 1;
  p.kchunk = (int)((g.nz + chunks - 1) / chunks);
  p.chunks = (int)((g.nz + p.kchunk - 1) / p.kchunk);
  p.rg = VT_TH;
  p.smem = VT_SMEM_ALLOC;
  return p;
}

int launch_var_tma(const float* u, const float* a, const float* f, float* out, const Grid& g, const double* w,
                   cudaStream_t s) {
  const ZPlan p = plan_var_tma(g);
  if (int rc = check_launch_grid(p.tiles_x, p.tiles_y, p.chunks)) return rc;
  CUtensorMap mu, ma, mf;
  if (int rc = encode(&mu, u, g)) return rc;
  if (int rc = encode(&ma, a, g)) return rc;
  if (int rc = encode(&mf, f, g)) return rc;
  static std::atomic<bool> attr_set[64];
  int dev = 0;
  STN_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64 || !attr_set[dev].load(std::memory_order_relaxed)) {
    STN_CUDA_TRY(cudaFuncSetAttribute(var_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, VT_SMEM_ALLOC));
    if (dev >= 0 && dev < 64) attr_set[dev].store(true, std::memory_order_relaxed);
  }
  VtW hw{(float)(0.5 * w[1]), (float)(0.5 * w[2])};
  dim3 grid(p.tiles_x, p.tiles_y, p.chunks);
  var_tma_kernel<<<grid, VT_THREADS, VT_SMEM_ALLOC, s>>>(mu, ma, mf, out, (int)g.nx, (int)g.ny, (int)g.nz,
                                                         (int)g.NX(), (int)g.NY(), p.kchunk, hw);
  STN_CUDA_TRY(cudaGetLastError());
  return STN_OK;
}

int var_tma_status(bool clear, int* status) {
  int v = 0;
  STN_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_var_tma_status, sizeof(int)));
  if (clear && v != 0) {
    const int zero = 0;
    STN_CUDA_TRY(cudaMemcpyToSymbol(g_var_tma_status, &zero, sizeof(int)));
  }
  *status = v;
  return STN_OK;
}

}  // namespace stn
