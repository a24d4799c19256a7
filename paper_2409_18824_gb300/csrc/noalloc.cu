// residual_norm_f64_noalloc: the residual norm without any allocation.
//
// Some callers cannot let a library allocate device memory: a serving process
// that has already handed its whole HBM budget to its own pools, code that
// must not call cudaMalloc because cudaMalloc can synchronise the device and
// stall every other stream of the process, and hosts embedding the library
// in a loop where an allocation failure has no way to be reported.  For them
// this entry point keeps its scratch (the per-block partial sums of the
// reduction and the result slots) in a fixed array in the library's own
// device image, so the only memory it touches is that array and the caller's
// grids.
//
// The array is file-scope device memory: every GPU that loads libstencil.so
// holds it until the process exits, and every call on that GPU shares it.
// Calls that overlap on the GPU (different streams, or different host
// threads) therefore race on it; callers must order them.  Nothing here
// accumulates across calls: each call's reduction kernel writes every partial
// slot it later reads, and the finalising kernel writes the result slots, so
// no slot needs clearing between calls.
#include <mutex>

#include "internal.h"

namespace stn {

namespace {

// Maximum number of per-block partial sums (one per block of the residual
// kernel's launch plan): 65536 doubles = 512 KiB, plus 8 result slots.
constexpr i64 kNoAllocPartials = 65536;
constexpr int kNoAllocSlots = 8;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocPartials + kNoAllocSlots];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device.  The symbol's
// name in host code is only a host-side handle, never a device address, so
// the address is looked up once per device with that device current.
int scratch_address(double** out) {
  int dev = 0;
  STN_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal out of range for the no-allocation scratch");
    return STN_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_addr[dev] = (double*)p;
  }
  *out = g_addr[dev];
  return STN_OK;
}

}  // namespace

static int noalloc_residual(const double* u, const double* b, i64 nx, i64 ny, i64 nz,
                            const double* coeffs, int radius, double* norm_out, void* stream) {
  clear_error();
  if (!u) {
    set_error("invalid argument: NULL grid");
    return STN_EINVAL;
  }
  if (!coeffs || !norm_out) {
    set_error("invalid argument: NULL coeffs or norm_out");
    return STN_EINVAL;
  }
  if (radius != 1 && radius != 2) {
    set_error("invalid argument: radius must be 1 or 2");
    return STN_EINVAL;
  }
  if (nx < 1 || ny < 1 || nz < 1 || nx > (1 << 28) || ny > (1 << 28) || nz > (1 << 28)) {
    set_error("invalid argument: interior extents must be in [1, 2^28]");
    return STN_EINVAL;
  }
  const Grid g{nx, ny, nz, radius};
  // A first look at the plan, to refuse oversize grids before any CUDA call;
  // launch_star checks the plan it actually launches against the same limit.
  if (star_blocks(g, sizeof(double), u, b, nullptr) > kNoAllocPartials) {
    set_error("invalid argument: grid needs more than 65536 partial sums, the size of the "
              "no-allocation scratch (use residual_norm_f64)");
    return STN_EINVAL;
  }
  cudaPointerAttributes at;
  for (const void* q : {(const void*)u, (const void*)b}) {
    if (!q) continue;
    STN_CUDA_TRY(cudaPointerGetAttributes(&at, q));
    if (!(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)) {
      set_error("invalid argument: residual_norm_f64_noalloc takes device grids only");
      return STN_EINVAL;
    }
  }
  double* scratch = nullptr;
  if (int rc = scratch_address(&scratch)) return rc;
  double* partials = scratch;
  double* slots = scratch + kNoAllocPartials;
  cudaStream_t s = (cudaStream_t)stream;
  // The plan is formed once inside launch_star: the partial count it checks
  // against the array, the grid it launches and the count `nb` reduced below
  // are the same, whatever another host thread does to the tuning knobs or
  // the tuning cache meanwhile.
  i64 nb = 0;
  if (int rc = launch_star<double>(u, b, nullptr, g, coeffs, kResidualOnly, partials, s,
                                   kNoAllocPartials, &nb))
    return rc;
  if (int rc = launch_finalize(partials, nb, slots, nullptr, 0.0, s)) return rc;
  STN_CUDA_TRY(cudaMemcpyAsync(norm_out, slots + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  STN_CUDA_TRY(cudaStreamSynchronize(s));
  return STN_OK;
}

}  // namespace stn

extern "C" int residual_norm_f64_noalloc(const double* u, const double* b, int64_t nx, int64_t ny,
                                         int64_t nz, const double* coeffs, int radius,
                                         double* norm_out, void* stream) {
  return stn::noalloc_residual(u, b, nx, ny, nz, coeffs, radius, norm_out, stream);
}
