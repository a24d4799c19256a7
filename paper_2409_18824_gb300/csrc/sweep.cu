// Host-side planning of the star-stencil kernels (star.cuh) and the tuning
// override; the kernels themselves are instantiated per element type in
// sweep_f64.cu and sweep_f32.cu so that the two compile in parallel.
#include <atomic>

#include "star.cuh"

namespace stn {

// Process-wide knobs, read by planners on any host thread: atomic, so a
// concurrent set is seen whole (each launch forms its plan once).
static std::atomic<int> g_star_variant_override{-1};

int tune_set_star_variant(int v) {
  if (v < -1 || v > 3) return STN_EINVAL;
  g_star_variant_override = v;
  return STN_OK;
}
int tune_get_star_variant() { return g_star_variant_override; }

static std::atomic<int> g_temporal_depth{0};
int tune_set_temporal_depth(int d) {
  if (d < 0 || d > 4) return STN_EINVAL;
  g_temporal_depth = d;
  return STN_OK;
}
int tune_get_temporal_depth() { return g_temporal_depth; }

static std::atomic<int> g_star_chunks{0};
int tune_set_star_chunks(int c) {
  if (c < 0 || c > 65535) return STN_EINVAL;
  g_star_chunks = c;
  return STN_OK;
}
int tune_get_star_chunks() { return g_star_chunks; }

StarChoice& star_force() {
  static thread_local StarChoice f;
  return f;
}

StarChoice& star_last() {
  static thread_local StarChoice f;
  return f;
}

int device_sms() {
  static std::atomic<int> cache[64];  // per device ordinal, 0 = not queried yet
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    (void)cudaGetLastError();
    return 152;
  }
  const int known = cache[dev].load(std::memory_order_relaxed);
  if (known > 0) return known;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
    (void)cudaGetLastError();
    return 152;
  }
  cache[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

template <typename K>
static int occupancy(K kernel, int threads) {
  int v = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, threads, 0) != cudaSuccess || v < 1) {
    (void)cudaGetLastError();
    v = 4;  // no device (planning only): a fixed estimate
  }
  return v;
}

// Blocks of a star kernel resident per SM, queried once per (variant, element
// type, radius) on the sweep instance; every mode uses the same plan.
static int star_resident(int variant, size_t esize, int r) {
  static std::atomic<int> cache[3][2][3];  // 0 = not queried yet
  std::atomic<int>& slot = cache[variant][esize == 8 ? 1 : 0][r];
  const int known = slot.load(std::memory_order_relaxed);
  if (known != 0) return known;
  int c = 0;
  const int tc = 32 * SC_WARPS, tp = TX * TY;
  if (esize == 8) {
    if (variant == kStarColumn)
      c = r == 1 ? occupancy(star_col_kernel<double, 1, false, false, kSweep, SC_TJ, ColPF<double>::value>, tc)
                 : occupancy(star_col_kernel<double, 2, false, false, kSweep, SC_TJ, ColPF<double>::value>, tc);
    else if (variant == kStarPlane2)
      c = r == 1 ? occupancy(star2_kernel<double, 1, false, false, kSweep>, tp)
                 : occupancy(star2_kernel<double, 2, false, false, kSweep>, tp);
    else
      c = r == 1 ? occupancy(star_kernel<double, 1, false, false, kSweep>, tp)
                 : occupancy(star_kernel<double, 2, false, false, kSweep>, tp);
  } else {
    if (variant == kStarColumn)
      c = r == 1 ? occupancy(star_col_kernel<float, 1, false, false, kSweep, SC_TJ, ColPF<float>::value>, tc)
                 : occupancy(star_col_kernel<float, 2, false, false, kSweep, SC_TJ, ColPF<float>::value>, tc);
    else if (variant == kStarPlane2)
      c = r == 1 ? occupancy(star2_kernel<float, 1, false, false, kSweep>, tp)
                 : occupancy(star2_kernel<float, 2, false, false, kSweep>, tp);
    else
      c = r == 1 ? occupancy(star_kernel<float, 1, false, false, kSweep>, tp)
                 : occupancy(star_kernel<float, 2, false, false, kSweep>, tp);
  }
  slot.store(c, std::memory_order_relaxed);
  return c;
}

// Ring layout of the staged kernel for this grid: rows per block so that the
// SG_PF + 2R + 1 stages fit kStagedSmemMax (at most 64 rows); false when even
// one row does not fit.
static bool staged_layout(const Grid& g, size_t esize, int* rg, int* stage_elems, int* smem) {
  const int S = 2 * g.r + 1 + SG_PF;
  const i64 row_bytes = g.NX() * (i64)esize;
  const i64 stage_max = (kStagedSmemMax / S) & ~(i64)15;
  i64 rows = (stage_max - 32) / row_bytes - 2 * g.r;
  if (rows < 1) return false;
  if (rows > 64) rows = 64;
  if (rows > g.ny) rows = g.ny;
  const i64 stage_bytes = ((rows + 2 * g.r) * row_bytes + 32 + 15) & ~(i64)15;
  *rg = (int)rows;
  *stage_elems = (int)(stage_bytes / (i64)esize);
  *smem = (int)(stage_bytes * S);
  return true;
}

bool staged_applicable(const Grid& g, size_t esize) {
  int a, b, c;
  return staged_layout(g, esize, &a, &b, &c);
}

// Rows per staged block for this grid (0 when the ring does not fit).
static int staged_rows(const Grid& g, size_t esize) {
  int rg = 0, b, c;
  return staged_layout(g, esize, &rg, &b, &c) ? rg : 0;
}

// Blocks of the staged kernel resident per SM with `smem` bytes of ring.
static int staged_resident(size_t esize, int r, int smem) {
  // last query per (type, radius): (smem << 32) | blocks, 0 = none yet
  static std::atomic<unsigned long long> cache[2][3];
  const int e = esize == 8 ? 1 : 0;
  const unsigned long long known = cache[e][r].load(std::memory_order_relaxed);
  if (known != 0 && (int)(known >> 32) == smem) return (int)(known & 0xffffffffu);
  int v = 0;
  auto query = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kStagedSmemMax);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, 32 * SG_WARPS, smem);
    return e;
  };
  cudaError_t err;
  if (esize == 8)
    err = r == 1 ? query(star_staged_kernel<double, 1, false, false, kSweep>)
                 : query(star_staged_kernel<double, 2, false, false, kSweep>);
  else
    err = r == 1 ? query(star_staged_kernel<float, 1, false, false, kSweep>)
                 : query(star_staged_kernel<float, 2, false, false, kSweep>);
  if (err != cudaSuccess || v < 1) {
    (void)cudaGetLastError();
    return 2;  // no device (planning only): the design point
  }
  cache[e][r].store(((unsigned long long)(unsigned)smem << 32) | (unsigned)v, std::memory_order_relaxed);
  return v;
}

ZPlan plan_star(const Grid& g, int variant, size_t esize) {
  ZPlan p;
  const i64 max_chunks = (g.nz + 3) / 4;  // chunks of >= 4 planes
  i64 chunks;
  if (variant == kStarStaged && !staged_layout(g, esize, &p.rg, &p.stage_elems, &p.smem)) variant = kStarScalar;
  if (variant == kStarStaged) {
    // whole rows per block, one block per SM.  At most one wave: a partial
    // second wave of these long blocks nearly doubles the time (512^3 float,
    // 21 row groups: 7 chunks = 147 blocks 704 GLUP/s, 8 chunks = 168 blocks
    // 417).  When one wave leaves more than a quarter of the SMs idle (many
    // row groups), many short chunks instead: at least 8 waves, so the tail
    // is short (768 x 768 x 384 radius 2: 277 GLUP/s in 120 blocks, 401 in
    // 1560).
    p.tiles_x = 1;
    p.tiles_y = (int)((g.ny + p.rg - 1) / p.rg);
    const i64 slots = (i64)device_sms() * staged_resident(esize, g.r, p.smem);
    const i64 tiles = p.tiles_y;
    chunks = slots / tiles;
    if (chunks < 1 || 4 * chunks * tiles < 3 * slots) chunks = (8 * slots + tiles - 1) / tiles;
  } else if (variant == kStarColumn) {
    // one wave at most: k chunks = resident slots / tiles (measured: a partial
    // wave beats 1.2-1.9 waves by 15-20 % on this memory-bound kernel)
    p.tiles_x = (int)((g.nx + (32 - 2 * g.r) - 1) / (32 - 2 * g.r));
    p.tiles_y = (int)((g.ny + SC_WARPS * SC_TJ - 1) / (SC_WARPS * SC_TJ));
    const i64 slots = (i64)device_sms() * star_resident(variant, esize, g.r);
    const i64 tiles = (i64)p.tiles_x * p.tiles_y;
    chunks = slots / (tiles > 0 ? tiles : 1);
  } else {
    p.tiles_x = (int)((g.nx + TX - 1) / TX);
    p.tiles_y = (int)((g.ny + TY - 1) / TY);
    const i64 slots = (i64)device_sms() * star_resident(variant, esize, g.r);
    const i64 tiles = (i64)p.tiles_x * p.tiles_y;
    // waves of resident blocks: one for the float plane kernel; two for
    // double, whose blocks keep the FP64 pipe busy only while resident (128^3:
    // 60 -> 73 GLUP/s); four for the float two-plane kernel, the radius-2
    // float default (512^3: 229 GLUP/s for the column kernel, 355 here)
    const i64 waves = esize == 8 ? 2 : (variant == kStarPlane2 ? 4 : 1);
    chunks = (waves * slots + tiles - 1) / tiles;
    if (esize == 8) {
      // double sweeps are bound by the FP64 pipe, so the extra halo planes of
      // short chunks cost little while many short blocks keep every SM's pipe
      // busy to the end (measured at 512^3: 79 -> 86 GLUP/s from one chunk to
      // chunks of 16 planes; at 320^3: 71 -> 85).  At most 32768 blocks.
      i64 c16 = (g.nz + 15) / 16;
      const i64 cap = 32768 / (tiles > 0 ? tiles : 1);
      if (c16 > cap) c16 = cap;
      if (c16 > chunks) chunks = c16;
    }
  }
  // precedence: the autotuner's trial, the knob, the tuning cache, the plan
  StarChoice tc;
  if (star_force().chunks > 0)
    chunks = star_force().chunks;
  else if (const int kc = g_star_chunks.load(); kc > 0)
    chunks = kc;
  else if (tune_cache_lookup(g, esize, &tc) && tc.variant == variant && tc.chunks > 0)
    chunks = tc.chunks;
  if (chunks > max_chunks) chunks = max_chunks;
  if (chunks < 1) chunks = 1;
  p.kchunk = (int)((g.nz + chunks - 1) / chunks);
  p.chunks = (int)((g.nz + p.kchunk - 1) / p.kchunk);
  p.variant = variant;
  return p;
}

int star_variant(const Grid& g, size_t esize, const void* a, const void* b, const void* c) {
  (void)a;
  (void)b;
  (void)c;
  // the column kernel addresses rows with 32-bit offsets: TJ + 2R rows of NX
  if ((i64)(SC_TJ + 4) * g.NX() >= ((i64)1 << 31)) return kStarScalar;
  int v = -1;
  StarChoice tc;
  if (star_force().variant >= 0)
    v = star_force().variant;
  else if (const int ko = g_star_variant_override.load(); ko >= 0)
    v = ko;
  else if (tune_cache_lookup(g, esize, &tc) && tc.variant >= 0)
    v = tc.variant;
  // the staged kernel needs a ring stage of at least one row and its halo
  if (v == kStarStaged && !staged_applicable(g, esize)) v = -1;
  if (v >= 0) return v;
  // float sweeps are memory-bound.  Large grids take the staged kernel,
  // whose shared-memory ring keeps the most bytes in flight (512^3: 705
  // GLUP/s against 639 for the column kernel; radius 2: 482 against 338).
  // Below about 3e7 points, or with rows so long that a block holds fewer
  // than 8, its blocks are too few or too short: at radius 1 the column
  // kernel issues the fewest instructions per update; at radius 2 its
  // register rings cost too much occupancy and the two-plane kernel is
  // faster (1.3-1.6x).  Double sweeps are bound by the FP64 pipe: the plane
  // kernel keeps every lane of every FP64 instruction useful.
  if (esize == 4) {
    if ((double)g.interior() >= 3e7 && staged_rows(g, esize) >= 8) return kStarStaged;
    return g.r == 1 ? kStarColumn : kStarPlane2;
  }
  return kStarScalar;
}

i64 star_blocks(const Grid& g, size_t esize, const void* u, const void* b, const void* out) {
  return plan_star(g, star_variant(g, esize, u, b, out), esize).blocks();
}

LaunchPlan sweep_launch_plan(const Grid& g, size_t esize) {
  const ZPlan p = plan_star(g, star_variant(g, esize, nullptr, nullptr, nullptr), esize);
  LaunchPlan q;
  q.variant = p.variant;
  q.grid_x = p.tiles_x;
  q.grid_y = p.tiles_y;
  q.grid_z = p.chunks;
  q.kchunk = p.kchunk;
  if (p.variant == kStarStaged) {
    // whole rows: one warp per 32-wide i segment, at most SG_WARPS (launch_star_t)
    q.block_threads = 32 * (int)std::min<i64>((g.nx + 31) / 32, SG_WARPS);
    q.tile_w = (int)g.nx;
    q.tile_h = p.rg;
    q.stage_elems = p.stage_elems;
    q.smem = p.smem;
  } else if (p.variant == kStarColumn) {
    q.block_threads = 32 * SC_WARPS;
    q.tile_w = 32 - 2 * g.r;
    q.tile_h = SC_WARPS * SC_TJ;
  } else {
    q.block_threads = TX * TY;
    q.tile_w = TX;
    q.tile_h = TY;
  }
  return q;
}

}  // namespace stn
