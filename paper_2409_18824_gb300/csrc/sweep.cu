// Host-side planning of the star-stencil kernels (star.cuh) and the tuning
// override; the kernels themselves are instantiated per element type in
// sweep_f64.cu and sweep_f32.cu so that the two compile in parallel.
#include "star.cuh"

namespace stn {

static int g_star_variant_override = -1;

int tune_set_star_variant(int v) {
  if (v < -1 || v > 2) return STN_EINVAL;
  g_star_variant_override = v;
  return STN_OK;
}
int tune_get_star_variant() { return g_star_variant_override; }

static int g_temporal_depth = 0;
int tune_set_temporal_depth(int d) {
  if (d < 0 || d > 4) return STN_EINVAL;
  g_temporal_depth = d;
  return STN_OK;
}
int tune_get_temporal_depth() { return g_temporal_depth; }

ZPlan plan_star(const Grid& g, int variant, size_t esize) {
  ZPlan p;
  // blocks resident per SM for each variant (register-limited)
  i64 resident;
  if (variant == kStarColumn) {
    p.tiles_x = (int)((g.nx + (32 - 2 * g.r) - 1) / (32 - 2 * g.r));
    p.tiles_y = (int)((g.ny + SC_WARPS * SC_TJ - 1) / (SC_WARPS * SC_TJ));
    resident = esize == 4 ? 8 : 5;
  } else {
    p.tiles_x = (int)((g.nx + TX - 1) / TX);
    p.tiles_y = (int)((g.ny + TY - 1) / TY);
    resident = esize == 4 ? 8 : 5;
    if (variant == kStarPlane2) resident = esize == 4 ? 6 : 4;
  }
  const i64 want = 152 * resident;
  // enough blocks to fill every SM; chunks of >= 4 planes
  const i64 tiles = (i64)p.tiles_x * p.tiles_y;
  i64 chunks = (want + tiles - 1) / tiles;
  const i64 max_chunks = (g.nz + 3) / 4;
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
  const int ov = g_star_variant_override;
  if (ov >= 0) return ov;
  // float sweeps are memory-bound: the column kernel issues the fewest
  // instructions per update.  Double sweeps are bound by the FP64 pipe: the
  // plane kernel keeps every lane of every FP64 instruction useful.
  return esize == 4 ? kStarColumn : kStarScalar;
}

i64 star_blocks(const Grid& g, size_t esize, const void* u, const void* b, const void* out) {
  return plan_star(g, star_variant(g, esize, u, b, out), esize).blocks();
}

}  // namespace stn
