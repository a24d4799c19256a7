"""Launch plans of the sweeps, checked on the CPU (no GPU: the planners then
assume 152 SMs and a fixed residency per SM).

`stencil_plan_query` returns the grid, block, tile and ring that a sweep of
given extents would launch, from the same host code the sweeps call.  For a
wide set of extents (cubes, the benchmark shapes, ragged and degenerate ones,
rows too long for the staged ring, extents at the library's limits) every
plan must cover each interior point exactly once with no empty block, stay
within CUDA's grid and block limits and the shared memory of an SM, and keep
the 32-bit offsets of the column kernels in range.  The staged kernel's copy
arithmetic (16-byte asynchronous copies of the span a plane contributes, with
element copies at the grid's ends) is replayed here for every alignment of
the grid's base address, the first and last row group and the first and last
k chunk: every copy must read inside the grid's bytes and land inside its
ring stage, and every ring element the update reads must be one the copy
wrote.
"""
import itertools

import pytest

SMEM_PER_BLOCK_MAX = 227 * 1024  # sm_103a, opt-in dynamic shared memory
STAGED_SMEM_MAX = 220 * 1024     # the staged kernel's ring budget
SG_PF = 1                        # planes in flight beyond the 2R+1 in use

SHAPES = [(512, 512, 512), (768, 768, 384), (320, 320, 320), (64, 64, 64), (1, 1, 1), (2, 3, 5), (33, 17, 9),
          (97, 61, 250), (1000, 7, 3), (5, 1000, 7), (3, 7, 1000), (100000, 2, 3), (60000, 40, 4),
          (26000, 64, 64), (2047, 2049, 31), (128, 96, 72), (4096, 4096, 16), (1 << 28, 1, 1), (1, 1 << 28, 1),
          (1, 1, 1 << 28)]


def cases():
    for (nx, ny, nz), esize, r in itertools.product(SHAPES, (4, 8), (1, 2)):
        yield nx, ny, nz, esize, r


def ceil_div(a, b):
    return -(-a // b)


def check_common(q, nx, ny, nz, r):
    assert q["block_threads"] % 32 == 0 and 32 <= q["block_threads"] <= 1024
    assert 1 <= q["grid_x"] < 2 ** 31 and 1 <= q["grid_y"] <= 65535 and 1 <= q["grid_z"] <= 65535
    # every interior point in exactly one block, and no block without points
    for n, tile, blocks in ((nx, q["tile_w"], q["grid_x"]), (ny, q["tile_h"], q["grid_y"]),
                            (nz, q["kchunk"], q["grid_z"])):
        assert tile >= 1 and blocks == ceil_div(n, tile), (n, tile, blocks)
    assert 0 <= q["smem_bytes"] <= SMEM_PER_BLOCK_MAX


def plan_or_rejected(lib, op, nx, ny, nz, esize, r):
    """The plan, or None when the extents need more than 65535 row tiles or k
    chunks in one launch (then the query, like the sweep, says so)."""
    from paper_2409_18824_gb300 import StencilError
    try:
        return lib.stencil_plan_query(op, nx, ny, nz, esize, r)
    except StencilError as e:
        assert e.code == -1 and "launch grid" in lib.last_error()
        return None


@pytest.mark.parametrize("nx,ny,nz,esize,r", list(cases()))
def test_sweep_plan_covers_the_grid_within_limits(lib, nx, ny, nz, esize, r):
    q = plan_or_rejected(lib, "sweep", nx, ny, nz, esize, r)
    if q is None:
        # only extents no tile height of any kernel (at most 64 rows) fits
        assert ny > 65535 * 8, (nx, ny, nz)
        return
    check_common(q, nx, ny, nz, r)
    NX = nx + 2 * r
    v = q["variant"]
    assert v in (0, 1, 2, 3)
    if v == 3:
        assert q["grid_x"] == 1 and q["tile_w"] == nx
        assert q["block_threads"] == 32 * min(ceil_div(nx, 32), 16)
        assert 1 <= q["tile_h"] <= min(64, ny)
        S = 2 * r + 1 + SG_PF
        assert q["smem_bytes"] == S * q["stage_elems"] * esize <= STAGED_SMEM_MAX
        # a stage holds the span's misalignment (< 16 bytes), its rows and the
        # rounding of the last 16-byte chunk
        assert q["stage_elems"] * esize >= (q["tile_h"] + 2 * r) * NX * esize + 32
    else:
        assert q["stage_elems"] == 0 and q["smem_bytes"] == 0
        if v == 1:
            assert (q["tile_w"], q["tile_h"], q["block_threads"]) == (32 - 2 * r, 32, 128)
            assert (8 + 2 * r) * NX < 2 ** 31  # the column kernel's 32-bit row offsets
        else:
            assert (q["tile_w"], q["tile_h"], q["block_threads"]) == (32, 8, 256)


@pytest.mark.parametrize("nx,ny,nz,esize,r", list(cases()))
def test_varcoef_plan_covers_the_grid_within_limits(lib, nx, ny, nz, esize, r):
    q = plan_or_rejected(lib, "varcoef_sweep", nx, ny, nz, esize, r)
    if q is None:
        assert ny > 65535 * 4, (nx, ny, nz)
        return
    check_common(q, nx, ny, nz, r)
    if q["variant"] == 2:
        # TMA-staged: float, radius 2, rows a multiple of 16 bytes
        assert esize == 4 and r == 2 and ((nx + 2 * r) * 4) % 16 == 0
        assert (q["tile_w"], q["tile_h"], q["block_threads"]) == (64, 16, 288)
        assert q["smem_bytes"] == VT_SMEM_ALLOC and q["stage_elems"] == 0
        assert q["grid_z"] <= ceil_div(nz, 16)
        return
    assert q["smem_bytes"] == 0 and q["stage_elems"] == 0
    if q["variant"] == 1:
        tj = 4 if esize == 4 else 2
        assert (q["tile_w"], q["tile_h"], q["block_threads"]) == (32 - 2 * r, 2 * tj, 64)
        assert (tj + 2 * r) * (nx + 2 * r) < 2 ** 31
        # at most ceil(nz / 8) k chunks, and at most 32768 blocks unless the
        # (i, j) tiles alone are more
        assert q["grid_z"] <= ceil_div(nz, 8)
        assert q["grid_x"] * q["grid_y"] * q["grid_z"] <= max(32768, q["grid_x"] * q["grid_y"])
    else:
        assert q["variant"] == 0 and (q["tile_w"], q["tile_h"], q["block_threads"]) == (32, 8, 256)


# the TMA-staged variable-coefficient float sweep (radius 2)
VT_TW, VT_TH, VT_R, VT_S, VT_Q, VT_CWARPS = 64, 16, 2, 6, 5, 8
VT_PW, VT_PH = VT_TW + 2 * VT_R, VT_TH + 2 * VT_R
VT_FIELD = -(-(VT_PW * VT_PH) // 32) * 32
VT_SMEM_ALLOC = VT_S * 3 * VT_FIELD * 4 + 128


def tma_block_replay(nx, ny, nz, bx, by, bz, kchunk):
    """Replays one block of the TMA-staged kernel: the tensor-map box origin of
    every plane it stages (x a multiple of 16 bytes, z inside the grid); the
    producer/consumer protocol of its ring (the producer puts plane p into
    stage (p - pfirst) % S once every consumer warp has released plane p - S;
    consumers wait for a plane's copies before reading it and release it after
    its last read), run as a simulation in which the producer issues as early
    as the protocol lets it: every read must find its own plane in the stage
    and the simulation must never stall; and every shared-memory element and
    global store of the threads (inside the box, inside the interior, on
    8-byte boundaries)."""
    R = VT_R
    NX, NY, NZ = nx + 2 * R, ny + 2 * R, nz + 2 * R
    tx0, ty0 = bx * VT_TW, by * VT_TH
    k0 = R + bz * kchunk
    k1 = min(k0 + kchunk, nz + R)
    assert k0 < k1
    pfirst, plast = k0 - R, k1 - 1 + R
    assert (tx0 * 4) % 16 == 0 and tx0 < NX and ty0 < NY
    assert 0 <= pfirst and plast <= NZ - 1
    assert VT_SMEM_ALLOC <= SMEM_PER_BLOCK_MAX
    stage = {}          # stage -> plane it holds (issued)
    released = set()
    issued = []

    def produce():
        # the producer issues every plane the protocol allows now
        while len(issued) < plast - pfirst + 1:
            p = pfirst + len(issued)
            if p - VT_S >= pfirst and (p - VT_S) not in released:
                return
            stage[(p - pfirst) % VT_S] = p
            issued.append(p)

    def read(p):
        produce()
        assert p in issued, ("would wait forever for plane", p)
        assert stage[(p - pfirst) % VT_S] == p, ("stage overwritten before its last read", p)

    for p in range(pfirst, pfirst + 2 * R):   # prologue: queue fill
        read(p)
    released |= {pfirst, pfirst + 1}
    for k in range(k0, k1):
        read(k + R)      # queue fill of plane k + 2
        read(k)          # in-plane neighbours, f
        released.add(k)  # the warps' last read of plane k
    produce()
    assert issued == list(range(pfirst, plast + 1))
    # shared-memory reads and global accesses of every consumer thread
    for tid in range(32 * VT_CWARPS):
        lx, ly = tid & 31, tid >> 5
        c, rr = 2 * lx + R, 2 * ly + R
        for col in (c - 2, c, c + 2):      # 8-byte loads: columns col, col + 1
            assert col % 2 == 0 and 0 <= col and col + 1 < VT_PW
        for row in range(rr - 2, rr + 4):
            assert 0 <= row < VT_PH
        gi, gj = tx0 + c, ty0 + rr
        for t in (0, 1):
            if gj + t < ny + R and gi < nx + R:
                for k in range(k0, k1):
                    off = (k * NY + gj + t) * NX + gi
                    assert off % 2 == 0  # 8-byte out stores
                    assert R <= gj + t < ny + R and R <= gi and gi + 1 <= nx + R < NX


def test_tma_varcoef_is_automatic_on_large_grids_only(lib):
    """The TMA-staged float sweep is the automatic choice where it has at least
    four waves of blocks (the variable-coefficient workload's grid), the column
    kernel below that and on rows that are not a multiple of 16 bytes."""
    assert lib.stencil_plan_query("varcoef_sweep", 768, 768, 384, 4, 2)["variant"] == 2
    assert lib.stencil_plan_query("varcoef_sweep", 512, 512, 256, 4, 2)["variant"] == 2
    assert lib.stencil_plan_query("varcoef_sweep", 96, 96, 48, 4, 2)["variant"] == 1
    assert lib.stencil_plan_query("varcoef_sweep", 767, 768, 384, 4, 2)["variant"] == 1
    assert lib.stencil_plan_query("varcoef_sweep", 768, 768, 384, 4, 1)["variant"] == 1
    assert lib.stencil_plan_query("varcoef_sweep", 768, 768, 384, 8, 2)["variant"] == 1


@pytest.fixture
def tma_forced(lib):
    lib.stencil_tune_set("var_variant", 2)
    yield
    lib.stencil_tune_set("var_variant", -1)


@pytest.mark.parametrize("shape", [(768, 768, 384), (64, 16, 8), (68, 17, 5), (4, 1, 1), (196, 50, 23),
                                   (60, 15, 130), (8, 100, 2), (132, 7, 64), (256, 33, 17), (384, 96, 200),
                                   (512, 512, 256), (28, 20, 12)])
def test_tma_varcoef_addressing_stays_in_bounds(lib, tma_forced, shape):
    nx, ny, nz = shape
    q = lib.stencil_plan_query("varcoef_sweep", nx, ny, nz, 4, 2)
    assert q["variant"] == 2
    check_common(q, nx, ny, nz, 2)
    gx, gy, gz, kc = q["grid_x"], q["grid_y"], q["grid_z"], q["kchunk"]
    for bx in sorted({0, gx - 1}):
        for by in sorted({0, gy - 1}):
            for bz in sorted({0, min(1, gz - 1), gz - 1}):
                tma_block_replay(nx, ny, nz, bx, by, bz, kc)


def staged_copies_stay_in_bounds(nx, ny, nz, esize, r, q, base_misalign):
    """Replays the staged kernel's addressing for one grid base alignment:
    the planes a block stages, the 16-byte chunks it copies asynchronously
    (only chunks wholly inside the grid's bytes), the element copies of the
    first and last chunk (only elements inside the grid), where they land in
    the ring stage, and the ring elements the update reads."""
    NX, NY, NZ = nx + 2 * r, ny + 2 * r, nz + 2 * r
    epc = 16 // esize
    psz = NX * NY
    gbase = 4096 + base_misalign  # any address with this alignment
    gend = gbase + NX * NY * NZ * esize
    rg, kchunk, stage = q["tile_h"], q["kchunk"], q["stage_elems"]
    S = 2 * r + 1 + SG_PF
    for by in sorted({0, q["grid_y"] - 1}):
        for bz in sorted({0, q["grid_z"] - 1}):
            j0 = r + by * rg
            rows = min(rg, ny + r - j0)
            assert rows >= 1
            k0 = r + bz * kchunk
            k1 = min(k0 + kchunk, nz + r)
            assert k0 < k1
            pfirst, plast = k0 - r, k1 - 1 + r
            assert 0 <= pfirst and plast <= NZ - 1
            assert j0 - r >= 0 and j0 + rows + r - 1 <= NY - 1
            n_el = (rows + 2 * r) * NX
            first = lambda p: (p * NY + (j0 - r)) * NX  # noqa: E731
            shift0 = ((gbase + first(pfirst) * esize) & 15) // esize
            pstep = psz & (epc - 1)
            # only the first S + 2 planes and the last ones matter for the
            # bounds (the others are interior spans); cap the loop
            planes = list(range(pfirst, min(plast, pfirst + S + 2) + 1)) + list(range(max(pfirst, plast - S), plast + 1))
            for p in sorted(set(planes)):
                addr = gbase + first(p) * esize
                a0 = addr & ~15
                nch = (addr - a0 + n_el * esize + 15) >> 4
                c_lo = 1 if a0 < gbase else 0
                c_hi = nch - 1 if a0 + (nch << 4) > gend else nch
                # asynchronous chunks: whole 16 bytes inside the grid
                if c_hi > c_lo:
                    assert a0 + 16 * c_lo >= gbase and a0 + 16 * c_hi <= gend
                # the ring stage receives nch chunks
                assert nch * 16 <= stage * esize
                # the copy puts the span at shift elements into the stage
                shift = (shift0 + (p - pfirst) * pstep) & (epc - 1)
                assert shift == ((addr - a0) // esize)
                # the update reads elements shift + row * NX + i (i in
                # [0, NX)), rows 0 .. rows + 2r - 1 of the span: all copied,
                # and all inside the stage
                lo, hi = shift, shift + n_el - 1
                assert 0 <= lo and hi < stage and hi < nch * epc


@pytest.mark.parametrize("nx,ny,nz,esize,r", [c for c in cases() if c[3] == 4])
def test_staged_ring_copies_and_reads_stay_in_bounds(lib, nx, ny, nz, esize, r):
    lib.stencil_tune_set("star_variant", 3)  # the staged kernel on these extents, if its ring fits
    try:
        q = plan_or_rejected(lib, "sweep", nx, ny, nz, esize, r)
    finally:
        lib.stencil_tune_set("star_variant", -1)
    if q is None:
        assert ny > 65535 * 8
        return
    if q["variant"] != 3:
        # one row and its halo do not fit the ring: the plan falls back
        assert (1 + 2 * r) * (nx + 2 * r) * esize + 32 > STAGED_SMEM_MAX // (2 * r + 2)
        return
    for mis in range(0, 16, esize):
        staged_copies_stay_in_bounds(nx, ny, nz, esize, r, q, mis)


def test_variant_rules_and_precedence(lib):
    """Float grids of >= 3e7 points take the staged kernel, smaller float grids
    the column kernel (radius 1) or the two-plane kernel (radius 2), double
    grids the plane kernel; a knob asking for a kernel that cannot run on the
    extents does not get it; a cache entry steers the plan."""
    q = lib.stencil_plan_query
    assert q("sweep", 512, 512, 512, 4, 1)["variant"] == 3
    assert q("sweep", 64, 64, 64, 4, 1)["variant"] == 1
    assert q("sweep", 64, 64, 64, 4, 2)["variant"] == 2
    assert q("sweep", 512, 512, 512, 8, 1)["variant"] == 0
    built_in = q("sweep", 60000, 600, 4, 4, 1)
    assert built_in["variant"] != 3  # rows too long for the ring
    lib.stencil_tune_set("star_variant", 3)
    try:
        assert q("sweep", 60000, 600, 4, 4, 1) == built_in  # the knob cannot have it: the built-in rule
        assert q("sweep", 64, 64, 64, 8, 1)["variant"] == 3
    finally:
        lib.stencil_tune_set("star_variant", -1)
    lib.stencil_tune_cache_clear()
    try:
        lib.stencil_tune_cache_put(70, 45, 100, 4, 1, 2, 13, 1)
        p = q("sweep", 70, 45, 100, 4, 1)
        assert p["variant"] == 2 and p["grid_z"] == 13
        assert q("sweep", 70, 45, 101, 4, 1)["variant"] == 1  # other extents: the built-in rule
    finally:
        lib.stencil_tune_cache_clear()


def test_plan_query_rejects_bad_arguments(lib):
    from paper_2409_18824_gb300 import StencilError
    for args in (("sweep", 0, 4, 4, 8, 1), ("sweep", 4, 4, 4, 2, 1), ("sweep", 4, 4, 4, 8, 3),
                 ("stencil", 4, 4, 4, 8, 1), ("varcoef_sweep", 4, -1, 4, 4, 2), ("sweep", 1 << 29, 1, 1, 8, 1)):
        with pytest.raises(StencilError):
            lib.stencil_plan_query(*args)
    assert "invalid argument" in lib.last_error()


SHAPES2D = [(1024, 1024), (1001, 1024), (1000, 37), (1, 1), (5, 3), (2, 7), (33, 2), (4096, 4096), (300, 5000),
            (16, 100000), (20000, 20000), (512, 152), (512, 153), (64, 64), (8, 1 << 20)]
J2_COLS = 4  # interior columns per thread when halo rows come through registers


@pytest.mark.parametrize("ctas", [1, 2])
@pytest.mark.parametrize("nx,ny", SHAPES2D)
@pytest.mark.parametrize("esize,r", [(8, 1), (4, 1), (8, 2), (4, 2)])
def test_sweep2d_plan_bands_layout_and_bulk_copies(lib, nx, ny, esize, r, ctas):
    """The paper's 2-D jacobi.  Resident plan: bands partition the rows (each
    at least r rows when there are several, at most tile_h), two copies of a
    band fit the shared memory, every row's interior starts on a 16-byte
    boundary, and each halo-row bulk copy (source in the exchange slots,
    destination in either copy of the band) is 16-byte aligned, a multiple of
    16 bytes long and inside its buffer; without bulk copies the registers
    cover the row.  Per-sweep plan: a grid-stride loop over 32 x 8 tiles."""
    lib.stencil_tune_set("sweep2d_ctas_per_sm", ctas)
    try:
        q = plan_or_rejected(lib, "sweep2d", nx, ny, 1, esize, r)
    finally:
        lib.stencil_tune_set("sweep2d_ctas_per_sm", 1)
    assert q is not None
    NX = nx + 2 * r
    assert q["grid_y"] == q["grid_z"] == 1 and q["block_threads"] % 32 == 0 and q["block_threads"] <= 1024
    if q["variant"] == 0:
        assert q["block_threads"] == 256 and (q["tile_w"], q["tile_h"]) == (32, 8)
        assert q["grid_x"] == min(ceil_div(nx, 32) * ceil_div(ny, 8), 152 * 8)
        assert q["smem_bytes"] == 0 and q["scratch_bytes"] == 0
        # resident is refused only when even bands of ceil(ny / (152 ctas))
        # rows do not fit, or the rows are too wide for registers
        nblk = min(max(ny // r, 1), 152 * ctas)
        ns = ceil_div(NX + 16 // esize, 16 // esize) * (16 // esize)
        small = 2 * (ceil_div(ny, nblk) + 2 * r) * ns * esize + 1024 <= SMEM_PER_BLOCK_MAX
        assert not small or (nx * esize % 16 and nx > J2_COLS * 1024 // ctas)
        return
    nblk, nbmax, ns, pad, thr = q["grid_x"], q["tile_h"], q["row_stride"], q["row_pad"], q["block_threads"]
    assert q["tile_w"] == nx and 1 <= nblk <= max(1, min(ny // r, 152 * ctas))
    assert nbmax == ceil_div(ny, nblk)
    bands = [((b + 1) * ny) // nblk - (b * ny) // nblk for b in range(nblk)]
    assert sum(bands) == ny and max(bands) <= nbmax and (nblk == 1 or min(bands) >= r)
    per16 = 16 // esize
    assert ns >= pad + NX and (ns * esize) % 16 == 0 and ((pad + r) * esize) % 16 == 0 and 0 <= pad < per16
    rows = nbmax + 2 * r
    assert q["smem_bytes"] == 2 * rows * ns * esize and q["smem_bytes"] + 1024 <= SMEM_PER_BLOCK_MAX
    assert rows * ns < 2 ** 31
    # the SM's 1024 threads are shared by its bands (the knob asks for `ctas`
    # per SM; the planner takes fewer when that many do not fit)
    per_sm = ceil_div(nblk, 152)
    assert per_sm <= ctas and 32 <= thr <= 1024 // per_sm and thr <= ceil_div(nbmax * nx, 32) * 32
    # global scratch: nblk 64-bit flags, the status word, then the exchange
    # slots: 2 parities x nblk bands x 2 sides x r rows of nx values
    xo, scratch = q["xchg_offset"], q["scratch_bytes"]
    assert xo >= 8 * nblk + 4 and xo % 256 == 0
    assert scratch == xo + 2 * nblk * 2 * r * nx * esize
    if not q["bulk_copy"]:
        assert nx <= J2_COLS * thr
        return
    assert (nx * esize) % 16 == 0
    nbytes = nx * esize
    buf = rows * ns * esize  # one copy of the band
    slot = r * nx            # one side's rows in an exchange slot, elements
    for b in sorted({0, 1, nblk // 2, nblk - 2, nblk - 1} & set(range(nblk))):
        up, down = b > 0, b + 1 < nblk
        for par in (0, 1):
            for t in (0, 1):
                for rr in range(r):
                    for side, ok, src_slot, dst_row in (("up", up, 2 * (b - 1) + 1, rr),
                                                        ("down", down, 2 * (b + 1), r + bands[b] + rr)):
                        if not ok:
                            continue
                        src = xo + ((par * nblk * 2 + src_slot) * slot + rr * nx) * esize
                        dst = t * buf + (dst_row * ns + pad + r) * esize
                        assert src % 16 == 0 and dst % 16 == 0 and nbytes % 16 == 0, (side, b)
                        assert xo <= src and src + nbytes <= scratch
                        assert t * buf <= dst and dst + nbytes <= (t + 1) * buf


def test_batched_unit_split_covers_each_problem_once(lib):
    """The batched solvers' and the server's split of a problem into work
    units (tile shape x k chunk), over the benchmark's 2048-problem mix
    (sizes log-uniform in [16, 128]), the serving mix ([32, 256]) and edge
    extents: the tiles and chunks cover the interior exactly once with no
    empty unit, the shape is the one with the fewest tiles (ties to the wider
    rows), chunks are 128-256 planes (fewer only when nz is), and every shape's
    shared plane (tile plus a halo of 2 on each side) fits the kernel's one
    plane buffer.  The shape counts over the 2048 mix are those the
    scheduler's measurements were taken with: 1050, 420 and 578."""
    import stencil_inputs as si
    mix = [tuple(int(v) for v in s) for s in si.log_uniform_sizes(2048, 16, 128, 4)]
    serve = [tuple(int(v) for v in s) for s in si.log_uniform_sizes(48, 32, 256, 6)]
    edge = [(1, 1, 1), (1, 1000, 3), (1000, 1, 3), (8, 32, 64), (9, 33, 65), (4096, 4096, 4096), (1 << 20, 1, 1)]
    shapes = [0, 0, 0]
    widths = {0: 32, 1: 16, 2: 8}
    for k, (nx, ny, nz) in enumerate(mix + serve + edge):
        q = lib.stencil_plan_query("batch_unit", nx, ny, nz, 8, 1)
        tw, th = q["tile_w"], q["tile_h"]
        assert q["block_threads"] == tw * th == 256 and tw == widths[q["variant"]]
        assert (q["grid_x"], q["grid_y"], q["grid_z"]) == (ceil_div(nx, tw), ceil_div(ny, th), ceil_div(nz, q["kchunk"]))
        tiles = {s: ceil_div(nx, w) * ceil_div(ny, 256 // w) for s, w in widths.items()}
        assert tiles[q["variant"]] == min(tiles.values())
        assert all(tiles[s] > tiles[q["variant"]] for s in range(q["variant"]))  # ties to the wider shape
        assert q["kchunk"] <= 256 and (q["kchunk"] >= 128 or q["kchunk"] == nz)
        for w in widths.values():
            assert (256 // w + 4) * (w + 4) <= q["stage_elems"]
        if k < len(mix):
            shapes[q["variant"]] += 1
    assert shapes == [1050, 420, 578]


def test_batched_entry_rejects_problems_beyond_its_counters(lib):
    """Checked on the host before any allocation or launch: a problem whose
    units per pass exceed what a slot's claim word counts (2^22), and a batch
    whose scratch exceeds any device's memory, are refused (no CUDA call is
    made, so this runs on the CPU); the plan query refuses the former too."""
    import ctypes
    from paper_2409_18824_gb300 import Problem, StencilError
    so = lib._lib
    coeffs = (ctypes.c_double * 2)(0.0, 1.0 / 6.0)
    fake = 1 << 40  # never dereferenced: the calls fail validation first
    big = (Problem * 1)(Problem(1 << 20, 1 << 20, 8, None, fake))
    assert so.jacobi_solve_batched_f64(big, 1, coeffs, 1, 1e-8, 10, 1, None, None) == -1
    assert "work units" in lib.last_error()
    with pytest.raises(StencilError):
        lib.stencil_plan_query("batch_unit", 1 << 20, 1 << 20, 8, 8, 1)
    # 2^17 x 2^10 x 2^11: 4096 x 128 tiles x 8 chunks of 256 planes = 2^22 units, the most
    # allowed; one more column of tiles is refused
    assert lib.stencil_plan_query("batch_unit", 1 << 17, 1 << 10, 1 << 11, 8, 1)
    with pytest.raises(StencilError):
        lib.stencil_plan_query("batch_unit", (1 << 17) + 1, 1 << 10, 1 << 11, 8, 1)
    # 1000 problems of that size: each within its limits, 2.2e15 bytes in all
    many = (Problem * 1000)(*[Problem(1 << 17, 1 << 10, 1 << 11, None, fake + i * 4096) for i in range(1000)])
    assert so.jacobi_solve_batched_f64(many, 1000, coeffs, 1, 1e-8, 10, 1, None, None) == -2
    assert "scratch" in lib.last_error()


def random_extents(n, seed, dims, hi):
    import numpy as np
    rng = np.random.default_rng(seed)
    return [tuple(int(v) for v in np.exp(rng.uniform(0.0, np.log(hi), size=dims)).round().clip(1, None))
            for _ in range(n)]


def test_random_extents_all_plans(lib):
    """The same checks on 300 seeded random extents (log-uniform in
    [1, 4000] per axis) for both types and radii, with the staged kernel's
    copy replay forced on wherever its ring fits."""
    import numpy as np
    rng = np.random.default_rng(91)
    for (nx, ny, nz) in random_extents(300, 90, 3, 4000):
        esize, r = int(rng.choice([4, 8])), int(rng.choice([1, 2]))
        test_sweep_plan_covers_the_grid_within_limits(lib, nx, ny, nz, esize, r)
        test_varcoef_plan_covers_the_grid_within_limits(lib, nx, ny, nz, esize, r)
        if esize == 4:
            test_staged_ring_copies_and_reads_stay_in_bounds(lib, nx, ny, nz, esize, r)


def test_random_extents_2d_plans(lib):
    import numpy as np
    rng = np.random.default_rng(93)
    for (nx, ny) in random_extents(150, 92, 2, 20000):
        esize, r = int(rng.choice([4, 8])), int(rng.choice([1, 2]))
        test_sweep2d_plan_bands_layout_and_bulk_copies(lib, nx, ny, esize, r, 1)


@pytest.mark.parametrize("op,esize,r", [("sweep", 8, 1), ("sweep", 8, 2), ("sweep", 4, 1), ("sweep", 4, 2),
                                        ("varcoef_sweep", 8, 2), ("varcoef_sweep", 4, 2)])
def test_rejection_starts_one_row_past_65535_tiles(lib, op, esize, r):
    """For a 1-column, 1-plane grid, the planned tile height h fixes the
    limit: ny = 65535 h plans exactly 65535 blocks in y and is accepted,
    ny = 65535 h + 1 is refused (unless the planner then picks a kernel with
    taller tiles, in which case that plan must be within the limit)."""
    h = lib.stencil_plan_query(op, 1, 1000, 1, esize, r)["tile_h"]
    q = lib.stencil_plan_query(op, 1, 65535 * h, 1, esize, r)
    if q["tile_h"] == h:
        assert q["grid_y"] == 65535
    after = plan_or_rejected(lib, op, 1, 65535 * h + 1, 1, esize, r)
    assert after is None or (after["grid_y"] <= 65535 and after["tile_h"] > h)


# The scheduler's radius-1 unit ring (sched.cu): stages of a 12 x 36 plane
# with halo plus the tile's 256 source-term values; 27.5 KB, 5 double stages
# or 10 float stages, at both 4 and 5 blocks per SM.
SCHED_STAGE_ELEMS = 12 * 36 + 256


def sched_ring(esize, minb):
    nbytes = 5 * SCHED_STAGE_ELEMS * 8
    assert minb * (nbytes + 1024 + 512) <= 233472
    stages = min(12, nbytes // (SCHED_STAGE_ELEMS * esize))
    pairs = stages >= 6
    return stages, pairs, stages - 5 if pairs else stages - 3


def sched_ring_replay(k0, k1, S, pairs, PF):
    """Replays a unit's ring: one cp.async commit group per issued plane slot
    (empty past the last plane), cp.async.wait_group PF - 1 then a block
    barrier per step, the step's issues into the stages its planes free, then
    its reads.  Every read plane must have landed (its group is not among the
    PF - 1 most recent) and still sit in its stage; an issue may only
    overwrite a plane no step from this one on reads."""
    R = 1
    pfirst, plast = k0 - R, k1 - 1 + R
    groups, stage = [], {}

    def issue(p):
        if p <= plast:
            old = stage.get((p - pfirst) % S)
            assert old is None or old == p - S
            stage[(p - pfirst) % S] = p
        groups.append(p)
        return stage.get((p - pfirst) % S) if p <= plast else None

    step = 2 if pairs else 1
    for p in range(pfirst, pfirst + (2 * R + 1 + PF if pairs else S - 1)):
        issue(p)
    for k in range(k0, k1, step):
        landed = set(g for g in groups[:len(groups) - (PF - 1)] if g <= plast)
        reads = [k - 1, k, k + 1] + ([k + 2] if pairs and k + 1 < k1 else [])
        first_read_now = k - 1
        news = [k + R + PF + 1, k + R + PF + 2] if pairs else [k + R + PF]
        for p in news:
            if p <= plast:
                assert p - S < first_read_now, ("overwrites a plane still read", p - S, k)
            issue(p)
        for p in reads:
            assert pfirst <= p <= plast
            assert p in landed, ("read before its copy landed", p, k)
            assert stage[(p - pfirst) % S] == p, ("stage overwritten before its read", p, k)
    assert sorted(set(g for g in groups if g <= plast)) == list(range(pfirst, plast + 1))


@pytest.mark.parametrize("esize,minb", [(4, 5), (8, 5), (4, 4), (8, 4)])
def test_sched_unit_ring_protocol(esize, minb):
    S, pairs, PF = sched_ring(esize, minb)
    assert PF >= 1 and S * SCHED_STAGE_ELEMS * esize <= 5 * SCHED_STAGE_ELEMS * 8
    expect = {(4, 5): (10, True, 5), (8, 5): (5, False, 2), (4, 4): (10, True, 5), (8, 4): (5, False, 2)}
    assert (S, pairs, PF) == expect[(esize, minb)]
    for k0 in (1, 65, 129):
        for n in range(1, 140):
            sched_ring_replay(k0, k0 + n, S, pairs, PF)
    # the replay catches a ring one stage too small, and a wait one group too lax
    with pytest.raises(AssertionError):
        sched_ring_replay(1, 40, S - 1, pairs, PF)
    with pytest.raises(AssertionError):
        sched_ring_replay(1, 40, S, pairs, PF + 1)


def sched_unit_bounds_replay(nx, ny, nz, shape, q):
    """The addresses of one scheduler unit's radius-1 ring sweep (sched.cu,
    star_tile_async / star_tile_async2), replayed for every thread of the
    block: each copy reads inside the padded grid and writes inside its
    stage (plane with halo, then the tile's source-term values), every cell an
    updating thread reads was written by some thread's copy, and every store
    goes to an interior point of the unit's tile and planes."""
    R, BT = 1, 256
    tw = {0: 32, 1: 16, 2: 8}[shape]
    th = BT // tw
    NX, NY, NZ = nx + 2, ny + 2, nz + 2
    tiles_x, tiles_y = ceil_div(nx, tw), ceil_div(ny, th)
    tiles = tiles_x * tiles_y
    klen = min(max(ceil_div(nz * tiles, 256), 128), 256, nz)
    kci, tq = divmod(q, tiles)
    tyi, txi = divmod(tq, tiles_x)
    k0 = R + kci * klen
    k1 = min(k0 + klen, nz + R)
    pitch = tw + 2
    plane_elems = (8 + 4) * (32 + 4)
    written, reads, stores = set(), [], []
    for flat in range(BT):
        tx, ty = flat % tw, flat // tw
        gi, gj = txi * tw + tx + R, tyi * th + ty + R
        inx, iny = gi < NX, gj < NY
        active = gi < nx + R and gj < ny + R
        hx = tx < R or tx >= tw - R
        hx_i = gi - R if tx < R else gi + R
        hx_lx = tx if tx < R else tx + 2 * R
        hx_ok = hx and hx_i < NX and iny
        hy = ty < R or ty >= th - R
        hy_j = gj - R if ty < R else gj + R
        hy_ly = ty if ty < R else ty + 2 * R
        hy_ok = hy and hy_j < NY and inx
        me = (ty + R) * pitch + tx + R
        copies = []
        if inx and iny:
            copies.append((me, gi, gj))
        if hx_ok:
            copies.append(((ty + R) * pitch + hx_lx, hx_i, gj))
        if hy_ok:
            copies.append((hy_ly * pitch + tx + R, gi, hy_j))
        for cell, i, j in copies:
            assert 0 <= cell < plane_elems and 0 <= i < NX and 0 <= j < NY
            written.add(cell)
        if active:
            assert plane_elems + flat < plane_elems + BT
            reads += [me, me - 1, me + 1, me - pitch, me + pitch]
            stores.append((gi, gj))
    for cell in reads:
        assert cell in written, ("read of a cell no copy fills", cell)
    for gi, gj in stores:
        assert 1 <= gi <= nx and 1 <= gj <= ny
    # planes copied: k0 - 1 .. k1 (the Dirichlet planes at the ends included)
    assert 0 <= k0 - R and k1 - 1 + R <= NZ - 1 and k0 < k1


@pytest.mark.parametrize("ext", [(16, 16, 16), (37, 19, 11), (130, 7, 40), (1, 1, 1), (33, 40, 3), (8, 30, 12),
                                 (64, 20, 9), (123, 123, 122), (9, 300, 200), (300, 9, 130), (17, 256, 5)])
def test_sched_unit_addresses_in_bounds(lib, ext):
    nx, ny, nz = ext
    p = lib.stencil_plan_query("batch_unit", nx, ny, nz, 8, 1)
    shape = p["variant"]
    n = p["grid_x"] * p["grid_y"] * p["grid_z"]
    assert p["kchunk"] == min(max(ceil_div(nz * p["grid_x"] * p["grid_y"], 256), 128), 256, nz)
    for q in sorted({0, 1, n // 2, n - 1} & set(range(n))):
        sched_unit_bounds_replay(nx, ny, nz, shape, q)
