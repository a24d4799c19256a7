"""C-ABI checks that need no GPU: the library loads, exports every entry point
that include/stencil.h declares, and rejects bad arguments with STN_EINVAL
before touching CUDA."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "stencil.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int64_t|int|void|char|stn_server)\s*\**\s*(\w+)\s*\(", src,
                       flags=re.M)
    return sorted(set(names))


def test_header_declares_the_path():
    names = declared_functions()
    for required in ("stencil_sweep_f64", "residual_norm_f64", "jacobi_solve_f64"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    so = lib.lib()
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing
    # and the binding wraps each of them
    assert set(declared_functions()) <= set(lib.SIGNATURES)


def test_version_and_empty_error(lib):
    assert "sm_103a" in lib.version()
    assert lib.last_error() == ""


FAKE_A = 0x7F0000000000
FAKE_B = 0x7F0100000000


def call(lib, name, *args):
    return getattr(lib.lib(), name)(*args)


def c3(*v):
    arr = (ctypes.c_double * len(v))(*v)
    return ctypes.cast(arr, ctypes.POINTER(ctypes.c_double)), arr


@pytest.mark.parametrize("nx,ny,nz,r,iters,why", [
    (0, 4, 4, 1, 1, "extents"), (4, -1, 4, 1, 1, "extents"), (4, 4, 4, 3, 1, "radius"),
    (4, 4, 4, 0, 1, "radius"), (4, 4, 4, 1, -1, "iters"), (1 << 29, 4, 4, 1, 1, "too large")])
def test_sweep_rejects_bad_arguments(lib, nx, ny, nz, r, iters, why):
    cp, _k = c3(0.0, 1 / 6, 0.0)
    for name in ("stencil_sweep_f64", "stencil_sweep_f32"):
        rc = call(lib, name, FAKE_A, FAKE_B, nx, ny, nz, cp, r, iters, None)
        assert rc == lib.STN_EINVAL, (name, why)
        assert "invalid argument" in lib.last_error()


def test_sweep_rejects_null_and_aliasing(lib):
    cp, _k = c3(0.0, 1 / 6)
    f = lib.lib().stencil_sweep_f64
    assert f(None, FAKE_B, 4, 4, 4, cp, 1, 1, None) == lib.STN_EINVAL
    assert f(FAKE_A, None, 4, 4, 4, cp, 1, 1, None) == lib.STN_EINVAL
    assert f(FAKE_A, FAKE_B, 4, 4, 4, None, 1, 1, None) == lib.STN_EINVAL
    assert f(FAKE_A, FAKE_A, 4, 4, 4, cp, 1, 1, None) == lib.STN_EINVAL
    # out starts inside in's 6*6*6 doubles
    assert f(FAKE_A, FAKE_A + 8 * 100, 4, 4, 4, cp, 1, 1, None) == lib.STN_EINVAL
    assert "overlap" in lib.last_error()


def test_residual_and_solvers_reject_bad_arguments(lib):
    cp, _k = c3(0.0, 1 / 6)
    out = ctypes.c_double()
    L = lib.lib()
    assert L.residual_norm_f64(None, None, 4, 4, 4, cp, 1, ctypes.byref(out), None) == lib.STN_EINVAL
    assert L.residual_norm_f64(FAKE_A, None, 4, 4, 4, cp, 1, None, None) == lib.STN_EINVAL
    assert L.residual_norm_f32(FAKE_A, None, 4, 4, 4, cp, 5, ctypes.byref(out), None) == lib.STN_EINVAL
    info = lib.SolveInfo()
    J = L.jacobi_solve_f64
    assert J(None, FAKE_A, 4, 4, 4, cp, 1, -1.0, 10, 1, ctypes.byref(info), None) == lib.STN_EINVAL
    assert J(None, FAKE_A, 4, 4, 4, cp, 1, 1e-6, -1, 1, ctypes.byref(info), None) == lib.STN_EINVAL
    assert J(None, FAKE_A, 4, 4, 4, cp, 1, 1e-6, 10, 0, ctypes.byref(info), None) == lib.STN_EINVAL
    assert J(None, FAKE_A, 4, 4, 4, cp, 1, float("nan"), 10, 1, ctypes.byref(info), None) == lib.STN_EINVAL
    assert J(FAKE_A, FAKE_A, 4, 4, 4, cp, 1, 1e-6, 10, 1, ctypes.byref(info), None) == lib.STN_EINVAL
    wp, _w = c3(0.0, 1.0, 0.25)
    assert L.varcoef_sweep_f64(FAKE_A, FAKE_B, None, FAKE_B + 4096, 4, 4, 4, wp, 2, 1, None) == lib.STN_EINVAL
    assert L.varcoef_sweep_f32(FAKE_A, FAKE_B, FAKE_B + (1 << 20), FAKE_A, 4, 4, 4, wp, 2, 1, None) == lib.STN_EINVAL
    assert L.varcoef_apply_f64(FAKE_A, FAKE_B, FAKE_A, 4, 4, 4, wp, 2, None) == lib.STN_EINVAL
    assert L.jacobi_solve_varcoef_refined(FAKE_A, FAKE_B, FAKE_B + (1 << 30), 4, 4, 4, wp, 2, 1e-10, -1, 3,
                                          ctypes.byref(info), None) == lib.STN_EINVAL


@pytest.mark.parametrize("nx,ny,r,iters,why", [
    (0, 4, 1, 1, "extents"), (4, -1, 1, 1, "extents"), (4, 4, 3, 1, "radius"), (4, 4, 1, -1, "iters"),
    (1 << 29, 4, 1, 1, "too large")])
def test_sweep2d_rejects_bad_arguments(lib, nx, ny, r, iters, why):
    cp, _k = c3(0.0, 0.25, 0.0)
    for name in ("stencil_sweep2d_f64", "stencil_sweep2d_f32"):
        assert call(lib, name, FAKE_A, FAKE_B, nx, ny, cp, r, iters, None) == lib.STN_EINVAL, (name, why)
        assert "invalid argument" in lib.last_error()
    L = lib.lib()
    assert L.stencil_sweep2d_f64(None, FAKE_B, 4, 4, cp, 1, 1, None) == lib.STN_EINVAL
    assert L.stencil_sweep2d_f64(FAKE_A, FAKE_A + 8 * 10, 4, 4, cp, 1, 1, None) == lib.STN_EINVAL
    assert "overlap" in lib.last_error()
    out = ctypes.c_double()
    assert L.residual_norm2d_f64(None, None, 4, 4, cp, 1, ctypes.byref(out), None) == lib.STN_EINVAL
    assert L.residual_norm2d_f32(FAKE_A, None, 4, 4, cp, 1, None, None) == lib.STN_EINVAL
    assert L.residual_norm2d_f64(FAKE_A, None, 4, 0, cp, 1, ctypes.byref(out), None) == lib.STN_EINVAL


def test_sum_and_dot_reject_bad_arguments(lib):
    L = lib.lib()
    out = ctypes.c_double()
    assert L.reduce_sum_f64(None, 10, ctypes.byref(out), None) == lib.STN_EINVAL
    assert L.reduce_sum_f64(FAKE_A, -1, ctypes.byref(out), None) == lib.STN_EINVAL
    assert L.reduce_sum_f64(FAKE_A, 10, None, None) == lib.STN_EINVAL
    assert L.reduce_sum_f64(FAKE_A + 4, 10, ctypes.byref(out), None) == lib.STN_EINVAL
    assert "aligned" in lib.last_error()
    assert L.dot_f64(FAKE_A, None, 10, ctypes.byref(out), None) == lib.STN_EINVAL
    assert L.dot_f64(FAKE_A, FAKE_B + 2, 10, ctypes.byref(out), None) == lib.STN_EINVAL


def test_advect_rejects_bad_arguments(lib):
    L = lib.lib()
    cp, _k = c3(0.25, 0.25, 0.25)
    outs = (ctypes.c_void_p * 3)(FAKE_B, FAKE_B + (1 << 20), FAKE_B + (2 << 20))
    assert L.advect_f64(None, FAKE_A, FAKE_A, None, 3, outs, 4, 4, 4, cp, None) == lib.STN_EINVAL
    assert L.advect_f64(FAKE_A, FAKE_A, FAKE_A, None, 3, None, 4, 4, 4, cp, None) == lib.STN_EINVAL
    assert L.advect_f64(FAKE_A, FAKE_A, FAKE_A, None, 3, outs, 4, 4, 4, None, None) == lib.STN_EINVAL
    nan, _n = c3(0.25, float("nan"), 0.25)
    assert L.advect_f32(FAKE_A, FAKE_A, FAKE_A, None, 3, outs, 4, 4, 4, nan, None) == lib.STN_EINVAL
    assert L.advect_f64(FAKE_A, FAKE_A, FAKE_A, None, 3, outs, 0, 4, 4, cp, None) == lib.STN_EINVAL
    qs = (ctypes.c_void_p * 7)(*([FAKE_A] * 7))
    assert L.advect_f64(FAKE_A, FAKE_A, FAKE_A, qs, 7, outs, 4, 4, 4, cp, None) == lib.STN_EINVAL
    same = (ctypes.c_void_p * 3)(FAKE_A, FAKE_B, FAKE_B + (1 << 20))
    assert L.advect_f64(FAKE_A, FAKE_A + (1 << 24), FAKE_A + (2 << 24), None, 3, same, 4, 4, 4, cp, None) \
        == lib.STN_EINVAL
    assert "overlap" in lib.last_error()


def test_binding_fails_loudly_without_library(tmp_path):
    """The package refuses to import when libstencil.so is absent (no fallback)."""
    import shutil
    import subprocess
    import sys
    pkg = os.path.join(ROOT, "paper_2409_18824_gb300")
    dst = tmp_path / "paper_2409_18824_gb300"
    shutil.copytree(pkg, dst, ignore=shutil.ignore_patterns("*.so", "_build", "__pycache__"))
    r = subprocess.run([sys.executable, "-c", "import paper_2409_18824_gb300"], cwd=tmp_path,
                       capture_output=True, text=True)
    assert r.returncode != 0 and "libstencil.so is missing" in r.stderr


def test_tuning_knobs(lib):
    assert lib.stencil_tune_get("star_variant") == -1
    for bad in (-2, 4, 99):
        with pytest.raises(lib.StencilError):
            lib.stencil_tune_set("star_variant", bad)
    with pytest.raises(lib.StencilError):
        lib.stencil_tune_set("no_such_knob", 0)
    lib.stencil_tune_set("star_variant", 1)
    assert lib.stencil_tune_get("star_variant") == 1
    lib.stencil_tune_set("star_variant", -1)
    for knob, good, bad in (("temporal_depth", 3, 5), ("batch_engine", 2, 3), ("solve_graph", 0, 2),
                            ("star_chunks", 7, -1), ("var_variant", 2, 3), ("repeat_graph", 0, 2),
                            ("sweep2d_resident", 0, 2), ("sweep2d_chunk", 100, 0),
                            ("fault_withhold_2d", 0, 2), ("sweep2d_tma", 0, 2),
                            ("sweep2d_ctas_per_sm", 2, 5)):
        before = lib.stencil_tune_get(knob)
        with pytest.raises(lib.StencilError):
            lib.stencil_tune_set(knob, bad)
        lib.stencil_tune_set(knob, good)
        assert lib.stencil_tune_get(knob) == good
        lib.stencil_tune_set(knob, before)


def test_header_parser_sees_every_return_type():
    names = declared_functions()
    assert "stencil_tune_cache_size" in names and "stencil_last_error" in names and "stn_server_create" in names


@pytest.fixture
def empty_cache(lib):
    lib.stencil_tune_cache_clear()
    yield
    lib.stencil_tune_cache_clear()


def test_tune_cache_put_get_save_load(lib, empty_cache, tmp_path):
    """The tuning cache round-trips through its JSON file: every field, device
    names with quotes and braces, replacement of an entry with the same key."""
    lib.stencil_tune_cache_put(512, 512, 512, 8, 1, 0, 32, 1, device="GPU A", glups=86.25, default_glups=85.5)
    lib.stencil_tune_cache_put(70, 45, 100, 4, 2, 1, 3, 2, device='odd "name" {x}')
    lib.stencil_tune_cache_put(512, 512, 512, 8, 1, 2, 16, 1, device="GPU A")  # replaces the first
    assert lib.stencil_tune_cache_size() == 2
    e = lib.stencil_tune_cache_get(512, 512, 512, 8, 1, device="GPU A")
    assert (e["variant"], e["chunks"], e["depth"], e["glups"]) == (2, 16, 1, 0.0)
    assert lib.stencil_tune_cache_get(512, 512, 512, 8, 2, device="GPU A") is None  # other radius
    assert lib.stencil_tune_cache_get(512, 512, 512, 4, 1, device="GPU A") is None  # other type
    assert lib.stencil_tune_cache_get(512, 512, 512, 8, 1, device="GPU B") is None  # other device
    path = str(tmp_path / "tune.json")
    lib.stencil_tune_cache_save(path)
    import json
    doc = json.load(open(path))
    assert doc["stencil_tune_cache"] == 1 and len(doc["entries"]) == 2
    lib.stencil_tune_cache_clear()
    assert lib.stencil_tune_cache_size() == 0
    assert lib.stencil_tune_cache_load(path) == 2
    e = lib.stencil_tune_cache_get(70, 45, 100, 4, 2, device='odd "name" {x}')
    assert (e["nx"], e["ny"], e["nz"], e["variant"], e["chunks"], e["depth"]) == (70, 45, 100, 1, 3, 2)
    # a hand-written file with fields in another order and extra keys loads too
    other = tmp_path / "hand.json"
    other.write_text('{"entries": [{"depth": 3, "chunks": 5, "variant": 0, "nz": 9, "ny": 8, "nx": 7, '
                     '"radius": 1, "esize": 8, "device": "GPU C", "note": "x"}], "stencil_tune_cache": 1}')
    assert lib.stencil_tune_cache_load(str(other)) == 1
    assert lib.stencil_tune_cache_get(7, 8, 9, 8, 1, device="GPU C")["depth"] == 3


def test_tune_cache_rejects_bad_entries_and_files(lib, empty_cache, tmp_path):
    good = dict(nx=8, ny=8, nz=8, esize=8, radius=1, variant=0, chunks=1, depth=1, device="d")
    for field, bad in (("esize", 2), ("radius", 3), ("variant", 4), ("variant", -1), ("chunks", 0),
                       ("chunks", 65536), ("depth", 0), ("depth", 5), ("nx", 0), ("nz", -4)):
        args = dict(good, **{field: bad})
        with pytest.raises(lib.StencilError) as ei:
            lib.stencil_tune_cache_put(**args)
        assert ei.value.code == lib.STN_EINVAL
    with pytest.raises(lib.StencilError):
        lib.stencil_tune_cache_get(8, 8, 8, 3, 1)
    assert lib.lib().stencil_tune_cache_save(None) == lib.STN_EINVAL
    assert lib.lib().stencil_tune_cache_load(None) == lib.STN_EINVAL
    assert lib.lib().stencil_tune_cache_put(None) == lib.STN_EINVAL
    with pytest.raises(lib.StencilError):
        lib.stencil_tune_cache_load(str(tmp_path / "missing.json"))
    with pytest.raises(lib.StencilError):
        lib.stencil_tune_cache_save(str(tmp_path / "no_dir" / "x.json"))
    bad_files = [
        '{"something_else": 1}',
        '{"stencil_tune_cache": 1}',
        '{"stencil_tune_cache": 1, "entries": [{"device": "d", "esize": 8}]}',  # fields missing
        '{"stencil_tune_cache": 1, "entries": [{"device": "d", "esize": 8, "radius": 1, "nx": 8, "ny": 8, '
        '"nz": 8, "variant": 7, "chunks": 1, "depth": 1}]}',  # out of range
        '{"stencil_tune_cache": 1, "entries": [{"device": "d", "esize": 8, "radius": 1, "nx": 8.5, "ny": 8, '
        '"nz": 8, "variant": 0, "chunks": 1, "depth": 1}]}',  # not an integer
        '{"stencil_tune_cache": 1, "entries": [{"device": "d", "esize": 8',  # truncated
    ]
    for i, text in enumerate(bad_files):
        f = tmp_path / f"bad{i}.json"
        f.write_text(text)
        with pytest.raises(lib.StencilError):
            lib.stencil_tune_cache_load(str(f))
    assert lib.stencil_tune_cache_size() == 0  # a bad file adds nothing
    # a file with one good entry before a bad one adds nothing either
    f = tmp_path / "half.json"
    f.write_text('{"stencil_tune_cache": 1, "entries": [{"device": "d", "esize": 8, "radius": 1, "nx": 8, '
                 '"ny": 8, "nz": 8, "variant": 0, "chunks": 1, "depth": 1}, {"device": "d"}]}')
    with pytest.raises(lib.StencilError):
        lib.stencil_tune_cache_load(str(f))
    assert lib.stencil_tune_cache_size() == 0


def test_tune_cache_loads_from_environment(tmp_path):
    """STN_TUNE_CACHE names a file that the first lookup in a process loads."""
    import subprocess
    import sys
    f = tmp_path / "env.json"
    f.write_text('{"stencil_tune_cache": 1, "entries": [{"device": "E", "esize": 4, "radius": 2, "nx": 3, '
                 '"ny": 4, "nz": 5, "variant": 1, "chunks": 2, "depth": 1}]}')
    code = ("import paper_2409_18824_gb300 as s; e = s.stencil_tune_cache_get(3, 4, 5, 4, 2, device='E'); "
            "print(s.stencil_tune_cache_size(), e['variant'], e['chunks'])")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120,
                       env=dict(os.environ, STN_TUNE_CACHE=str(f)))
    assert r.returncode == 0, r.stderr
    assert r.stdout.split() == ["1", "1", "2"]


def test_autotune_rejects_bad_arguments(lib):
    so = lib.lib()
    e = lib.TuneEntry()
    for args in ((0, 8, 8, 8, 1), (8, 8, 8, 2, 1), (8, 8, 8, 8, 3), (1 << 29, 8, 8, 8, 1)):
        assert so.stencil_autotune_sweep(*args, None, 0, ctypes.byref(e), None) == lib.STN_EINVAL
    assert so.stencil_autotune_sweep(8, 8, 8, 8, 1, None, -1, ctypes.byref(e), None) == lib.STN_EINVAL
    assert so.stencil_autotune_sweep(8, 8, 8, 8, 1, None, 0, None, None) == lib.STN_EINVAL


def test_read_only_plan_knobs_exist(lib):
    for knob in ("last_star_variant", "last_star_chunks", "last_temporal_depth"):
        lib.stencil_tune_get(knob)


def test_server_rejects_bad_options(lib):
    o = lib.ServerOpts()
    o.hbm_budget = 1 << 20
    o.radius = 3  # invalid
    o.tol = 1e-8
    o.check_every = 10
    o.max_inflight = 4
    o.queue_capacity = 16
    assert not lib.lib().stn_server_create(ctypes.byref(o))
    assert "out of range" in lib.last_error()
    o.radius = 1
    o.hbm_budget = 0
    assert not lib.lib().stn_server_create(ctypes.byref(o))
    o.hbm_budget = 1 << 20
    for engine, inflight in ((2, 4), (-1, 4), (1, 65)):  # unknown engine; too many worker streams
        o.engine, o.max_inflight = engine, inflight
        assert not lib.lib().stn_server_create(ctypes.byref(o))
        assert "out of range" in lib.last_error()
    assert not lib.lib().stn_server_create(None)


def _fuzz_cases():
    """Seeded mutations of a valid cache file (truncations, byte flips,
    inserted structural characters, deep nesting) and random text."""
    import random
    good = ('{"stencil_tune_cache": 1, "entries": [{"device": "d \\"q\\" {x}", "nx": 8, "ny": 9, "nz": 10, '
            '"esize": 8, "radius": 1, "variant": 2, "chunks": 3, "depth": 1, "glups": 1.5e2, '
            '"default_glups": -0.0}]}')
    rng = random.Random(20261204)
    cases = [good[:n] for n in range(0, len(good), 7)]
    alphabet = '{}[]":,\\ \n\t0123456789.-+eE' + "abcdefxyz" + "\x00\x7f\xff"
    for _ in range(300):
        s = list(good)
        for _ in range(rng.randint(1, 6)):
            op, pos = rng.randint(0, 2), rng.randrange(len(s) + 1)
            if op == 0 and s:
                del s[min(pos, len(s) - 1)]
            elif op == 1:
                s.insert(pos, rng.choice(alphabet))
            elif s:
                s[min(pos, len(s) - 1)] = rng.choice(alphabet)
        cases.append("".join(s))
    cases += ["".join(rng.choice(alphabet) for _ in range(rng.randint(0, 200))) for _ in range(100)]
    cases += ["[" * 5000, "{" * 5000, '"' + "\\" * 4999, '{"entries": ' + "[" * 3000]
    return cases


def test_tune_cache_reader_survives_malformed_files(lib, empty_cache, tmp_path):
    """The cache file reader never crashes and never half-loads: every input
    either loads whole (returns the entry count) or is refused with
    STN_EINVAL and adds nothing."""
    path = tmp_path / "fuzz.json"
    so = lib.lib()
    for i, text in enumerate(_fuzz_cases()):
        path.write_bytes(text.encode("latin-1", errors="replace"))
        lib.stencil_tune_cache_clear()
        rc = so.stencil_tune_cache_load(os.fsencode(str(path)))
        assert rc == lib.STN_EINVAL or rc >= 0, (i, rc)
        if rc == lib.STN_EINVAL:
            assert lib.stencil_tune_cache_size() == 0, i
        else:
            assert lib.stencil_tune_cache_size() == rc, i
    lib.stencil_tune_cache_clear()


def test_tune_cache_round_trips_random_entries(lib, empty_cache, tmp_path):
    import random
    rng = random.Random(7)
    entries = {}
    for _ in range(200):
        key = (rng.randint(1, 1 << 28), rng.randint(1, 1 << 28), rng.randint(1, 1 << 28), rng.choice([4, 8]),
               rng.choice([1, 2]))
        dev = "".join(rng.choice('ab "\\{}[],:xyz\t') for _ in range(rng.randint(0, 40)))
        val = (rng.randint(0, 3), rng.randint(1, 65535), rng.randint(1, 4), rng.uniform(0, 1e4))
        lib.stencil_tune_cache_put(*key, *val[:3], device=dev, glups=val[3])
        entries[(dev,) + key] = val
    path = str(tmp_path / "rt.json")
    lib.stencil_tune_cache_save(path)
    lib.stencil_tune_cache_clear()
    assert lib.stencil_tune_cache_load(path) == len(entries)
    for (dev, *key), (v, c, d, g) in entries.items():
        e = lib.stencil_tune_cache_get(*key, device=dev)
        assert (e["variant"], e["chunks"], e["depth"]) == (v, c, d) and e["glups"] == g


def test_tune_cache_device_names_that_look_like_fields(lib, empty_cache, tmp_path):
    """A device name ending in '"nx' is written as ...\\"nx" -- the text '"nx"'
    appears inside the string.  The reader takes fields in order, so such
    names (and ones holding whole fake fields, tabs or newlines) load back
    exactly, with every number intact."""
    names = ['gpu"nx', 'a"esize', 'x", "nx": 1, "y', 'tab\there', 'nl\nx', 'q\\"depth"', '"variant": 3}']
    for k, dev in enumerate(names):
        lib.stencil_tune_cache_put(100 + k, 200 + k, 300 + k, 8, 2, 1, 7 + k, 2, device=dev, glups=1.25 * k)
    path = str(tmp_path / "names.json")
    lib.stencil_tune_cache_save(path)
    import json
    assert [e["device"] for e in json.load(open(path))["entries"]] == sorted(names)  # valid JSON, names exact
    lib.stencil_tune_cache_clear()
    assert lib.stencil_tune_cache_load(path) == len(names)
    for k, dev in enumerate(names):
        e = lib.stencil_tune_cache_get(100 + k, 200 + k, 300 + k, 8, 2, device=dev)
        assert e is not None, dev
        assert (e["nx"], e["ny"], e["nz"], e["variant"], e["chunks"], e["depth"], e["glups"]) == (
            100 + k, 200 + k, 300 + k, 1, 7 + k, 2, 1.25 * k)


def test_binding_refuses_grids_the_kernels_would_overrun(lib):
    """The binding checks every array and tensor it passes: floats of the
    call's element size, contiguous, and at least as many elements as the
    extents need (explicit extents included), before the library sees it.
    These raise without reaching the library, so they run on the CPU."""
    import numpy as np
    import torch
    u64 = np.zeros((6, 7, 8))
    u32 = np.zeros((6, 7, 8), dtype=np.float32)
    c = (0.0, 1.0 / 6.0)
    with pytest.raises(TypeError, match="4-byte"):
        lib.stencil_sweep_f32(u64, u64.copy(), c, 1, 1)
    with pytest.raises(TypeError, match="8-byte"):
        lib.stencil_sweep_f64(u32, u32.copy(), c, 1, 1)
    with pytest.raises(TypeError):
        lib.stencil_sweep_f64(np.zeros((6, 7, 8), dtype=np.int64), u64, c, 1, 1)
    with pytest.raises(ValueError, match="holds 336 elements"):
        lib.stencil_sweep_f64(u64, u64.copy(), c, 1, 1, nx=7, ny=5, nz=4)  # needs 9 x 7 x 6 = 378
    with pytest.raises(ValueError, match="contiguous"):
        lib.stencil_sweep_f64(np.zeros((8, 7, 6)).transpose(2, 1, 0), u64, c, 1, 1)
    t = torch.zeros(1, 1, 8, dtype=torch.float64).expand(6, 7, 8)  # stride-0 view of 8 doubles
    with pytest.raises(ValueError, match="contiguous"):
        lib.stencil_sweep_f64(t, u64, c, 1, 1)
    with pytest.raises(TypeError):
        lib.dot_f64(np.zeros(16), np.zeros(16, dtype=np.float32))
    with pytest.raises(ValueError):
        lib.reduce_sum_f64(np.zeros(16), n=17)
    with pytest.raises(ValueError):
        lib.stencil_sweep2d_f64(np.zeros((5, 6)), np.zeros((5, 6)), (0.0, 0.25), 1, 1, nx=4, ny=4)
    with pytest.raises(TypeError):
        lib.advect_f64(u64, u64, u32, [u64, u64, u64], (0.1, 0.1, 0.1))
    with pytest.raises(ValueError):
        lib.jacobi_solve_batched_f64([np.zeros((6, 6, 6))], [np.zeros((6, 6, 5))], c, 1, 1e-8, 10)
    # a grid of the right kind gets past the binding to the library (which
    # has no GPU here: it reports the failed staging, not a binding error)
    with pytest.raises(lib.StencilError):
        lib.stencil_sweep_f64(u64, u64.copy(), c, 1, 2)
