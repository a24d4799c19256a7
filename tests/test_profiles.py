"""The bench's `traffic` figures against the ncu summaries they come from.

Every roofline line of bench.py carries the DRAM bytes (read + write) of its
timed kernel, taken from an ncu capture summarised under profiles/.  Here each
constant is recomputed from the summary's own numbers (the column of the
current build), so that a stale or mistyped figure fails.  Each summary must
also give the full command that made it, with the clock control left off.
"""
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

PROFILES = os.path.join(ROOT, "profiles")
UNIT = {"KB": 1e3, "MB": 1e6, "GB": 1e9}


def read(name):
    with open(os.path.join(PROFILES, name)) as f:
        return f.read()


def dram_bytes(text):
    """Read + write DRAM bytes of the first (current) column of a summary's
    table: either one row 'dram__bytes_read.sum / write | R / W' or two rows."""
    m = re.search(r"\| dram__bytes_read\.sum / write \| ([\d.]+) (KB|MB|GB) / ([\d.]+) (KB|MB|GB)", text)
    if m:
        return float(m.group(1)) * UNIT[m.group(2)] + float(m.group(3)) * UNIT[m.group(4)]
    r = re.search(r"\| dram__bytes_read\.sum \| ([\d.]+) (KB|MB|GB)", text)
    w = re.search(r"\| dram__bytes_write\.sum \| ([\d.]+) (KB|MB|GB)", text)
    assert r and w, "no DRAM rows"
    return float(r.group(1)) * UNIT[r.group(2)] + float(w.group(1)) * UNIT[w.group(2)]


CASES = [
    # summary, units the captured launch processed, the bench's bytes per unit
    ("star_kernel_f64_sweep320_full.md", 320 ** 3, bench.TRAFFIC_BYTES_PER_LUP[("f64", 0)]),
    ("star_col_kernel_f32_sweep320_full.md", 320 ** 3, bench.TRAFFIC_BYTES_PER_LUP[("f32", 1)]),
    ("star_staged_kernel_f32_sweep320_full.md", 320 ** 3, bench.TRAFFIC_BYTES_PER_LUP[("f32", 3)]),
    ("j2d_resident_kernel_f64_jacobi1024_full.md", 1, bench.TRAFFIC_J2D_LAUNCH),
    ("vec_reduce_kernel_dot_2e27_full.md", 2 ** 27, bench.TRAFFIC_DOT_PER_PAIR),
    ("sum_kernel_f64_2e27_full.md", 2 ** 27, bench.TRAFFIC_SUM_PER_ELEMENT),
    ("advect_kernel_f64_512x512x256_full.md", 512 * 512 * 256, bench.TRAFFIC_ADVECT_PER_CELL),
    ("var_tma_kernel_f32_512x512x256_full.md", 512 * 512 * 256, bench.TRAFFIC_VARCOEF_F32_PER_LUP),
]


@pytest.mark.parametrize("name,units,per_unit", CASES)
def test_bench_traffic_matches_the_summary(name, units, per_unit):
    got = dram_bytes(read(name))
    assert abs(per_unit * units - got) <= 1e-9 * got, (name, per_unit * units, got)


def test_automatic_float_plan_uses_the_staged_figure():
    assert bench.TRAFFIC_BYTES_PER_LUP[("f32", -1)] == bench.TRAFFIC_BYTES_PER_LUP[("f32", 3)]


@pytest.mark.parametrize("name", sorted(os.listdir(PROFILES)))
def test_summary_is_short_text_with_its_command(name):
    assert name.endswith((".md", ".txt")), name
    text = read(name)
    assert len(text) < 16 * 1024
    # the command: indented lines, continued with backslashes, running ncu
    lines = text.splitlines()
    commands, cur = [], ""
    for ln in lines:
        if ln.startswith("    ") and ln.strip():
            cur += " " + ln.strip().rstrip("\\")
            if not ln.rstrip().endswith("\\"):
                commands.append(cur)
                cur = ""
        elif cur:
            commands.append(cur)
            cur = ""
    assert commands, f"{name}: no command"
    # summaries of in-kernel counters (stencil_sched_stats) have no ncu
    # command; every ncu command keeps the clocks unlocked
    for c in commands:
        if re.search(r"(^|\s)ncu\s", c):
            assert "--clock-control none" in c, (name, c)
