"""The paper's own figures that the bench quotes, against the cited fixture
tests/golden/paper_figures.json (workload sizes from Sec. 4 and 6.1, runtimes
from Tables 2 and 3, speed-ups from Table 4, GPU runtimes from Table 5), so
that a mistyped constant in bench.py fails here."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

FIG = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_figures.json")))


def test_every_entry_is_cited():
    for group in ("workloads",):
        for name, entry in FIG[group].items():
            assert entry.get("cite", "").startswith("Sec. "), name
    for group in ("runtime_seconds", "intrinsics_seconds", "openmp_speedup", "gpu_pw_advection_seconds"):
        assert FIG[group]["cite"].startswith("Sec. ") and "Table" in FIG[group]["cite"], group


def test_workload_sizes():
    j = FIG["workloads"]["jacobi"]
    assert (bench.JACOBI2D["nx"], bench.JACOBI2D["ny"]) == tuple(j["grid"])
    assert bench.JACOBI2D["sweeps"] == j["iterations"]
    pw = FIG["workloads"]["pw_advection"]
    assert [bench.ADVECT["nx"], bench.ADVECT["ny"], bench.ADVECT["nz"]] == pw["grid"]
    assert bench.INTRINSICS["sum"]["n"] == FIG["workloads"]["sum"]["array"][0] * FIG["workloads"]["sum"]["array"][1]
    # "134 million elements": read as 2^27 = 134,217,728
    n_dot = bench.INTRINSICS["dot"]["n"]
    assert n_dot == 2 ** 27 and round(n_dot / 1e6) == FIG["workloads"]["dotproduct"]["elements_millions"]


def test_quoted_runtimes_and_speedups():
    rt = FIG["runtime_seconds"]["jacobi"]
    assert abs(bench.PAPER_JACOBI2D_GLUPS - 1024 * 1024 * 100000 / rt["mlir_flow"] / 1e9) < 1e-12
    for kind in ("sum", "dotproduct"):
        w = bench.INTRINSICS["sum" if kind == "sum" else "dot"]
        assert (w["paper_s"], w["flang_s"]) == (FIG["intrinsics_seconds"][kind]["mlir_flow"],
                                                FIG["intrinsics_seconds"][kind]["flang_v20"])
    for const, key in ((bench.PAPER_OPENMP_JACOBI_SPEEDUP, "jacobi"), (bench.PAPER_OPENMP_PW_SPEEDUP, "pw_advection")):
        assert {str(k): v for k, v in const.items()} == FIG["openmp_speedup"][key]


def test_quoted_figures_in_the_bench_source():
    """The figures quoted as context inside bench.py's JSON lines."""
    src = open(os.path.join(ROOT, "bench.py")).read()
    rt = FIG["runtime_seconds"]["jacobi"]
    for v in (rt["mlir_flow"], rt["flang_v20"], rt["cray"], rt["gnu"]):
        assert repr(v) in src, v
    assert repr(FIG["runtime_seconds"]["pw_advection"]["mlir_flow"]) in src
    assert repr(FIG["gpu_pw_advection_seconds"]["cells"]["1.1 billion"]) in src
