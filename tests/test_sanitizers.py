"""The two plain host libraries under gcc's AddressSanitizer and
UndefinedBehaviorSanitizer: the CPU oracle (oracle/oracle.c) and the
multi-core host path (paper_2409_18824_gb300/host/stencil_host.cpp).

Both are rebuilt with -fsanitize=address,undefined (every undefined-behaviour
report fatal) into a temporary copy of the sources, and their CPU tests run
there in a subprocess with the sanitizer runtimes preloaded: an out-of-bounds
access, a use after free, a signed overflow or a misaligned load in either
library fails this test.  Skipped where gcc has no sanitizer runtimes.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SAN = ["-O1", "-g", "-fsanitize=address,undefined", "-fno-omit-frame-pointer", "-fno-sanitize-recover=undefined",
       "-ffp-contract=off", "-fPIC", "-shared"]
TESTS = ["test_oracle.py", "test_oracle_2d.py", "test_oracle_advect.py", "test_oracle_reduce.py",
         "test_host_path.py", "test_properties.py"]


def runtime(name):
    gcc = shutil.which("gcc")
    if not gcc:
        return None
    path = subprocess.run([gcc, f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
    return path if os.path.isabs(path) and os.path.exists(path) else None


@pytest.mark.slow
def test_oracle_and_host_library_are_clean_under_asan_and_ubsan(tmp_path):
    asan, ubsan = runtime("libasan.so"), runtime("libubsan.so")
    if not (asan and ubsan and shutil.which("g++")):
        pytest.skip("gcc sanitizer runtimes not available")
    work = tmp_path / "w"
    work.mkdir()
    for d in ("oracle", "stencil_inputs", "include", "paper_2409_18824_gb300"):
        shutil.copytree(os.path.join(ROOT, d), work / d, ignore=shutil.ignore_patterns("__pycache__", "_build"))
    (work / "tests").mkdir()
    for f in ["conftest.py", *TESTS]:
        shutil.copy(os.path.join(ROOT, "tests", f), work / "tests" / f)
    # instrumented builds, newer than their sources so the loaders keep them
    subprocess.run(["gcc", *SAN, "-std=c11", "-o", str(work / "oracle" / "liboracle.so"),
                    str(work / "oracle" / "oracle.c"), "-lm"], check=True)
    subprocess.run(["g++", *SAN, "-std=c++17", "-pthread", "-I", str(work / "include"), "-o",
                    str(work / "paper_2409_18824_gb300" / "libstencil_host.so"),
                    str(work / "paper_2409_18824_gb300" / "host" / "stencil_host.cpp")], check=True)
    env = dict(os.environ, LD_PRELOAD=f"{asan}:{ubsan}", ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    check = subprocess.run([sys.executable, "-c", "import sys; sys.path.insert(0, '.'); import oracle, "
                            "paper_2409_18824_gb300.host as h; print(oracle._load()._name); print(h.lib()._name)"],
                           cwd=work, env=env, capture_output=True, text=True, timeout=300)
    assert check.returncode == 0, check.stderr[-3000:]
    assert str(work) in check.stdout.splitlines()[0] and str(work) in check.stdout.splitlines()[1]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        *[os.path.join("tests", t) for t in TESTS]],
                       cwd=work, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    assert "passed" in r.stdout and "failed" not in r.stdout


@pytest.mark.slow
def test_gpu_librarys_host_code_is_clean_under_asan_and_ubsan(tmp_path):
    """The host code of libstencil.so that runs without a GPU (argument
    checks, knobs, the launch planners and the plan query, the tuning cache
    and its JSON reader and writer) rebuilt with the sanitizers through nvcc
    (device code unchanged), and the ABI and plan tests run against it.  This
    found a signed overflow in the work-unit count for rejected extents."""
    import concurrent.futures as cf
    asan, ubsan = runtime("libasan.so"), runtime("libubsan.so")
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if not (asan and ubsan and nvcc):
        pytest.skip("nvcc or gcc sanitizer runtimes not available")
    work = tmp_path / "w"
    work.mkdir()
    for d in ("oracle", "stencil_inputs", "include"):
        shutil.copytree(os.path.join(ROOT, d), work / d, ignore=shutil.ignore_patterns("__pycache__"))
    pkg = work / "paper_2409_18824_gb300"
    shutil.copytree(os.path.join(ROOT, "paper_2409_18824_gb300"), pkg,
                    ignore=shutil.ignore_patterns("__pycache__", "_build", "libstencil.so"))
    (work / "tests").mkdir()
    for f in ("conftest.py", "test_abi.py", "test_plan.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), work / "tests" / f)
    flags = ["-gencode", "arch=compute_103a,code=sm_103a", "-O1", "-std=c++17", "--expt-relaxed-constexpr",
             "-Xcompiler", "-fPIC", "-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fsanitize=undefined",
             "-Xcompiler", "-fno-omit-frame-pointer", "-I", str(work / "include"), "-I", str(pkg / "csrc")]
    srcs = sorted(p for p in (pkg / "csrc").iterdir() if p.suffix == ".cu")
    objs = [tmp_path / (p.stem + ".o") for p in srcs]

    def compile_one(pair):
        src, obj = pair
        return subprocess.run([nvcc, *flags, "-c", str(src), "-o", str(obj)], capture_output=True, text=True)

    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        for res in ex.map(compile_one, zip(srcs, objs)):
            assert res.returncode == 0, res.stderr[-3000:]
    link = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-Xcompiler",
                           "-fsanitize=address", "-Xcompiler", "-fsanitize=undefined", "-o",
                           str(pkg / "libstencil.so"), *map(str, objs), "-lpthread"], capture_output=True, text=True)
    assert link.returncode == 0, link.stderr[-3000:]
    env = dict(os.environ, LD_PRELOAD=f"{asan}:{ubsan}",
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=1:protect_shadow_gap=0",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-s", "-p", "no:cacheprovider", "-m", "not gpu",
                        "tests/test_abi.py", "tests/test_plan.py"],
                       cwd=work, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    assert "passed" in r.stdout and "runtime error" not in r.stdout + r.stderr


@pytest.mark.slow
def test_host_library_threads_are_race_free_under_tsan(tmp_path):
    """The multi-core host path's workers and their barrier under gcc's
    ThreadSanitizer: the host-path tests (1 to 64 threads) run against an
    instrumented build, any data race fatal."""
    tsan = runtime("libtsan.so")
    if not (tsan and shutil.which("g++")):
        pytest.skip("gcc thread sanitizer runtime not available")
    work = tmp_path / "w"
    work.mkdir()
    for d in ("oracle", "stencil_inputs", "include", "paper_2409_18824_gb300"):
        shutil.copytree(os.path.join(ROOT, d), work / d, ignore=shutil.ignore_patterns("__pycache__", "_build"))
    (work / "tests").mkdir()
    for f in ("conftest.py", "test_host_path.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), work / "tests" / f)
    subprocess.run(["g++", "-O1", "-g", "-fsanitize=thread", "-ffp-contract=off", "-pthread", "-fPIC", "-shared",
                    "-std=c++17", "-I", str(work / "include"), "-o",
                    str(work / "paper_2409_18824_gb300" / "libstencil_host.so"),
                    str(work / "paper_2409_18824_gb300" / "host" / "stencil_host.cpp")], check=True)
    env = dict(os.environ, LD_PRELOAD=tsan, TSAN_OPTIONS="halt_on_error=1:report_signal_unsafe=0")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-s", "-p", "no:cacheprovider",
                        "tests/test_host_path.py"], cwd=work, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    assert "passed" in r.stdout and "ThreadSanitizer" not in r.stdout + r.stderr
