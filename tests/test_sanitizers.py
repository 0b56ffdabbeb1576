"""Host code under AddressSanitizer and UndefinedBehaviorSanitizer (no GPU).

The oracle's C source is built with -fsanitize=address,undefined into a temporary
library and the pin suite runs against it; the library's translation units are
built the same way (host code instrumented, device code unchanged) and the CPU
ABI and host tests run against that copy.  Any out-of-bounds access, use after
free, signed overflow or other undefined behaviour aborts the run.

Opt-in (about four minutes): EGN_RUN_SANITIZERS=1 python -m pytest tests/test_sanitizers.py
"""
import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "egn_oracle.c")


def _runtime(name):
    out = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
    return out if os.path.isabs(out) and os.path.exists(out) else None


@pytest.mark.skipif(os.environ.get("EGN_RUN_SANITIZERS") != "1", reason="opt-in: EGN_RUN_SANITIZERS=1")
def test_oracle_pins_under_asan_ubsan():
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not (asan and ubsan):
        pytest.skip("gcc sanitizer runtimes not found")
    with tempfile.TemporaryDirectory() as td:
        so = os.path.join(td, "liboracle_san.so")
        subprocess.run(["gcc", "-O1", "-g", "-std=c11", "-fPIC", "-shared", "-fno-omit-frame-pointer",
                        "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-o", so, SRC, "-lm"],
                       check=True, capture_output=True)
        env = dict(os.environ, EGN_ORACLE_LIB=so, LD_PRELOAD=f"{asan} {ubsan}", ASAN_OPTIONS="detect_leaks=0",
                   UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1", EGN_RUN_SANITIZERS="0")
        pins = [os.path.join(ROOT, "tests", f) for f in
                ("test_oracle_isrs.py", "test_oracle_mu.py", "test_oracle_islands.py", "test_oracle_egn.py",
                 "test_oracle_3d.py")]
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] + pins,
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
        assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]


@pytest.mark.skipif(os.environ.get("EGN_RUN_SANITIZERS") != "1", reason="opt-in: EGN_RUN_SANITIZERS=1")
def test_library_host_code_under_asan_ubsan():
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not (asan and ubsan):
        pytest.skip("gcc sanitizer runtimes not found")
    sys.path.insert(0, ROOT)
    from paper_2412_11614_gb300 import _build
    san = "-fPIC,-fsanitize=address,-fsanitize=undefined,-fno-sanitize-recover=undefined,-fno-omit-frame-pointer"
    with tempfile.TemporaryDirectory() as td:
        def compile_one(src):
            obj = os.path.join(td, os.path.basename(src) + ".o")
            subprocess.run([_build.nvcc(), *_build.ARCH, "-O1", "-std=c++17", "--extended-lambda", "-Xcompiler", san,
                            "-c", src, "-o", obj], check=True, capture_output=True)
            return obj
        with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
            objs = list(ex.map(compile_one, _build.sources()))
        so = os.path.join(td, "libegn_san.so")
        subprocess.run([_build.nvcc(), *_build.ARCH, "-shared", "-Xcompiler", san, "-o", so, *objs,
                        "-lcudart_static", "-lrt", "-ldl", "-lpthread"], check=True, capture_output=True)
        with open(os.path.join(td, "egn_sanitized_lib.py"), "w") as f:  # pytest plugin: load the copy
            f.write("import paper_2412_11614_gb300._build as B\nimport paper_2412_11614_gb300.egn as E\n"
                    f"B.build = lambda *a, **k: {so!r}\nE.library_path = lambda: {so!r}\n")
        env = dict(os.environ, PYTHONPATH=td + os.pathsep + ROOT, LD_PRELOAD=f"{asan} {ubsan}",
                   ASAN_OPTIONS="detect_leaks=0:protect_shadow_gap=0", UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1",
                   EGN_RUN_SANITIZERS="0")
        tests = [os.path.join(ROOT, "tests", f) for f in ("test_abi.py", "test_surrogate_host.py")]
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            "-p", "egn_sanitized_lib", "-k", "not in_tree"] + tests,
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
        assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
