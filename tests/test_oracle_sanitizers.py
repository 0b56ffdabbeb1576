"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer: its C source is
built with -fsanitize=address,undefined into a temporary library and the pin
suite runs against it (any out-of-bounds access, use after free, signed overflow
or other undefined behaviour aborts the run).

Opt-in (about two minutes): EGN_RUN_SANITIZERS=1 python -m pytest tests/test_oracle_sanitizers.py
"""
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
