"""The CPU oracle under AddressSanitizer and UndefinedBehaviorSanitizer: a
C++ driver (tests/oracle_sanitize_main.cpp) runs every exported oracle
function on small seeded inputs -- empty, single-key, ragged, duplicate-heavy,
both key widths, both bucket maps -- and cross-checks the results.  An
out-of-bounds access, a use of uninitialised or freed memory, or an undefined
operation (signed overflow, an oversized shift) in the oracle fails the test,
so the parity tests compare the GPU against a reference without such faults."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_runs_clean_under_sanitizers(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "oracle_sanitized")
    srcs = [os.path.join(ROOT, "tests", "oracle_sanitize_main.cpp"),
            os.path.join(ROOT, "oracle", "hg_oracle.cpp"), os.path.join(ROOT, "oracle", "hg_oracle_learned.cpp")]
    cmd = [cxx, "-std=c++17", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
           "-fno-omit-frame-pointer", "-ffp-contract=off", "-fno-fast-math", "-o", exe] + srcs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and ("asan" in r.stderr or "ubsan" in r.stderr):
        pytest.skip("sanitizer runtimes not available: " + r.stderr.strip().splitlines()[-1])
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "runtime error" not in run.stderr and "ERROR: AddressSanitizer" not in run.stderr, run.stderr
    assert "oracle checks passed" in run.stdout
