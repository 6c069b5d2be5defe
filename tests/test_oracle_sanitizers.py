"""The FP64 oracle under AddressSanitizer and UndefinedBehaviorSanitizer:
a C harness (tests/sanitize/oracle_harness.c) drives every entry point on
tiny and ragged lattices and through its argument checks; any sanitizer
report aborts it."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.mark.parametrize("openmp", [False, True])
def test_oracle_is_clean_under_asan_and_ubsan(tmp_path, openmp):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    exe = str(tmp_path / "harness")
    cmd = [gcc, "-std=c99", "-O1", "-g", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-Wno-unknown-pragmas",
           "-I", os.path.join(ROOT, "oracle"), os.path.join(HERE, "sanitize", "oracle_harness.c"),
           os.path.join(ROOT, "oracle", "rclbm_oracle.c"), "-lm", "-o", exe]
    if openmp:
        cmd.insert(1, "-fopenmp")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr and "cannot find" in r.stderr:
        pytest.skip("sanitizer runtimes not installed")
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1", OMP_NUM_THREADS="2")
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
