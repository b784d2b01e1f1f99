"""The CPU oracle under AddressSanitizer and UndefinedBehaviorSanitizer.

tests/oracle_sanitized.c calls every oracle entry point on small frames of
every bit depth and chroma format, with buffers of exactly the sizes the
calls are documented to use; built here with gcc's sanitizers (aborting on
the first report), it must run to completion.  This checks the oracle's
memory accesses and integer arithmetic, not its values (the pins do that).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_clean_under_asan_and_ubsan(tmp_path):
    if not shutil.which("gcc"):
        pytest.skip("gcc not found")
    exe = tmp_path / "oracle_sanitized"
    r = subprocess.run(["gcc", "-std=c99", "-O1", "-g", "-fno-omit-frame-pointer", "-ffp-contract=off",
                        "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
                        "-I", os.path.join(ROOT, "oracle"), os.path.join(ROOT, "tests", "oracle_sanitized.c"),
                        os.path.join(ROOT, "oracle", "cdef_ref.c"), "-lm", "-o", str(exe)],
                       capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr and "not supported" in r.stderr:
        pytest.skip("sanitizers not available")
    assert r.returncode == 0, r.stderr[-3000:]
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=900, env=env)
    assert run.returncode == 0, (run.stdout[-2000:] + run.stderr[-4000:])
    assert "nothing reported" in run.stdout
