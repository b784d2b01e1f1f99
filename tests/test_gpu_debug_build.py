"""The index-checking build of the CUDA library against the parity tests.

libcdef_gb300_debug.so (build(debug=True)) checks every shared-memory tap
load, output staging write and 16-byte row store of the filter and search
kernels before it is made.  The parity tests below run in a child process on
that library (CDEF_GB300_LIBRARY) with CDEF_EXPECT_INDEX_CHECKS=1, which makes
tests/conftest.py read the device's fault count after every test: they must
stay bit-exact against the oracle and no access may have been out of range.
The sizes cover ragged frame edges, 8x8 and single-row frames, every chroma
format and bit depth, coded maps, both metrics and every launch
configuration of the search.
"""
import os
import re
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# the parity tests that run on the checking library (the largest frames and
# the fuzz loops stay on the release library: same kernels, more oracle time)
SELECTION = ("find_dir or filter_parity or filter_every_strength or filter_extreme "
             "or filter_batch_mixed or filter_coded or filter_chroma_formats "
             "or search_parity or search_every_launch or search_preset_refinement "
             "or search_coded_parity or search_eq14 or search_formats or search_subset "
             "or search_coded_formats or search_444 or filter_444 or consecutive_frames "
             "or filter_rounds")


@pytest.fixture(scope="module")
def debug_lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1602_05975_gb300 import build
    build.build()
    return build.build(debug=True)


def test_library_reports_its_checks(debug_lib):
    """The checking library says so; the release library says it does not."""
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_1602_05975_gb300 import cdef\n"
            "c = cdef.Context(0)\n"
            "print(cdef.debug_checks(c))\n") % ROOT
    for lib, want in ((debug_lib, "(True, 0)"), ("", "(False, 0)")):
        env = dict(os.environ, CDEF_GB300_LIBRARY=lib)
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                           text=True, timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        assert r.stdout.strip().splitlines()[-1] == want


def test_parity_suite_on_checking_build(debug_lib):
    env = dict(os.environ, CDEF_GB300_LIBRARY=debug_lib, CDEF_EXPECT_INDEX_CHECKS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join("tests", "test_gpu_parity.py"),
                        "-m", "gpu", "-q", "-x", "-p", "no:cacheprovider", "-k", SELECTION],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = r.stdout[-3000:] + r.stderr[-2000:]
    assert r.returncode == 0, tail
    m = re.search(r"(\d+) passed", r.stdout)
    assert m and "failed" not in r.stdout, tail
    # every selected parity test ran (none skipped away)
    assert int(m.group(1)) >= 80, tail
