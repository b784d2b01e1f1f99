import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def ref():
    from oracle import ref as _ref
    _ref.lib()
    return _ref


_checks_ctx = []


@pytest.fixture(autouse=True)
def _no_index_faults():
    """With CDEF_EXPECT_INDEX_CHECKS=1 (set by tests/test_gpu_debug_build.py
    for the parity tests it runs on the index-checking library): after every
    test that loaded the CUDA library, that library must be the checking
    build and its kernels must have skipped no access out of range."""
    yield
    if os.environ.get("CDEF_EXPECT_INDEX_CHECKS") != "1":
        return
    mod = sys.modules.get("paper_1602_05975_gb300.cdef")
    if mod is None or mod._lib is None:
        return
    if not _checks_ctx:
        _checks_ctx.append(mod.Context(0))
    checked, faults = mod.debug_checks(_checks_ctx[0], clear=True)
    assert checked, f"{mod.library_path()} was built without index checks"
    assert faults == 0, f"kernels skipped {faults} out-of-range accesses"
