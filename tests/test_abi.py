"""The C-ABI library builds, loads without a GPU, exports every entry point
the header declares, and its struct layouts match the Python binding."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cdef_gb300.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1602_05975_gb300 import build
    path = build.build()
    return C.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cdef_[a-z_]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("cdef_find_dir", "cdef_filter_frame", "cdef_search_strengths",
              "cdef_ctx_create", "cdef_ctx_destroy", "cdef_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_host_only_calls(lib):
    lib.cdef_strerror.restype = C.c_char_p
    lib.cdef_version.restype = C.c_char_p
    assert lib.cdef_strerror(0) == b"ok"
    assert b"sm_103a" in lib.cdef_version()
    assert lib.cdef_strerror(-2) == b"invalid frame size"


def test_null_arguments_rejected_without_device(lib):
    # argument checks come before any device work
    assert lib.cdef_ctx_create(None, 0, 0) == -1
    assert lib.cdef_find_dir(None, None, 8, None, None, None) == -1
    assert lib.cdef_filter_frame(None, None, None, None, None, None, None) == -1
    assert lib.cdef_ctx_destroy(None) == 0
    # the wait-limit test aid is host state: checked without a device
    lib.cdef_debug_set_waits.argtypes = [C.c_int64, C.c_int32]
    assert lib.cdef_debug_set_waits(-1, 0) == -1
    assert lib.cdef_debug_set_waits(0, -1) == -1
    assert lib.cdef_debug_set_waits(0, 0) == 0
    lib.cdef_probe_int_mix.argtypes = [C.c_void_p, C.c_int32, C.c_int32,
                                       C.POINTER(C.c_double), C.c_void_p]
    r = C.c_double(0.0)
    assert lib.cdef_probe_int_mix(None, 0, 16, C.byref(r), None) == -1


def test_struct_layout_matches_binding(tmp_path):
    from paper_1602_05975_gb300 import cdef
    prog = tmp_path / "layout.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "cdef_gb300.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu\\n\","
        "sizeof(cdef_plane), sizeof(cdef_frame), offsetof(cdef_frame, bitdepth),"
        "sizeof(cdef_fb_params), offsetof(cdef_fb_params, damping), sizeof(cdef_preset),"
        "offsetof(cdef_plane, pitch_bytes));return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert vals == [C.sizeof(cdef.Plane), C.sizeof(cdef.FrameDesc),
                    cdef.FrameDesc.bitdepth.offset, 8, 4, C.sizeof(cdef.Preset),
                    cdef.Plane.pitch_bytes.offset]


def test_binding_fails_loudly_without_library(monkeypatch):
    from paper_1602_05975_gb300 import cdef
    monkeypatch.setattr(cdef, "_lib", None)
    monkeypatch.setattr(cdef, "LIB_PATH", "/nonexistent/libcdef_gb300.so")
    with pytest.raises(RuntimeError):
        cdef.load()


def test_frame_descriptor_follows_the_planes():
    """The descriptor kept on a frame is rebuilt when a plane, its pitch or
    a field of the frame changes (a stale pointer would reach the device)."""
    torch = pytest.importorskip("torch")
    from paper_1602_05975_gb300 import cdef
    f = cdef.alloc_frame(128, 64, 8, device="cpu")
    d0 = f.desc()
    assert f.desc() is d0
    assert d0.y.data == f.y.data_ptr() and d0.y.width == 128 and d0.u.height == 32
    f.y = torch.zeros_like(f.y)
    d1 = f.desc()
    assert d1 is not d0 and d1.y.data == f.y.data_ptr()
    f.bitdepth = 10
    assert f.desc().bitdepth == 10
    wide = torch.zeros((64, 256), dtype=f.y.dtype)[:, :160]
    f.y = wide
    assert f.desc().y.pitch_bytes == 256 * wide.element_size()


def test_search_results_parsed_per_frame():
    """Host-side parsing of the search's preset arrays: eight presets per
    frame, the first four (or, with the skip bits, five) bytes of each."""
    pytest.importorskip("torch")
    from paper_1602_05975_gb300 import cdef
    p = (cdef.Preset * 16)()
    for i in range(16):
        p[i].pri_y, p[i].sec_y, p[i].pri_uv, p[i].sec_uv = i, 1, 2, 3
    out = cdef._search_results(p, 4, 2, [3, 8], [10, 20])
    assert out[1]["presets"][0] == (8, 1, 2, 3) and len(out[0]["presets"]) == 8
    assert (out[0]["npresets"], out[1]["cost"]) == (3, 20)
    q = (cdef.PresetCoded * 8)()
    q[5].pri_y, q[5].skip, q[5].reserved[0] = 7, 3, 9
    out = cdef._search_results(q, 5, 1, [8], [0])
    assert out[0]["presets"][5] == (7, 0, 0, 0, 3)
