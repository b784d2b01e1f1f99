"""Python access to the plain-C CDEF oracle (``oracle/cdef_ref.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  The CUDA
library never calls it; it shares no code with it.

The oracle is compiled with gcc by :func:`build` into ``oracle/libcdef_ref.so``.
All arrays are numpy; samples are passed as uint16 whatever the bit depth.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cdef_ref.c")
_LIB = os.path.join(_HERE, "libcdef_ref.so")
_lib = None

_u16p = np.ctypeslib.ndpointer(np.uint16, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")


class EffParams(C.Structure):
    _fields_ = [("pri", C.c_int64), ("sec", C.c_int64),
                ("damping", C.c_int64), ("parity", C.c_int)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no vectorisation flags; -O2 only;
    floating-point expressions evaluated as written: no fused multiply-add
    contraction, on any host)."""
    stale = (not os.path.exists(_LIB)
             or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
             or os.path.getmtime(_LIB) < os.path.getmtime(os.path.join(_HERE, "cdef_ref.h")))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        path = os.environ.get("CDEF_REF_LIB")  # a planted-mistake copy (tests)
        if not path:
            path = build()
        L = C.CDLL(path)
        L.cdef_ref_line_number.argtypes = [C.c_int, C.c_int, C.c_int]
        L.cdef_ref_line_number.restype = C.c_int
        L.cdef_ref_direction_costs.argtypes = [_i32p, _i64p]
        L.cdef_ref_direction_costs.restype = None
        L.cdef_ref_find_dir_block.argtypes = [_u16p, C.c_ssize_t, C.c_int,
                                              C.POINTER(C.c_int64)]
        L.cdef_ref_find_dir_block.restype = C.c_int
        L.cdef_ref_find_dir.argtypes = [_u16p, C.c_int, C.c_int, C.c_ssize_t,
                                        C.c_int, _u8p, _i32p]
        L.cdef_ref_find_dir.restype = C.c_int
        L.cdef_ref_constrain.argtypes = [C.c_int64, C.c_int64, C.c_int64]
        L.cdef_ref_constrain.restype = C.c_int64
        L.cdef_ref_adjust_strength.argtypes = [C.c_int, C.c_int64]
        L.cdef_ref_adjust_strength.restype = C.c_int
        L.cdef_ref_round16.argtypes = [C.c_int64]
        L.cdef_ref_round16.restype = C.c_int64
        L.cdef_ref_block_params.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int,
                                            C.c_int, C.c_int64,
                                            C.POINTER(EffParams)]
        L.cdef_ref_block_params.restype = None
        L.cdef_ref_filter_sample.argtypes = [_u16p, C.c_int, C.c_int,
                                             C.c_ssize_t, C.c_int, C.c_int,
                                             C.c_int, C.POINTER(EffParams)]
        L.cdef_ref_filter_sample.restype = C.c_int64
        L.cdef_ref_filter_frame.argtypes = (
            [C.c_int, C.c_int, C.c_int] + [_u16p, C.c_ssize_t] * 3
            + [_u8p, _u8p, _i32p] + [_u16p, C.c_ssize_t] * 3)
        L.cdef_ref_filter_frame.restype = C.c_int
        L.cdef_ref_filter_frame_coded.argtypes = (
            [C.c_int, C.c_int, C.c_int] + [_u16p, C.c_ssize_t] * 3
            + [_u8p, C.c_void_p, _u8p, _i32p] + [_u16p, C.c_ssize_t] * 3)
        L.cdef_ref_filter_frame_coded.restype = C.c_int
        L.cdef_ref_filter_frame_format.argtypes = (
            [C.c_int, C.c_int, C.c_int, C.c_int] + [_u16p, C.c_ssize_t] * 3
            + [_u8p, C.c_void_p, _u8p, _i32p] + [_u16p, C.c_ssize_t] * 3)
        L.cdef_ref_filter_frame_format.restype = C.c_int
        L.cdef_ref_distortion.argtypes = (
            [C.c_int, C.c_int, C.c_int, C.c_int] + [_u16p, C.c_ssize_t] * 6
            + [_i64p, _i64p])
        L.cdef_ref_distortion.restype = C.c_int
        L.cdef_ref_select_presets.argtypes = [
            C.c_int, _i64p, _i64p, C.c_int64, _i32p, C.POINTER(C.c_int32),
            _u8p, C.POINTER(C.c_int64), _i64p]
        L.cdef_ref_select_presets.restype = C.c_int
        L.cdef_ref_refine_presets.argtypes = [
            C.c_int, _i64p, _i64p, _i32p, C.c_int, C.c_int, C.POINTER(C.c_int64),
            C.POINTER(C.c_int)]
        L.cdef_ref_refine_presets.restype = C.c_int
        L.cdef_ref_select_presets_refined.argtypes = [
            C.c_int, _i64p, _i64p, C.c_int64, C.c_int, _i32p, C.POINTER(C.c_int32),
            _u8p, C.POINTER(C.c_int64)]
        L.cdef_ref_select_presets_refined.restype = C.c_int
        L.cdef_ref_distortion_coded.argtypes = (
            [C.c_int, C.c_int, C.c_int, C.c_int] + [_u16p, C.c_ssize_t] * 6
            + [C.c_void_p, _i64p, _i64p, _u8p])
        L.cdef_ref_distortion_coded.restype = C.c_int
        L.cdef_ref_select_presets_general.argtypes = [
            C.c_int, _i64p, _i64p, C.c_int, C.c_void_p, C.c_int64, C.c_int, _i32p,
            C.POINTER(C.c_int32), _u8p, C.POINTER(C.c_int64)]
        L.cdef_ref_select_presets_general.restype = C.c_int
        L.cdef_ref_select_presets_subset.argtypes = [
            C.c_int, _i64p, _i64p, C.c_int, C.c_void_p, C.c_uint64, C.c_uint64, C.c_int64,
            C.c_int, _i32p, C.POINTER(C.c_int32), _u8p, C.POINTER(C.c_int64)]
        L.cdef_ref_select_presets_subset.restype = C.c_int
        L.cdef_ref_distortion_format.argtypes = (
            [C.c_int] * 5 + [_u16p, C.c_ssize_t] * 6 + [_i64p, _i64p])
        L.cdef_ref_distortion_format.restype = C.c_int
        L.cdef_ref_distortion_coded_format.argtypes = (
            [C.c_int] * 5 + [_u16p, C.c_ssize_t] * 6 + [C.c_void_p, _i64p, _i64p, _u8p])
        L.cdef_ref_distortion_coded_format.restype = C.c_int
        L.cdef_ref_distortion_eq14.argtypes = (
            [C.c_int, C.c_int, C.c_int, C.c_int] + [_u16p, C.c_ssize_t] * 6 + [_i64p, _i64p])
        L.cdef_ref_distortion_eq14.restype = C.c_int
        L.cdef_ref_distortion_eq14_format.argtypes = (
            [C.c_int] * 5 + [_u16p, C.c_ssize_t] * 6 + [_i64p, _i64p])
        L.cdef_ref_distortion_eq14_format.restype = C.c_int
        L.cdef_ref_distortion_eq14_coded_format.argtypes = (
            [C.c_int] * 5 + [_u16p, C.c_ssize_t] * 6 + [C.c_void_p, _i64p, _i64p, _u8p])
        L.cdef_ref_distortion_eq14_coded_format.restype = C.c_int
        L.cdef_ref_eq14_term.argtypes = [C.c_int64] * 6 + [C.c_int]
        L.cdef_ref_eq14_term.restype = C.c_int64
        _lib = L
    return _lib


def _u16(a):
    return np.ascontiguousarray(a, dtype=np.uint16)


# ---------------------------------------------------------------- scalar API
def line_number(d: int, i: int, j: int) -> int:
    return lib().cdef_ref_line_number(d, i, j)


def direction_costs(x64) -> np.ndarray:
    """840 * s_d for d = 0..7 of a centred 8x8 block (Algorithm 1)."""
    x = np.ascontiguousarray(np.asarray(x64, dtype=np.int32).reshape(64))
    s = np.zeros(8, np.int64)
    lib().cdef_ref_direction_costs(x, s)
    return s


def find_dir_block(block, bitdepth: int = 8):
    b = _u16(block)
    v = C.c_int64(0)
    d = lib().cdef_ref_find_dir_block(b, b.shape[1], bitdepth, C.byref(v))
    return d, v.value


def constrain(diff: int, strength: int, damping: int) -> int:
    return lib().cdef_ref_constrain(diff, strength, damping)


def adjust_strength(strength: int, contrast: int) -> int:
    return lib().cdef_ref_adjust_strength(strength, contrast)


def round16(s: int) -> int:
    return lib().cdef_ref_round16(s)


def block_params(pri, sec, damping, is_chroma, bitdepth, contrast=0):
    e = EffParams()
    lib().cdef_ref_block_params(pri, sec, damping, int(is_chroma), bitdepth,
                                contrast, C.byref(e))
    return e


def filter_sample(plane, i, j, d, eff: EffParams) -> int:
    p = _u16(plane)
    h, w = p.shape
    return lib().cdef_ref_filter_sample(p, w, h, w, i, j, d, C.byref(eff))


# ----------------------------------------------------------------- frame API
def find_dir(luma, bitdepth: int):
    y = _u16(luma)
    h, w = y.shape
    dirs = np.zeros((h // 8, w // 8), np.uint8)
    var = np.zeros((h // 8, w // 8), np.int32)
    if lib().cdef_ref_find_dir(y, w, h, w, bitdepth, dirs, var) != 0:
        raise ValueError("oracle rejected find_dir arguments")
    return dirs, var


def filter_frame(y, u, v, bitdepth: int, params, dirs=None, var=None, coded=None):
    """Filter a 4:2:0 frame.  params: uint8 array (fb_rows, fb_cols, 8);
    coded: optional (h/8, w/8) array, nonzero where the 8x8 block has coded
    residual (section 4 skip semantics; None = all coded)."""
    y, u, v = _u16(y), _u16(u), _u16(v)
    h, w = y.shape
    if dirs is None:
        dirs, var = find_dir(y, bitdepth)
    prm = np.ascontiguousarray(params, dtype=np.uint8)
    cod = None if coded is None else np.ascontiguousarray(coded, dtype=np.uint8)
    if cod is not None and cod.shape != (h // 8, w // 8):
        raise ValueError("coded map shape")
    oy, ou, ov = np.zeros_like(y), np.zeros_like(u), np.zeros_like(v)
    rc = lib().cdef_ref_filter_frame_coded(
        w, h, bitdepth, y, w, u, u.shape[1], v, v.shape[1],
        prm.reshape(-1), None if cod is None else cod.ctypes.data,
        np.ascontiguousarray(dirs, np.uint8).reshape(-1),
        np.ascontiguousarray(var, np.int32).reshape(-1),
        oy, w, ou, ou.shape[1], ov, ov.shape[1])
    if rc != 0:
        raise ValueError("oracle rejected filter_frame arguments")
    return oy, ou, ov


def distortion(rec, src, bitdepth: int, damping: int):
    """Per filter block, 64 luma and 64 chroma SSE values (section 5)."""
    ry, ru, rv = (_u16(p) for p in rec)
    sy, su, sv = (_u16(p) for p in src)
    h, w = ry.shape
    nb = ((h + 63) // 64) * ((w + 63) // 64)
    dl = np.zeros(nb * 64, np.int64)
    dc = np.zeros(nb * 64, np.int64)
    rc = lib().cdef_ref_distortion(
        w, h, bitdepth, damping, ry, w, ru, ru.shape[1], rv, rv.shape[1],
        sy, w, su, su.shape[1], sv, sv.shape[1], dl, dc)
    if rc != 0:
        raise ValueError("oracle rejected distortion arguments")
    return dl.reshape(nb, 64), dc.reshape(nb, 64)


def select_presets(dist_luma, dist_chroma, lam: int):
    dl = np.ascontiguousarray(dist_luma, np.int64).reshape(-1)
    dc = np.ascontiguousarray(dist_chroma, np.int64).reshape(-1)
    nb = dl.size // 64
    presets = np.zeros(8, np.int32)
    n = C.c_int32(0)
    ids = np.zeros(nb, np.uint8)
    cost = C.c_int64(0)
    costs = np.zeros(8, np.int64)
    rc = lib().cdef_ref_select_presets(nb, dl, dc, lam, presets, C.byref(n),
                                       ids, C.byref(cost), costs)
    if rc != 0:
        raise ValueError("oracle rejected select_presets arguments")
    return dict(presets=presets, npresets=n.value, block_ids=ids,
                cost=cost.value, costs=costs)


def refine_presets(dist_luma, dist_chroma, presets, max_passes: int):
    """Section 5: re-optimise one preset at a time (reading R17)."""
    dl = np.ascontiguousarray(dist_luma, np.int64).reshape(-1)
    dc = np.ascontiguousarray(dist_chroma, np.int64).reshape(-1)
    p = np.ascontiguousarray(presets, np.int32).copy()
    total = C.c_int64(0)
    passes = C.c_int(0)
    if lib().cdef_ref_refine_presets(dl.size // 64, dl, dc, p, p.size, max_passes,
                                     C.byref(total), C.byref(passes)) != 0:
        raise ValueError("oracle rejected refine_presets arguments")
    return p, total.value, passes.value


def select_presets_refined(dist_luma, dist_chroma, lam: int, max_passes: int):
    dl = np.ascontiguousarray(dist_luma, np.int64).reshape(-1)
    dc = np.ascontiguousarray(dist_chroma, np.int64).reshape(-1)
    nb = dl.size // 64
    presets = np.zeros(8, np.int32)
    n = C.c_int32(0)
    ids = np.zeros(nb, np.uint8)
    cost = C.c_int64(0)
    if lib().cdef_ref_select_presets_refined(nb, dl, dc, lam, max_passes, presets, C.byref(n),
                                             ids, C.byref(cost)) != 0:
        raise ValueError("oracle rejected select_presets_refined arguments")
    return dict(presets=presets, npresets=n.value, block_ids=ids, cost=cost.value)


def search_strengths(rec, src, bitdepth: int, damping: int, lam: int, refine_passes: int = 0):
    dl, dc = distortion(rec, src, bitdepth, damping)
    if refine_passes:
        out = select_presets_refined(dl, dc, lam, refine_passes)
    else:
        out = select_presets(dl, dc, lam)
    out["dist_luma"] = dl
    out["dist_chroma"] = dc
    return out


def distortion_coded(rec, src, bitdepth: int, damping: int, coded=None):
    """Section 5 with section 4's skip semantics (reading R21): per filter
    block 128 luma and 128 chroma SSE values, and the skipped-block flags."""
    ry, ru, rv = (_u16(p) for p in rec)
    sy, su, sv = (_u16(p) for p in src)
    h, w = ry.shape
    nb = ((h + 63) // 64) * ((w + 63) // 64)
    cod = None if coded is None else np.ascontiguousarray(coded, dtype=np.uint8)
    dl = np.zeros(nb * 128, np.int64)
    dc = np.zeros(nb * 128, np.int64)
    sk = np.zeros(nb, np.uint8)
    rc = lib().cdef_ref_distortion_coded(
        w, h, bitdepth, damping, ry, w, ru, ru.shape[1], rv, rv.shape[1],
        sy, w, su, su.shape[1], sv, sv.shape[1], None if cod is None else cod.ctypes.data,
        dl, dc, sk)
    if rc != 0:
        raise ValueError("oracle rejected distortion_coded arguments")
    return dl.reshape(nb, 128), dc.reshape(nb, 128), sk


def select_presets_general(dist_luma, dist_chroma, width: int, skipped, lam: int,
                           max_passes: int = 0):
    dl = np.ascontiguousarray(dist_luma, np.int64).reshape(-1)
    dc = np.ascontiguousarray(dist_chroma, np.int64).reshape(-1)
    nb = dl.size // width
    sk = None if skipped is None else np.ascontiguousarray(skipped, np.uint8)
    presets = np.zeros(8, np.int32)
    n = C.c_int32(0)
    ids = np.zeros(nb, np.uint8)
    cost = C.c_int64(0)
    if lib().cdef_ref_select_presets_general(nb, dl, dc, width,
                                             None if sk is None else sk.ctypes.data, lam,
                                             max_passes, presets, C.byref(n), ids,
                                             C.byref(cost)) != 0:
        raise ValueError("oracle rejected select_presets_general arguments")
    return dict(presets=presets, npresets=n.value, block_ids=ids, cost=cost.value)


def distortion_format(rec, src, bitdepth: int, damping: int, fmt: int):
    """Section 5's tables for chroma format 420, 422 or 444 (reading R25),
    any bit depth: (B, 64) luma and chroma int64 arrays."""
    ry, ru, rv = (_u16(p) for p in rec)
    sy, su, sv = (_u16(p) for p in src)
    h, w = ry.shape
    nb = ((h + 63) // 64) * ((w + 63) // 64)
    dl = np.zeros(nb * 64, np.int64)
    dc = np.zeros(nb * 64, np.int64)
    rc = lib().cdef_ref_distortion_format(
        w, h, bitdepth, damping, fmt, ry, w, ru, ru.shape[1], rv, rv.shape[1],
        sy, w, su, su.shape[1], sv, sv.shape[1], dl, dc)
    if rc != 0:
        raise ValueError("oracle rejected distortion_format arguments")
    return dl.reshape(nb, 64), dc.reshape(nb, 64)


def distortion_coded_format(rec, src, bitdepth: int, damping: int, fmt: int, coded=None):
    """The 128-combination tables (reading R21) for chroma format 420, 422
    or 444 at any bit depth, and the skipped-block flags."""
    ry, ru, rv = (_u16(p) for p in rec)
    sy, su, sv = (_u16(p) for p in src)
    h, w = ry.shape
    nb = ((h + 63) // 64) * ((w + 63) // 64)
    cod = None if coded is None else np.ascontiguousarray(coded, dtype=np.uint8)
    dl = np.zeros(nb * 128, np.int64)
    dc = np.zeros(nb * 128, np.int64)
    sk = np.zeros(nb, np.uint8)
    rc = lib().cdef_ref_distortion_coded_format(
        w, h, bitdepth, damping, fmt, ry, w, ru, ru.shape[1], rv, rv.shape[1],
        sy, w, su, su.shape[1], sv, sv.shape[1], None if cod is None else cod.ctypes.data,
        dl, dc, sk)
    if rc != 0:
        raise ValueError("oracle rejected distortion_coded_format arguments")
    return dl.reshape(nb, 128), dc.reshape(nb, 128), sk


def search_strengths_coded_format(rec, src, bitdepth: int, damping: int, lam: int, fmt: int,
                                  coded=None, refine_passes: int = 0):
    dl, dc, sk = distortion_coded_format(rec, src, bitdepth, damping, fmt, coded)
    out = select_presets_general(dl, dc, 128, sk, lam, refine_passes)
    out.update(dist_luma=dl, dist_chroma=dc, skipped=sk)
    return out


def search_strengths_format(rec, src, bitdepth: int, damping: int, lam: int, fmt: int,
                            refine_passes: int = 0):
    dl, dc = distortion_format(rec, src, bitdepth, damping, fmt)
    out = select_presets_general(dl, dc, 64, None, lam, refine_passes)
    out.update(dist_luma=dl, dist_chroma=dc)
    return out


def select_presets_subset(dist_luma, dist_chroma, width: int, skipped, luma_pairs: int,
                          chroma_pairs: int, lam: int, max_passes: int = 0):
    """Reading R26: the selection over presets whose luma and chroma
    (S_p, S_s) pairs are allowed by the two 64-bit masks."""
    dl = np.ascontiguousarray(dist_luma, np.int64).reshape(-1)
    dc = np.ascontiguousarray(dist_chroma, np.int64).reshape(-1)
    nb = dl.size // width
    sk = None if skipped is None else np.ascontiguousarray(skipped, np.uint8)
    presets = np.zeros(8, np.int32)
    n = C.c_int32(0)
    ids = np.zeros(nb, np.uint8)
    cost = C.c_int64(0)
    if lib().cdef_ref_select_presets_subset(nb, dl, dc, width,
                                            None if sk is None else sk.ctypes.data,
                                            luma_pairs, chroma_pairs, lam, max_passes, presets,
                                            C.byref(n), ids, C.byref(cost)) != 0:
        raise ValueError("oracle rejected select_presets_subset arguments")
    return dict(presets=presets, npresets=n.value, block_ids=ids, cost=cost.value)


def search_strengths_subset(rec, src, bitdepth: int, damping: int, lam: int, luma_pairs: int,
                            chroma_pairs: int, refine_passes: int = 0, coded=None,
                            metric: str = "sse"):
    """The low-complexity search: full tables (squared error, eq. 14, or the
    128 combinations when `coded` is given), selection over the subset."""
    sk = None
    if coded is not None:
        dl, dc, sk = distortion_coded(rec, src, bitdepth, damping, coded)
        width = 128
    elif metric == "eq14":
        dl, dc = distortion_eq14(rec, src, bitdepth, damping)
        width = 64
    else:
        dl, dc = distortion(rec, src, bitdepth, damping)
        width = 64
    out = select_presets_subset(dl, dc, width, sk, luma_pairs, chroma_pairs, lam, refine_passes)
    out.update(dist_luma=dl, dist_chroma=dc, skipped=sk)
    return out


def search_strengths_coded(rec, src, bitdepth: int, damping: int, lam: int, coded=None,
                           refine_passes: int = 0):
    dl, dc, sk = distortion_coded(rec, src, bitdepth, damping, coded)
    out = select_presets_general(dl, dc, 128, sk, lam, refine_passes)
    out.update(dist_luma=dl, dist_chroma=dc, skipped=sk)
    return out


def filter_frame_format(y, u, v, bitdepth: int, params, fmt: int, coded=None):
    """The filter for chroma format 420, 422 or 444 (reading R25)."""
    y, u, v = _u16(y), _u16(u), _u16(v)
    h, w = y.shape
    dirs, var = find_dir(y, bitdepth)
    prm = np.ascontiguousarray(params, dtype=np.uint8)
    cod = None if coded is None else np.ascontiguousarray(coded, dtype=np.uint8)
    oy, ou, ov = np.zeros_like(y), np.zeros_like(u), np.zeros_like(v)
    rc = lib().cdef_ref_filter_frame_format(
        w, h, bitdepth, fmt, y, w, u, u.shape[1], v, v.shape[1], prm.reshape(-1),
        None if cod is None else cod.ctypes.data, np.ascontiguousarray(dirs, np.uint8).reshape(-1),
        np.ascontiguousarray(var, np.int32).reshape(-1), oy, w, ou, ou.shape[1], ov, ov.shape[1])
    if rc != 0:
        raise ValueError("oracle rejected filter_frame_format arguments")
    return oy, ou, ov


def distortion_eq14(rec, src, bitdepth: int, damping: int):
    """Section 5, eq. 14 (readings R22-R24): per filter block 64 luma and 64
    chroma entries, each the sum over 8x8 blocks of round(256 * D_8x8)."""
    ry, ru, rv = (_u16(p) for p in rec)
    sy, su, sv = (_u16(p) for p in src)
    h, w = ry.shape
    nb = ((h + 63) // 64) * ((w + 63) // 64)
    dl = np.zeros(nb * 64, np.int64)
    dc = np.zeros(nb * 64, np.int64)
    rc = lib().cdef_ref_distortion_eq14(
        w, h, bitdepth, damping, ry, w, ru, ru.shape[1], rv, rv.shape[1],
        sy, w, su, su.shape[1], sv, sv.shape[1], dl, dc)
    if rc != 0:
        raise ValueError("oracle rejected distortion_eq14 arguments")
    return dl.reshape(nb, 64), dc.reshape(nb, 64)


def distortion_eq14_format(rec, src, bitdepth: int, damping: int, fmt: int):
    """Eq. 14 tables for chroma format 420, 422 or 444 (readings R22-R25)."""
    ry, ru, rv = (_u16(p) for p in rec)
    sy, su, sv = (_u16(p) for p in src)
    h, w = ry.shape
    nb = ((h + 63) // 64) * ((w + 63) // 64)
    dl = np.zeros(nb * 64, np.int64)
    dc = np.zeros(nb * 64, np.int64)
    rc = lib().cdef_ref_distortion_eq14_format(
        w, h, bitdepth, damping, fmt, ry, w, ru, ru.shape[1], rv, rv.shape[1],
        sy, w, su, su.shape[1], sv, sv.shape[1], dl, dc)
    if rc != 0:
        raise ValueError("oracle rejected distortion_eq14_format arguments")
    return dl.reshape(nb, 64), dc.reshape(nb, 64)


def distortion_eq14_coded_format(rec, src, bitdepth: int, damping: int, fmt: int, coded=None):
    """Eq. 14 tables of the 128 combinations (readings R21-R25): per filter
    block 128 luma and 128 chroma entries and a skipped flag."""
    ry, ru, rv = (_u16(p) for p in rec)
    sy, su, sv = (_u16(p) for p in src)
    h, w = ry.shape
    nb = ((h + 63) // 64) * ((w + 63) // 64)
    cod = None if coded is None else np.ascontiguousarray(coded, dtype=np.uint8)
    dl = np.zeros(nb * 128, np.int64)
    dc = np.zeros(nb * 128, np.int64)
    sk = np.zeros(nb, np.uint8)
    rc = lib().cdef_ref_distortion_eq14_coded_format(
        w, h, bitdepth, damping, fmt, ry, w, ru, ru.shape[1], rv, rv.shape[1],
        sy, w, su, su.shape[1], sv, sv.shape[1], None if cod is None else cod.ctypes.data,
        dl, dc, sk)
    if rc != 0:
        raise ValueError("oracle rejected distortion_eq14_coded_format arguments")
    return dl.reshape(nb, 128), dc.reshape(nb, 128), sk


def eq14_term(n, s1s, s2s, s1d, s2d, sse, bitdepth: int) -> int:
    return lib().cdef_ref_eq14_term(n, s1s, s2s, s1d, s2d, sse, bitdepth)


def search_strengths_eq14(rec, src, bitdepth: int, damping: int, lam: int,
                          refine_passes: int = 0):
    dl, dc = distortion_eq14(rec, src, bitdepth, damping)
    out = select_presets_general(dl, dc, 64, None, lam, refine_passes)
    out.update(dist_luma=dl, dist_chroma=dc)
    return out
