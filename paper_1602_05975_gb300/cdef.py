"""Python binding of the cdef_gb300 C ABI (include/cdef_gb300.h).

Argument marshalling only: every step of the CDEF path runs in the CUDA
kernels of libcdef_gb300.so.  PyTorch provides device memory and streams.
There is no CPU fallback: if the library cannot be loaded, every call
raises.

Planes are 2-D CUDA tensors of shape (height, pitch_in_samples) with the
frame's width in the leading columns: torch.uint8 for 8-bit frames,
torch.int16 (holding unsigned values) for 10/12-bit frames.  Use
:func:`alloc_frame` to get correctly pitched planes.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcdef_gb300.so")

CDEF_OK = 0
ERRORS = {-1: "CDEF_ERR_ARG", -2: "CDEF_ERR_SIZE", -3: "CDEF_ERR_BITDEPTH",
          -4: "CDEF_ERR_NOMEM", -5: "CDEF_ERR_CUDA", -6: "CDEF_ERR_TIMEOUT",
          -7: "CDEF_ERR_DEVICE"}
SEC_VALUES = (0, 1, 2, 4)
MAX_BATCH = 48  # frames per cdef_filter_frames / cdef_search_strengths call


class CdefError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{what}: {ERRORS.get(status, status)} ({_strerror(status)})")
        self.status = status


class Plane(C.Structure):
    _fields_ = [("data", C.c_void_p), ("width", C.c_int32), ("height", C.c_int32),
                ("pitch_bytes", C.c_int64)]


class FrameDesc(C.Structure):
    _fields_ = [("y", Plane), ("u", Plane), ("v", Plane), ("bitdepth", C.c_int32)]


class Preset(C.Structure):
    _fields_ = [("pri_y", C.c_uint8), ("sec_y", C.c_uint8), ("pri_uv", C.c_uint8),
                ("sec_uv", C.c_uint8)]


class PresetCoded(C.Structure):
    _fields_ = [("pri_y", C.c_uint8), ("sec_y", C.c_uint8), ("pri_uv", C.c_uint8),
                ("sec_uv", C.c_uint8), ("skip", C.c_uint8), ("reserved", C.c_uint8 * 3)]


class Tuning(C.Structure):
    _fields_ = [("search_groups", C.c_int32), ("search_ctas_per_sm", C.c_int32),
                ("preset_kernel", C.c_int32), ("reserved", C.c_int32)]


_lib = None


def library_path() -> str:
    """The library load() opens: libcdef_gb300.so next to this file, or the
    one the CDEF_GB300_LIBRARY environment variable names (e.g. the
    index-checking build libcdef_gb300_debug.so, made by build(debug=True))."""
    return os.environ.get("CDEF_GB300_LIBRARY") or LIB_PATH


def load():
    """Load the CUDA library (built by build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; build it with "
                           "paper_1602_05975_gb300.build.build()")
    L = C.CDLL(path)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    L.cdef_ctx_create.argtypes = [C.POINTER(vp), C.c_int, C.c_size_t]
    L.cdef_ctx_destroy.argtypes = [vp]
    L.cdef_ctx_status.argtypes = [vp, C.c_int]
    L.cdef_find_dir.argtypes = [vp, C.POINTER(Plane), i32, vp, vp, vp]
    L.cdef_filter_frame.argtypes = [vp, C.POINTER(FrameDesc), vp, vp, vp,
                                    C.POINTER(FrameDesc), vp]
    L.cdef_filter_frame_coded.argtypes = [vp, C.POINTER(FrameDesc), vp, vp,
                                          C.POINTER(FrameDesc), vp]
    L.cdef_filter_frames.argtypes = [vp, i32, C.POINTER(FrameDesc), C.POINTER(vp),
                                     C.POINTER(FrameDesc), vp]
    L.cdef_search_strengths.argtypes = [vp, i32, C.POINTER(FrameDesc), C.POINTER(FrameDesc),
                                        C.POINTER(i32), C.POINTER(i64), vp, vp,
                                        C.POINTER(Preset), C.POINTER(i32), vp,
                                        C.POINTER(i64), vp]
    L.cdef_ctx_set_tuning.argtypes = [vp, C.POINTER(Tuning)]
    L.cdef_ctx_set_overlap.argtypes = [vp, C.c_int]
    L.cdef_ctx_set_search_refine.argtypes = [vp, C.c_int]
    L.cdef_ctx_set_search_metric.argtypes = [vp, C.c_int]
    L.cdef_ctx_get_tuning.argtypes = [vp, C.POINTER(Tuning)]
    L.cdef_ctx_set_stage_timing.argtypes = [vp, C.c_int]
    L.cdef_ctx_set_search_subset.argtypes = [vp, C.c_uint64, C.c_uint64]
    L.cdef_ctx_status_async.argtypes = [vp, vp, vp]
    L.cdef_ctx_get_stage_times.argtypes = [vp, C.POINTER(C.c_float), C.POINTER(C.c_float)]
    L.cdef_search_strengths_coded.argtypes = [
        vp, i32, C.POINTER(FrameDesc), C.POINTER(FrameDesc), C.POINTER(vp), C.POINTER(i32),
        C.POINTER(i64), vp, vp, C.POINTER(PresetCoded), C.POINTER(i32), vp, C.POINTER(i64), vp]
    L.cdef_debug_set_waits.argtypes = [i64, i32]
    L.cdef_debug_checks.argtypes = [vp, C.POINTER(i64), i32]
    L.cdef_probe_int_mix.argtypes = [vp, i32, i32, C.POINTER(C.c_double), vp]
    L.cdef_search_tables.argtypes = [vp, i32, C.POINTER(FrameDesc), C.POINTER(FrameDesc),
                                     C.POINTER(vp), C.POINTER(i32), C.POINTER(i32),
                                     C.POINTER(i32), vp, vp, vp, vp]
    L.cdef_preset_totals.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp]
    L.cdef_preset_argmin.argtypes = [vp, i32, vp, C.c_uint64, C.c_uint64, i32, vp, vp]
    L.cdef_preset_assign.argtypes = [vp, i32, i32, vp, vp, vp, C.POINTER(i32), i32, vp, vp, vp,
                                     vp]
    L.cdef_strerror.argtypes = [C.c_int]
    L.cdef_strerror.restype = C.c_char_p
    L.cdef_version.restype = C.c_char_p
    for name in ("cdef_ctx_create", "cdef_ctx_destroy", "cdef_ctx_status", "cdef_find_dir",
                 "cdef_filter_frame", "cdef_filter_frame_coded", "cdef_filter_frames",
                 "cdef_search_strengths",
                 "cdef_ctx_set_tuning", "cdef_ctx_get_tuning", "cdef_ctx_set_overlap",
                 "cdef_ctx_set_search_refine", "cdef_search_strengths_coded",
                 "cdef_ctx_set_search_metric", "cdef_ctx_set_stage_timing",
                 "cdef_ctx_get_stage_times", "cdef_ctx_set_search_subset",
                 "cdef_ctx_status_async", "cdef_debug_set_waits", "cdef_debug_checks",
                 "cdef_probe_int_mix",
                 "cdef_search_tables",
                 "cdef_preset_totals", "cdef_preset_argmin", "cdef_preset_assign"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _strerror(status):
    try:
        return load().cdef_strerror(status).decode()
    except Exception:  # noqa: BLE001 - only used inside an error message
        return "?"


def _check(rc, what):
    if rc != CDEF_OK:
        raise CdefError(rc, what)


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


# --------------------------------------------------------------- planes
def sample_dtype(bitdepth: int):
    return torch.uint8 if bitdepth == 8 else torch.int16


def pitch_samples(width: int, bitdepth: int) -> int:
    """Row pitch (in samples) rounded up to a multiple of 16 bytes."""
    b = 1 if bitdepth == 8 else 2
    return ((width * b + 15) // 16 * 16) // b


def chroma_size(width: int, height: int, chroma: int = 420):
    """Chroma plane size for format 420, 422 or 444."""
    return {420: (width // 2, height // 2), 422: (width // 2, height),
            444: (width, height)}[chroma]


@dataclass
class Frame:
    """A frame in device memory: y, u, v are pitched 2-D tensors; `chroma`
    is the format (420, 422 or 444)."""
    y: torch.Tensor
    u: torch.Tensor
    v: torch.Tensor
    width: int
    height: int
    bitdepth: int
    chroma: int = 420

    def planes(self):
        return (self.y, self.u, self.v)

    def desc(self) -> FrameDesc:
        """The C descriptor of the frame, kept on the frame while the planes'
        pointers, pitches and element sizes and the frame's fields stay."""
        y, u, v = self.y, self.u, self.v
        key = (y.data_ptr(), u.data_ptr(), v.data_ptr(), y.stride(0), u.stride(0), v.stride(0),
               y.element_size(), u.element_size(), v.element_size(), self.width, self.height,
               self.bitdepth, self.chroma)
        cached = self.__dict__.get("_desc")
        if cached is not None and cached[0] == key:
            return cached[1]
        d = FrameDesc()
        cw, ch = chroma_size(self.width, self.height, self.chroma)
        for name, t, w, h in (("y", self.y, self.width, self.height),
                              ("u", self.u, cw, ch), ("v", self.v, cw, ch)):
            p = getattr(d, name)
            p.data = t.data_ptr()
            p.width = w
            p.height = h
            p.pitch_bytes = t.stride(0) * t.element_size()
        d.bitdepth = self.bitdepth
        self.__dict__["_desc"] = (key, d)
        return d

    def to_numpy(self):
        """Host copies of the visible planes as uint16 arrays."""
        out = []
        cw = chroma_size(self.width, self.height, self.chroma)[0]
        for t, w in ((self.y, self.width), (self.u, cw), (self.v, cw)):
            a = t[:, :w].cpu().numpy()
            out.append(a.view(np.uint16) if a.dtype == np.int16 else a.astype(np.uint16))
        return tuple(out)


def alloc_frame(width: int, height: int, bitdepth: int, device="cuda", fill=None,
                chroma: int = 420) -> Frame:
    dt = sample_dtype(bitdepth)
    cw, ch = chroma_size(width, height, chroma)
    planes = []
    for w, h in ((width, height), (cw, ch), (cw, ch)):
        t = torch.empty((h, pitch_samples(w, bitdepth)), dtype=dt, device=device)
        if fill is not None:
            t.fill_(fill)
        planes.append(t)
    return Frame(*planes, width, height, bitdepth, chroma)


def packed_layout(width: int, height: int, bitdepth: int, extra_bytes: int = 0):
    """Byte offsets of the y, u, v planes (and of `extra_bytes` after them)
    in one flat buffer, each 256-byte aligned, and the buffer's size."""
    b = 1 if bitdepth == 8 else 2
    offs, o = [], 0
    for w, h in ((width, height), (width // 2, height // 2), (width // 2, height // 2)):
        offs.append(o)
        o += -(-h * pitch_samples(w, bitdepth) * b // 256) * 256
    offs.append(o)
    return offs, o + -(-extra_bytes // 256) * 256


def alloc_packed(width: int, height: int, bitdepth: int, device="cuda", pin=False,
                 extra_bytes: int = 0):
    """A frame whose three planes are views into one flat uint8 buffer (one
    copy moves the whole frame).  Returns (flat, frame, extra) where `extra`
    is a uint8 view of `extra_bytes` after the planes (e.g. parameters)."""
    offs, size = packed_layout(width, height, bitdepth, extra_bytes)
    flat = torch.empty(size, dtype=torch.uint8, device=device)
    if pin:
        flat = flat.pin_memory()
    dt, b = sample_dtype(bitdepth), (1 if bitdepth == 8 else 2)
    planes = []
    for k, (w, h) in enumerate(((width, height), (width // 2, height // 2),
                                (width // 2, height // 2))):
        p = pitch_samples(w, bitdepth)
        planes.append(flat[offs[k]:offs[k] + h * p * b].view(dt).view(h, p))
    return flat, Frame(*planes, width, height, bitdepth), flat[offs[3]:offs[3] + extra_bytes]


def frame_from_numpy(planes, bitdepth: int, device="cuda", pin=False) -> Frame:
    """Copy host uint16 planes (y, u, v) into a pitched frame (or, with
    device='cpu' and pin=True, a pinned host frame)."""
    y = planes[0]
    h, w = y.shape
    ch, cw = np.asarray(planes[1]).shape
    chroma = {(w // 2, h // 2): 420, (w // 2, h): 422, (w, h): 444}[(cw, ch)]
    f = alloc_frame(w, h, bitdepth, device="cpu", chroma=chroma)
    for t, a in zip(f.planes(), planes):
        a = np.asarray(a)
        if bitdepth == 8:
            t[:, :a.shape[1]] = torch.from_numpy(a.astype(np.uint8))
        else:
            t[:, :a.shape[1]] = torch.from_numpy(a.astype(np.uint16).view(np.int16))
    if device == "cpu":
        if pin:
            f = Frame(*(t.pin_memory() for t in f.planes()), w, h, bitdepth, chroma)
        return f
    return Frame(*(t.to(device) for t in f.planes()), w, h, bitdepth, chroma)


def params_tensor(params: np.ndarray, device="cuda") -> torch.Tensor:
    """(fb_rows, fb_cols, 8) uint8 parameters as a flat device tensor."""
    p = np.ascontiguousarray(params, dtype=np.uint8)
    assert p.shape[-1] == 8
    return torch.from_numpy(p.reshape(-1)).to(device)


# --------------------------------------------------------------- context
class Context:
    """Owns a cdef_ctx (device scratch, pinned staging) on one GPU."""

    def __init__(self, device: int = 0, budget_bytes: int = 0):
        self._lib = load()
        h = C.c_void_p()
        _check(self._lib.cdef_ctx_create(C.byref(h), device, budget_bytes), "cdef_ctx_create")
        self.handle = h
        self.device = device
        self.pairs = ((1 << 64) - 1, (1 << 64) - 1)   # the search subset (luma, chroma)

    def close(self):
        if self.handle:
            self._lib.cdef_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def status(self, clear=True):
        return self._lib.cdef_ctx_status(self.handle, int(clear))

    def status_async(self, host_status: torch.Tensor, stream=None):
        """Enqueue a copy of the status word into host_status[0] (a pinned
        int32 CPU tensor) on `stream`; read it once the stream is past it."""
        _check(self._lib.cdef_ctx_status_async(self.handle, host_status.data_ptr(),
                                               _stream_ptr(stream)), "cdef_ctx_status_async")

    def set_search_refine(self, max_passes: int):
        """Re-optimise the searched presets one at a time for at most
        `max_passes` passes (0 = greedy only)."""
        _check(self._lib.cdef_ctx_set_search_refine(self.handle, int(max_passes)),
               "cdef_ctx_set_search_refine")

    def set_search_metric(self, metric: str):
        """'sse' (default) or 'eq14' (section 5's SSIM-weighted distortion)."""
        m = {"sse": 0, "eq14": 1}[metric]
        _check(self._lib.cdef_ctx_set_search_metric(self.handle, m), "cdef_ctx_set_search_metric")

    def set_search_subset(self, luma_pairs: int = (1 << 64) - 1, chroma_pairs: int = (1 << 64) - 1):
        """Allowed (S_p, S_s) pairs of later searches, bit p * 4 + s per plane
        group (default: all)."""
        _check(self._lib.cdef_ctx_set_search_subset(self.handle, luma_pairs, chroma_pairs),
               "cdef_ctx_set_search_subset")
        self.pairs = (luma_pairs, chroma_pairs)

    def set_stage_timing(self, enable: bool):
        """Record per-stage device times of later strength searches."""
        _check(self._lib.cdef_ctx_set_stage_timing(self.handle, int(bool(enable))),
               "cdef_ctx_set_stage_timing")

    def stage_times(self):
        """(distortion-table ms, preset-selection ms) of the last search."""
        a, b = C.c_float(), C.c_float()
        _check(self._lib.cdef_ctx_get_stage_times(self.handle, C.byref(a), C.byref(b)),
               "cdef_ctx_get_stage_times")
        return a.value, b.value

    def set_overlap(self, enable: bool):
        """Declare consecutive filter calls on a stream independent (see
        cdef_ctx_set_overlap): they may then run concurrently."""
        _check(self._lib.cdef_ctx_set_overlap(self.handle, int(bool(enable))),
               "cdef_ctx_set_overlap")

    def set_tuning(self, search_groups: int = 0, search_ctas_per_sm: int = 0,
                   preset_kernel: int = 0):
        """Fix the strength search's launch configuration (0 = autotune);
        preset_kernel 1: the preset selection always in the grid-wide
        kernel (0: one thread-block cluster per frame where frames fit)."""
        t = Tuning(search_groups, search_ctas_per_sm, preset_kernel)
        _check(self._lib.cdef_ctx_set_tuning(self.handle, C.byref(t)), "cdef_ctx_set_tuning")

    def tuning(self):
        """(search_groups, search_ctas_per_sm) of the last search."""
        t = Tuning()
        _check(self._lib.cdef_ctx_get_tuning(self.handle, C.byref(t)), "cdef_ctx_get_tuning")
        return t.search_groups, t.search_ctas_per_sm


def cdef_find_dir(ctx: Context, luma: torch.Tensor, width: int, height: int, bitdepth: int,
                  dirs: torch.Tensor, var: torch.Tensor, stream=None):
    p = Plane(luma.data_ptr(), width, height, luma.stride(0) * luma.element_size())
    assert dirs.dtype == torch.uint8 and var.dtype == torch.int32
    assert dirs.numel() >= (height // 8) * (width // 8) and var.numel() >= dirs.numel()
    _check(ctx._lib.cdef_find_dir(ctx.handle, C.byref(p), bitdepth, dirs.data_ptr(),
                                  var.data_ptr(), _stream_ptr(stream)), "cdef_find_dir")


def cdef_filter_frame(ctx: Context, src: Frame, params: torch.Tensor, out: Frame,
                      dirs: torch.Tensor | None = None, var: torch.Tensor | None = None,
                      stream=None):
    di, do = src.desc(), out.desc()
    _check(ctx._lib.cdef_filter_frame(
        ctx.handle, C.byref(di), params.data_ptr(),
        None if dirs is None else dirs.data_ptr(), None if var is None else var.data_ptr(),
        C.byref(do), _stream_ptr(stream)), "cdef_filter_frame")


def cdef_filter_frame_coded(ctx: Context, src: Frame, params: torch.Tensor, coded: torch.Tensor,
                            out: Frame, stream=None):
    """The filter with section 4's skip semantics; `coded` is a uint8 CUDA
    tensor of (H/8) x (W/8) coded-residual flags."""
    di, do = src.desc(), out.desc()
    _check(ctx._lib.cdef_filter_frame_coded(ctx.handle, C.byref(di), params.data_ptr(),
                                            coded.data_ptr(), C.byref(do), _stream_ptr(stream)),
           "cdef_filter_frame_coded")


def cdef_filter_frames(ctx: Context, srcs, params, outs, stream=None):
    n = len(srcs)
    ins = (FrameDesc * n)(*[f.desc() for f in srcs])
    os_ = (FrameDesc * n)(*[f.desc() for f in outs])
    prm = (C.c_void_p * n)(*[p.data_ptr() for p in params])
    _check(ctx._lib.cdef_filter_frames(ctx.handle, n, ins, prm, os_, _stream_ptr(stream)),
           "cdef_filter_frames")


def _search_results(presets, fields: int, n: int, npre, cost):
    """Per frame: its eight presets as tuples of their first `fields` bytes,
    N and J."""
    per = C.sizeof(presets) // (8 * n) if n else 0
    a = np.frombuffer(presets, dtype=np.uint8).reshape(n, 8, per)[:, :, :fields].tolist()
    return [dict(presets=[tuple(p) for p in a[i]], npresets=npre[i], cost=cost[i])
            for i in range(n)]


def cdef_search_strengths(ctx: Context, recs, srcs, damping, lambdas, block_ids: torch.Tensor,
                          dist_luma: torch.Tensor | None = None,
                          dist_chroma: torch.Tensor | None = None, stream=None):
    """Returns per frame: presets [(pri_y, sec_y, pri_uv, sec_uv)]*N, N, J."""
    n = len(recs)
    ri = (FrameDesc * n)(*[f.desc() for f in recs])
    si = (FrameDesc * n)(*[f.desc() for f in srcs])
    damp = (C.c_int32 * n)(*damping)
    lam = (C.c_int64 * n)(*lambdas)
    presets = (Preset * (8 * n))()
    npre = (C.c_int32 * n)()
    cost = (C.c_int64 * n)()
    _check(ctx._lib.cdef_search_strengths(
        ctx.handle, n, ri, si, damp, lam,
        None if dist_luma is None else dist_luma.data_ptr(),
        None if dist_chroma is None else dist_chroma.data_ptr(),
        presets, npre, block_ids.data_ptr(), cost, _stream_ptr(stream)),
        "cdef_search_strengths")
    return _search_results(presets, 4, n, npre, cost)


def cdef_search_strengths_noalloc(recs, srcs, damping, lambdas, block_ids: torch.Tensor,
                                  dist_luma: torch.Tensor, dist_chroma: torch.Tensor,
                                  stream=None):
    """The strength search through the entry point that allocates nothing
    (no context; the caller provides the distortion tables).  Runs on the
    current CUDA device.  Same result format as cdef_search_strengths."""
    L = load()
    fn = L.cdef_search_strengths_noalloc
    i32, i64, vp = C.c_int32, C.c_int64, C.c_void_p
    fn.argtypes = [i32, C.POINTER(FrameDesc), C.POINTER(FrameDesc), C.POINTER(i32),
                   C.POINTER(i64), vp, vp, C.POINTER(Preset), C.POINTER(i32), vp,
                   C.POINTER(i64), vp]
    fn.restype = C.c_int
    n = len(recs)
    ri = (FrameDesc * n)(*[f.desc() for f in recs])
    si = (FrameDesc * n)(*[f.desc() for f in srcs])
    presets = (Preset * (8 * n))()
    npre = (C.c_int32 * n)()
    cost = (C.c_int64 * n)()
    _check(fn(n, ri, si, (C.c_int32 * n)(*damping), (C.c_int64 * n)(*lambdas),
              dist_luma.data_ptr(), dist_chroma.data_ptr(), presets, npre,
              block_ids.data_ptr(), cost, _stream_ptr(stream)),
           "cdef_search_strengths_noalloc")
    return _search_results(presets, 4, n, npre, cost)


def cdef_search_strengths_coded(ctx: Context, recs, srcs, coded, damping, lambdas,
                                block_ids: torch.Tensor, dist_luma: torch.Tensor | None = None,
                                dist_chroma: torch.Tensor | None = None, stream=None):
    """The 128-combination search with section 4's skip semantics; `coded`
    is a list of uint8 CUDA tensors ((H/8) x (W/8) coded-residual flags).
    Returns per frame: presets [(pri_y, sec_y, pri_uv, sec_uv, skip)]*8, N, J."""
    n = len(recs)
    ri = (FrameDesc * n)(*[f.desc() for f in recs])
    si = (FrameDesc * n)(*[f.desc() for f in srcs])
    cm = (C.c_void_p * n)(*[c.data_ptr() for c in coded])
    damp = (C.c_int32 * n)(*damping)
    lam = (C.c_int64 * n)(*lambdas)
    presets = (PresetCoded * (8 * n))()
    npre = (C.c_int32 * n)()
    cost = (C.c_int64 * n)()
    _check(ctx._lib.cdef_search_strengths_coded(
        ctx.handle, n, ri, si, cm, damp, lam,
        None if dist_luma is None else dist_luma.data_ptr(),
        None if dist_chroma is None else dist_chroma.data_ptr(),
        presets, npre, block_ids.data_ptr(), cost, _stream_ptr(stream)),
        "cdef_search_strengths_coded")
    return _search_results(presets, 5, n, npre, cost)


def _ptr(t):
    return None if t is None else t.data_ptr()


def cdef_search_tables(ctx: Context, recs, srcs, damping, row_begin, row_count,
                       dist_luma: torch.Tensor, dist_chroma: torch.Tensor, coded=None,
                       skipped: torch.Tensor | None = None, stream=None):
    """Section 5's tables of a band of filter-block rows per frame (rows
    row_begin[i] .. row_begin[i] + row_count[i] - 1 of frame i); `coded`
    (list of device maps) with `skipped` (device flags) selects the 128
    combinations."""
    n = len(recs)
    ri = (FrameDesc * n)(*[f.desc() for f in recs])
    si = (FrameDesc * n)(*[f.desc() for f in srcs])
    cm = None if coded is None else (C.c_void_p * n)(*[c.data_ptr() for c in coded])
    _check(ctx._lib.cdef_search_tables(
        ctx.handle, n, ri, si, cm, (C.c_int32 * n)(*damping), (C.c_int32 * n)(*row_begin),
        (C.c_int32 * n)(*row_count), dist_luma.data_ptr(), dist_chroma.data_ptr(), _ptr(skipped),
        _stream_ptr(stream)), "cdef_search_tables")


def cdef_preset_totals(ctx: Context, nblocks: int, width: int, dist_luma, dist_chroma, skipped,
                       best, totals: torch.Tensor, stream=None):
    """totals[t] = sum over the blocks not skipped of min(best[b], D_b(t))."""
    _check(ctx._lib.cdef_preset_totals(ctx.handle, nblocks, width, _ptr(dist_luma),
                                       _ptr(dist_chroma), _ptr(skipped), _ptr(best),
                                       totals.data_ptr(), _stream_ptr(stream)),
           "cdef_preset_totals")


def cdef_preset_argmin(ctx: Context, width: int, totals: torch.Tensor, luma_pairs: int,
                       chroma_pairs: int, keep: int, result: torch.Tensor, stream=None):
    """result[0] = the least allowed preset (keep kept on ties with it),
    result[1] = its total (device int64[2])."""
    _check(ctx._lib.cdef_preset_argmin(ctx.handle, width, totals.data_ptr(), luma_pairs,
                                       chroma_pairs, keep, result.data_ptr(), _stream_ptr(stream)),
           "cdef_preset_argmin")


def cdef_preset_assign(ctx: Context, nblocks: int, width: int, dist_luma, dist_chroma, skipped,
                       presets, best=None, block_ids=None, sums=None, stream=None):
    """Per block: least distortion over `presets` (best), the first preset
    attaining it (block_ids); sums = (total of best, blocks not skipped)."""
    n = len(presets)
    arr = (C.c_int32 * max(n, 1))(*presets)
    _check(ctx._lib.cdef_preset_assign(ctx.handle, nblocks, width, _ptr(dist_luma),
                                       _ptr(dist_chroma), _ptr(skipped), arr, n, _ptr(best),
                                       _ptr(block_ids), _ptr(sums), _stream_ptr(stream)),
           "cdef_preset_assign")


def preset_index_coded(p) -> int:
    """(pri_y, sec_y, pri_uv, sec_uv, skip) -> luma_q * 128 + chroma_q with
    q = skip_bit * 64 + pri * 4 + secondary index."""
    ql = (p[4] & 1) * 64 + p[0] * 4 + SEC_VALUES.index(p[1])
    qc = ((p[4] >> 1) & 1) * 64 + p[2] * 4 + SEC_VALUES.index(p[3])
    return ql * 128 + qc


def preset_index(p) -> int:
    """(pri_y, sec_y, pri_uv, sec_uv) -> luma_pair * 64 + chroma_pair."""
    return (p[0] * 4 + SEC_VALUES.index(p[1])) * 64 + p[2] * 4 + SEC_VALUES.index(p[3])


def debug_set_waits(wait_cycles: int = 0, extra_tx_bytes: int = 0):
    """Test aid: the kernels' tile-load wait limit (SM cycles, 0 = default)
    and bytes added to every load's expected count that no load delivers
    (so that waits run out); process-wide, for later launches."""
    _check(load().cdef_debug_set_waits(int(wait_cycles), int(extra_tx_bytes)),
           "cdef_debug_set_waits")


def debug_checks(ctx, clear: bool = True):
    """Test aid: (whether the loaded library checks its kernels' indexes,
    accesses out of range that its kernels skipped on ctx's device since the
    last clear).  Waits for the device."""
    n = C.c_int64(0)
    r = load().cdef_debug_checks(ctx.handle, C.byref(n), 1 if clear else 0)
    if r < 0:
        _check(r, "cdef_debug_checks")
    return bool(r), int(n.value)


def probe_int_mix(ctx, mix: int = 0, iters: int = 4096, stream=None) -> float:
    """Measurement aid: lane instructions per second of the filter's tap
    mix (mix 0), of its integer-ALU operations alone (mix 1), or of the
    single-pipe mixes 2-6 (integer multiply-adds, multiplies-high, packed
    maxima with multiply-adds, logic operations with multiply-adds, fp32
    FMAs) on ctx's device."""
    r = C.c_double(0.0)
    _check(load().cdef_probe_int_mix(ctx.handle, int(mix), int(iters), C.byref(r),
                                     _stream_ptr(stream)), "cdef_probe_int_mix")
    return float(r.value)


def version() -> str:
    return load().cdef_version().decode()
