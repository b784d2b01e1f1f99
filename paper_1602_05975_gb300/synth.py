"""Seeded synthetic frames shaped like the paper's test material.

This module holds input generation only: no step of the CDEF method (no
direction search, constraint, filtering or distortion) lives here.  Both the
CUDA path's tests/benchmark and the oracle consume what it produces.

The paper evaluates on the AWCY objective-1-fast video set (section 6),
which is not available here; these frames stand in for it:

* source: 128 + three random oriented sinusoids (amplitude U[10,40],
  frequency U[1/64, 1/4] cycles/pixel, angle U[0, pi), phase U[0, 2 pi))
  plus 2-6 random step edges of height +-U[10,60], clipped to [16, 235];
  chroma planes use the same recipe at their own resolution (half in both
  directions for 4:2:0, the default) with halved amplitudes;
* decoded ("reconstructed") frame: each plane is coded by an orthonormal 8x8
  DCT-II in float64, coefficients quantised as rint(c/Q)*Q, inverse DCT,
  rint, clip to the sample range -- quantisation ringing of the kind CDEF is
  designed to remove;
* 10-bit: the 8-bit source is mapped into [64, 940] (x4 around 16) and the
  quantiser step is multiplied by 4;
* per 64x64 filter block: luma/chroma primary strength U{0..15}, secondary
  U{0,1,2,4}, damping U{3..6}.

Everything is drawn from numpy's PCG64 seeded by the caller.
"""
from __future__ import annotations

import hashlib
from dataclasses import dataclass

import numpy as np

SEC_VALUES = (0, 1, 2, 4)
PARAM_BYTES = 8  # pri_y, sec_y, pri_uv, sec_uv, damping, 3 unused


@dataclass
class Frame:
    """One synthetic frame: planes are uint16 numpy arrays (any bit depth)."""
    width: int
    height: int
    bitdepth: int
    q: int
    src: tuple  # (y, u, v)
    rec: tuple  # (y, u, v) decoded, before CDEF
    params: np.ndarray  # uint8 (fb_rows, fb_cols, 8)


def _dct_matrix(n: int = 8) -> np.ndarray:
    k = np.arange(n)[:, None]
    i = np.arange(n)[None, :]
    m = np.cos(np.pi * (2 * i + 1) * k / (2 * n)) * np.sqrt(2.0 / n)
    m[0, :] = np.sqrt(1.0 / n)
    return m


_DCT = _dct_matrix()


def _source_plane(rng, w, h, amp_scale):
    yy = np.arange(h, dtype=np.float64)[:, None]
    xx = np.arange(w, dtype=np.float64)[None, :]
    img = np.full((h, w), 128.0)
    for _ in range(3):
        a = rng.uniform(10, 40) * amp_scale
        f = rng.uniform(1 / 64, 1 / 4)
        th = rng.uniform(0, np.pi)
        ph = rng.uniform(0, 2 * np.pi)
        img += a * np.sin(2 * np.pi * f * (xx * np.cos(th) + yy * np.sin(th)) + ph)
    for _ in range(int(rng.integers(2, 7))):
        # a random line through the frame; one side is stepped
        px, py = rng.uniform(0, w), rng.uniform(0, h)
        th = rng.uniform(0, np.pi)
        step = rng.uniform(10, 60) * amp_scale * (1 if rng.random() < 0.5 else -1)
        side = (xx - px) * np.sin(th) - (yy - py) * np.cos(th) > 0
        img += step * side
    return np.clip(img, 16, 235)


def _code_plane(plane, q, maxval):
    """8x8 DCT quantisation round trip of a float plane (padded to 8)."""
    h, w = plane.shape
    ph, pw = -(-h // 8) * 8, -(-w // 8) * 8
    p = np.pad(plane, ((0, ph - h), (0, pw - w)), mode="edge")
    blocks = p.reshape(ph // 8, 8, pw // 8, 8).transpose(0, 2, 1, 3)
    c = _DCT @ blocks @ _DCT.T
    c = np.rint(c / q) * q
    r = _DCT.T @ c @ _DCT
    r = r.transpose(0, 2, 1, 3).reshape(ph, pw)[:h, :w]
    return np.clip(np.rint(r), 0, maxval)


def random_params(rng, width, height, damping=None):
    fbr, fbc = -(-height // 64), -(-width // 64)
    prm = np.zeros((fbr, fbc, PARAM_BYTES), np.uint8)
    prm[..., 0] = rng.integers(0, 16, (fbr, fbc))
    prm[..., 1] = np.asarray(SEC_VALUES)[rng.integers(0, 4, (fbr, fbc))]
    prm[..., 2] = rng.integers(0, 16, (fbr, fbc))
    prm[..., 3] = np.asarray(SEC_VALUES)[rng.integers(0, 4, (fbr, fbc))]
    prm[..., 4] = rng.integers(3, 7, (fbr, fbc)) if damping is None else damping
    return prm


def chroma_dims(width: int, height: int, chroma: int = 420):
    """(width, height) of a chroma plane: 4:2:0 halves both, 4:2:2 the
    width, 4:4:4 neither."""
    if chroma == 420:
        return width // 2, height // 2
    if chroma == 422:
        return width // 2, height
    if chroma == 444:
        return width, height
    raise ValueError("chroma format must be 420, 422 or 444")


def make_frame(width: int, height: int, bitdepth: int = 8, q=32,
               seed: int = 0, chroma: int = 420) -> Frame:
    """A source/decoded frame pair plus random per-64x64 CDEF parameters.
    q=None draws the quantiser step from {16, 32, 64}; `chroma` is the
    chroma format (the chroma recipe at the plane's own resolution)."""
    if width % 8 or height % 8:
        raise ValueError("width and height must be multiples of 8")
    cw, ch = chroma_dims(width, height, chroma)
    rng = np.random.Generator(np.random.PCG64(seed))
    maxval = (1 << bitdepth) - 1
    src = [_source_plane(rng, width, height, 1.0),
           _source_plane(rng, cw, ch, 0.5),
           _source_plane(rng, cw, ch, 0.5)]
    if q is None:
        q = (16, 32, 64)[int(rng.integers(0, 3))]
    qq = q
    if bitdepth > 8:
        # [16, 235] -> [16, 235] * 2^(bd-8); 10-bit gives [64, 940]
        scale = 1 << (bitdepth - 8)
        src = [s * scale for s in src]
        qq = q * scale
    src_i = tuple(np.rint(s).astype(np.uint16) for s in src)
    rec = tuple(_code_plane(s.astype(np.float64), qq, maxval).astype(np.uint16)
                for s in src_i)
    params = random_params(rng, width, height)
    return Frame(width, height, bitdepth, q, src_i, rec, params)


def random_frame_planes(rng, width, height, bitdepth):
    """Uniformly random planes (stress input for parity tests)."""
    maxval = (1 << bitdepth) - 1
    return tuple(rng.integers(0, maxval + 1, (h, w)).astype(np.uint16)
                 for (w, h) in ((width, height), (width // 2, height // 2),
                                (width // 2, height // 2)))


# The workloads the benchmark and the tests are built around (section 6 of
# the paper used CIF-to-1080p sequences; 4K 10-bit is the large case).
WORKLOADS = {
    "cif_8bit": dict(width=352, height=288, bitdepth=8, frames=1),
    "1080p_8bit_x30": dict(width=1920, height=1080, bitdepth=8, frames=30),
    "4k_10bit_x8": dict(width=3840, height=2160, bitdepth=10, frames=8),
}


def workload_frames(name: str, base_seed: int, nframes=None):
    """Frames of a named workload; frame f uses seed base_seed + f; the
    multi-frame workloads draw Q from {16, 32, 64} per frame."""
    cfg = WORKLOADS[name]
    n = cfg["frames"] if nframes is None else nframes
    out = []
    for f in range(n):
        q = 32 if cfg["frames"] == 1 else None
        out.append(make_frame(cfg["width"], cfg["height"], cfg["bitdepth"], q,
                              base_seed + f))
    return out


def frame_digest(f: Frame) -> str:
    """SHA-256 of a synthetic frame: its geometry, bit depth and quantiser,
    the source and decoded planes (as little-endian uint16) and the
    parameters.  Recorded per workload (tests/golden/synth_manifest.json) so
    that a change of the input recipe does not go unnoticed, and printed by
    the benchmark so that two runs can be seen to use the same inputs."""
    h = hashlib.sha256()
    h.update(np.array([f.width, f.height, f.bitdepth, f.q], dtype="<i8").tobytes())
    for p in tuple(f.src) + tuple(f.rec):
        a = np.ascontiguousarray(p, dtype="<u2")
        h.update(np.array(a.shape, dtype="<i8").tobytes())
        h.update(a.tobytes())
    h.update(np.ascontiguousarray(f.params, dtype=np.uint8).tobytes())
    return h.hexdigest()


def digest_of(frames) -> str:
    """One SHA-256 over the digests of a list of frames."""
    return hashlib.sha256("".join(frame_digest(f) for f in frames).encode()).hexdigest()
