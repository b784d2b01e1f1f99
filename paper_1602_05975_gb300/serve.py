"""Decode-side CDEF serving loop with continuous batching.

Requests are single 4:2:0 frames of any supported size and bit depth, each
with its own per-64x64 parameters (section 4: one primary/secondary strength
pair per plane group and a damping value per filter block).  The server

* admits queued requests in arrival order while their device buffers fit an
  HBM budget (input frame + parameters + output frame per request) and the
  next batch has room (requests are not given buffers earlier than the
  batch that will carry them needs them);
* launches every admitted request that is not yet on the device as one
  batch through the batched filter entry point (``cdef_filter_frames``: one
  launch for frames of mixed sizes and bit depths), as soon as fewer than
  ``max_inflight`` batches are on the device -- requests that arrive while a
  batch runs join the next one;
* overlaps the host-to-device copies of the next batch, the filter launch of
  the current one and the device-to-host copies of the previous one on three
  CUDA streams;
* frees a request's buffers when its output has reached the host.

The scheduling is host logic over a small backend interface, so that it can
be driven by a fake backend in tests (no GPU) and by :class:`CudaBackend`
on the GPU.  ``max_batch=1, max_inflight=1`` turns the same loop into the
one-frame-at-a-time server used as the comparison point.
"""
from __future__ import annotations

import collections
import dataclasses
import gc
import math
import time
from typing import Callable, Optional

import numpy as np

# Signalled ranges of section 4: primary 0..15 (19 for the skip mapping),
# secondary {0, 1, 2, 4} (7 for the skip mapping), damping 3..6; as a table
# of valid byte values per parameter field (pri_y, sec_y, pri_uv, sec_uv,
# damping), so that a request is checked with one lookup.
_PRI_OK = set(range(16)) | {19}
_SEC_OK = {0, 1, 2, 4, 7}
# _BITS[v]: bit k set where byte value v is valid for field k; a block's 8
# bytes mapped through it and read as one little-endian uint64 must have
# bit k of byte k set for k < 5 (bytes 5..7 are not checked here)
_BITS = np.zeros(256, dtype=np.uint8)
for _k, _ok in enumerate((_PRI_OK, _SEC_OK, _PRI_OK, _SEC_OK, range(3, 7))):
    _BITS[list(_ok)] |= np.uint8(1 << _k)
_WANT = np.uint64(sum((1 << k) << (8 * k) for k in range(5)))
_DAMP = np.uint64((1 << 4) << 32)


def validate_params(params: np.ndarray, width: int, height: int) -> Optional[str]:
    """Host-side check of a request's parameter array; None if valid."""
    rows, cols = -(-height // 64), -(-width // 64)
    if params.shape != (rows, cols, 8) or params.dtype != np.uint8:
        return f"params shape {params.shape} ({params.dtype}), expected {(rows, cols, 8)} uint8"
    m = np.take(_BITS, np.ascontiguousarray(params).reshape(-1)).view("<u8") & _WANT
    if (m == _WANT).all():
        return None
    return "damping out of range" if ((m & _DAMP) != _DAMP).any() else "strength out of range"


@dataclasses.dataclass(eq=False)
class Request:
    """One frame to filter.  `frame` is the backend's input (for
    :class:`CudaBackend`: a pinned host buffer in the packed frame layout of
    ``cdef.packed_layout``), `params` the (rows, cols, 8) uint8 parameters
    (`params_host`: optionally the same bytes in pinned host memory), and
    `arrival` seconds from the start of the run."""
    rid: int
    width: int
    height: int
    bitdepth: int
    frame: object
    params: np.ndarray
    arrival: float = 0.0
    # filled in by the server
    status: str = "new"            # queued, admitted, launched, ok, rejected, failed, cancelled
    error: str = ""
    t_submit: float = math.nan
    t_admit: float = math.nan
    t_launch: float = math.nan
    t_done: float = math.nan
    need: int = 0                  # device bytes held while admitted
    slot: object = None            # backend buffers
    out: object = None             # backend output (CudaBackend: (flat, Frame, _) in pinned
                                   # host memory, valid while on_done runs)
    params_host: object = None

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


class Backend:
    """What the server needs from a device."""

    def need_bytes(self, req: Request) -> int:
        raise NotImplementedError

    def reserve(self, req: Request) -> None:
        """Give `req` device buffers (called at admission)."""
        raise NotImplementedError

    def release(self, req: Request) -> None:
        raise NotImplementedError

    def launch(self, reqs: list) -> object:
        """Enqueue upload, filter and download of `reqs`; returns a handle.
        Raises on a launch error."""
        raise NotImplementedError

    def poll(self, handle) -> Optional[list]:
        """None while the batch runs, else one status per request: "ok" or
        an error text."""
        raise NotImplementedError


class Server:
    def __init__(self, backend: Backend, budget_bytes: int, max_batch: int = 48,
                 max_inflight: int = 2, clock: Callable[[], float] = time.perf_counter,
                 on_done: Optional[Callable[[Request], None]] = None,
                 max_ready: Optional[int] = None, max_batch_bytes: int = 0):
        if max_batch < 1 or max_inflight < 1:
            raise ValueError("max_batch and max_inflight must be >= 1")
        # a batch also ends before its device buffers pass this many bytes
        # (0: no limit), so that a burst of large frames does not become one
        # long launch that every later request waits for
        self.max_batch_bytes = int(max_batch_bytes)
        # admitted requests waiting for a launch: by default one batch
        self.max_ready = max_batch if max_ready is None else max_ready
        self.backend = backend
        self.budget = int(budget_bytes)
        self.max_batch = max_batch
        self.max_inflight = max_inflight
        self.clock = clock
        self.on_done = on_done
        self.queue: collections.deque = collections.deque()   # waiting for admission
        self.ready: list = []                                  # admitted, not launched
        self.inflight: list = []                               # (handle, [requests])
        self.in_use = 0
        self.peak_in_use = 0
        self.batches = 0
        self.batch_sizes: list = []
        self.finished: list = []
        self._by_id: dict = {}
        # host time spent in the backend's calls and in whole loop
        # iterations (wall clock): where a stall of the serving loop sits
        self.host = {"launch": _Stall(), "poll": _Stall(), "reserve": _Stall(), "loop": _Stall()}

    # ------------------------------------------------------------ requests
    def submit(self, req: Request, now: Optional[float] = None) -> bool:
        """Queue a request; False (and status "rejected") if it can never run."""
        req.t_submit = self.clock() if now is None else now
        self._by_id[req.rid] = req
        why = validate_params(req.params, req.width, req.height)
        if why is None and (req.width <= 0 or req.height <= 0 or req.width % 8 or req.height % 8):
            why = "frame size must be a positive multiple of 8"
        if why is None and req.bitdepth not in (8, 10, 12):
            why = "bit depth must be 8, 10 or 12"
        if why is None:
            req.need = self.backend.need_bytes(req)
            if req.need > self.budget:
                why = f"needs {req.need} device bytes, budget is {self.budget}"
        if why is not None:
            self._finish(req, "rejected", why, req.t_submit)
            return False
        req.status = "queued"
        self.queue.append(req)
        return True

    def cancel(self, rid: int) -> bool:
        """Withdraw a request that has not been launched."""
        req = self._by_id.get(rid)
        if req is None or req.status not in ("queued", "admitted"):
            return False
        if req.status == "queued":
            self.queue.remove(req)
        else:
            self.ready.remove(req)
            self._free(req)
        self._finish(req, "cancelled", "", self.clock())
        return True

    # ------------------------------------------------------------ the loop
    def step(self, now: Optional[float] = None) -> bool:
        """One scheduling pass; True if anything changed."""
        now = self.clock() if now is None else now
        progress = False
        # 1. completed batches
        still = []
        for handle, reqs in self.inflight:
            t0 = time.perf_counter()
            res = self.backend.poll(handle)
            self.host["poll"].add(time.perf_counter() - t0)
            if res is None:
                still.append((handle, reqs))
                continue
            progress = True
            for r, st in zip(reqs, res):
                self._free(r)
                if st == "ok":
                    self._finish(r, "ok", "", now)
                else:
                    self._finish(r, "failed", st, now)
        self.inflight = still
        # 2. admission, first come first served, under the budget
        while (self.queue and len(self.ready) < self.max_ready
               and self.in_use + self.queue[0].need <= self.budget):
            r = self.queue.popleft()
            t0 = time.perf_counter()
            self.backend.reserve(r)
            self.host["reserve"].add(time.perf_counter() - t0)
            self.in_use += r.need
            self.peak_in_use = max(self.peak_in_use, self.in_use)
            r.status, r.t_admit = "admitted", now
            self.ready.append(r)
            progress = True
        # 3. continuous batching: launch what is admitted while the device
        #    has room for another batch
        while self.ready and len(self.inflight) < self.max_inflight:
            cut, size = 0, 0
            while cut < min(len(self.ready), self.max_batch):
                size += self.ready[cut].need
                if cut > 0 and self.max_batch_bytes and size > self.max_batch_bytes:
                    break
                cut += 1
            batch, self.ready = self.ready[:cut], self.ready[cut:]
            try:
                t0 = time.perf_counter()
                handle = self.backend.launch(batch)
                self.host["launch"].add(time.perf_counter() - t0)
            except Exception as e:  # noqa: BLE001 - the batch fails, the server goes on
                for r in batch:
                    self._free(r)
                    self._finish(r, "failed", f"launch: {e}", now)
                progress = True
                continue
            for r in batch:
                r.status, r.t_launch = "launched", now
            self.inflight.append((handle, batch))
            self.batches += 1
            self.batch_sizes.append(len(batch))
            progress = True
        return progress

    def idle(self) -> bool:
        return not (self.queue or self.ready or self.inflight)

    def drain(self, timeout: float = 60.0) -> None:
        t_end = self.clock() + timeout
        while not self.idle():
            if not self.step() and self.clock() > t_end:
                raise TimeoutError("requests still pending")

    def run(self, requests: list, timeout: float = 600.0) -> dict:
        """Serve `requests` with real-time arrivals at start + r.arrival and
        return the statistics.  Python's cyclic garbage collector is paused
        for the run (a full collection over thousands of live requests stalls
        the loop for tens of milliseconds)."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        gc_was_on = gc.isenabled()
        gc.collect()
        gc.disable()
        start = self.clock()
        base = self.clock
        self.clock = lambda: base() - start          # run-relative times
        try:
            i, n = 0, len(reqs)
            loop, t_prev = self.host["loop"], time.perf_counter()
            while i < n or not self.idle():
                t = time.perf_counter()
                loop.add(t - t_prev)
                t_prev = t
                now = self.clock()
                if now > timeout:
                    raise TimeoutError(f"{n - len(self.finished)} requests unfinished")
                while i < n and reqs[i].arrival <= now:
                    self.submit(reqs[i], now)
                    i += 1
                if not self.step(now) and self.idle() and i < n:
                    # nothing to do before the next arrival: sleep through
                    # most of the gap, spin the rest (sleep overshoots)
                    gap = reqs[i].arrival - self.clock()
                    if gap > 300e-6:
                        time.sleep(gap - 200e-6)
                        t_prev = time.perf_counter()   # a chosen sleep is no stall
            wall = self.clock()
        finally:
            self.clock = base
            if gc_was_on:
                gc.enable()
        return summarize(reqs, wall, self)

    # ------------------------------------------------------------ internals
    def _free(self, r: Request) -> None:
        if r.slot is not None:
            self.backend.release(r)
            r.slot = None
        if r.status in ("admitted", "launched"):
            self.in_use -= r.need

    def _finish(self, r: Request, status: str, error: str, now: float) -> None:
        r.status, r.error, r.t_done = status, error, now
        self.finished.append(r)
        if self.on_done is not None:
            self.on_done(r)


class _Stall:
    """Durations of one kind of host call: count, total, maximum and how
    many took longer than 5 ms."""
    __slots__ = ("n", "total", "max", "over_5ms")

    def __init__(self):
        self.n, self.total, self.max, self.over_5ms = 0, 0.0, 0.0, 0

    def add(self, dt: float) -> None:
        self.n += 1
        self.total += dt
        if dt > self.max:
            self.max = dt
        if dt > 5e-3:
            self.over_5ms += 1

    def summary(self) -> dict:
        return {"calls": self.n, "total_ms": self.total * 1e3, "max_ms": self.max * 1e3,
                "over_5ms": self.over_5ms}


def percentile(xs, q):
    if not xs:
        return math.nan
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q))


def summarize(reqs, wall: float, server: Server) -> dict:
    ok = [r for r in reqs if r.status == "ok"]
    lat = [r.latency for r in ok]
    # where the slowest 1% spent their time: queued (arrival to admission),
    # admitted (to launch), launched (on the device and copies, to done)
    tail = {}
    if ok:
        cut = percentile(lat, 99)
        slow = [r for r in ok if r.latency >= cut]
        tail = {"queued_ms": float(np.mean([r.t_admit - r.arrival for r in slow])) * 1e3,
                "admitted_ms": float(np.mean([r.t_launch - r.t_admit for r in slow])) * 1e3,
                "launched_ms": float(np.mean([r.t_done - r.t_launch for r in slow])) * 1e3}
    px = sum(r.width * r.height for r in ok)
    counts = collections.Counter(r.status for r in reqs)
    return {
        "requests": len(reqs), "ok": len(ok), "status": dict(counts),
        "wall_s": wall, "frames_per_s": len(ok) / wall if wall > 0 else math.nan,
        "mpixel_per_s": px / wall / 1e6 if wall > 0 else math.nan,
        "p50_ms": percentile(lat, 50) * 1e3, "p99_ms": percentile(lat, 99) * 1e3,
        "mean_ms": float(np.mean(lat)) * 1e3 if lat else math.nan,
        "batches": server.batches,
        "mean_batch": float(np.mean(server.batch_sizes)) if server.batch_sizes else 0.0,
        "peak_device_bytes": server.peak_in_use,
        "buffer_allocs": getattr(server.backend, "allocs", 0),
        "p99_tail": tail,
        "host_calls": {k: v.summary() for k, v in server.host.items()},
        **device_stage_summary(getattr(server.backend, "batch_times", None)),
    }


def device_stage_summary(times) -> dict:
    """The device stage times of a timed CudaBackend's batches: maximum and
    99th percentile of each stage, and the slowest batch end to end."""
    if not times:
        return {}
    a = np.asarray(times, dtype=np.float64)
    out = {}
    for j, name in enumerate(("h2d_ms", "stream_wait_ms", "kernel_ms", "d2h_ms", "d2h_wait_ms",
                              "d2h_frames_ms", "d2h_status_ms"), start=2):
        out[name] = {"max": float(a[:, j].max()), "p99": float(np.percentile(a[:, j], 99)),
                     "mean": float(a[:, j].mean())}
    k = int(np.argmax(a[:, 2:6].sum(axis=1)))
    out["slowest_batch"] = {"frames": int(a[k, 0]), "bytes": int(a[k, 1]),
                            "stages_ms": [float(x) for x in a[k, 2:]]}
    times.clear()
    return {"device_stages": out}


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process of `rate` requests/s."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n))


# ---------------------------------------------------------------- CUDA
class CudaBackend(Backend):
    """Device buffers, copies and launches for the server.

    Each request's input frame and parameters travel in one host-to-device
    copy into one flat device buffer, and its output in one device-to-host
    copy into a pinned host buffer (``req.out``, valid once the request is
    done).  Buffers are cached per (size, bit depth) and reused; cached free
    buffers are dropped when a new size needs the room, so that the device
    memory held never exceeds the server's budget."""

    def __init__(self, ctx, budget_bytes: int, device: int = 0, timing: bool = False):
        import torch
        from . import cdef
        self.torch, self.cdef, self.ctx = torch, cdef, ctx
        self.device = torch.device("cuda", device)
        self.budget = budget_bytes
        self.up = torch.cuda.Stream(device=self.device)
        self.comp = torch.cuda.Stream(device=self.device)
        self.down = torch.cuda.Stream(device=self.device)
        self.free: dict = collections.defaultdict(list)   # key -> [slot]
        self.free_bytes = 0
        self.held_bytes = 0
        self.host_out: dict = collections.defaultdict(list)
        self.allocs = 0         # buffer sets allocated while serving (after prewarm)
        # status words of the batches in flight, copied back on the
        # device-to-host stream (no synchronous call in the loop)
        self.status_words = torch.zeros(256, dtype=torch.int32).pin_memory()
        self.next_word = 0
        # the events of each batch, reused round-robin with the status words
        # (a ring far longer than the batches in flight).  With `timing`,
        # four more (copy start, kernel start, read-back start, frames read
        # back) and every batch's stage times are kept in `batch_times`:
        # (frames, bytes, host-to-device ms, wait for the kernel stream ms,
        # kernel ms, device-to-host ms, of which: wait for the read-back
        # stream, the frames' copies, the status word's copy).
        self.timing = timing
        self.batch_times: list = []
        self.events = [tuple(torch.cuda.Event(enable_timing=timing) for _ in range(7 if timing else 3))
                       for _ in range(self.status_words.numel())]

    @staticmethod
    def key(req: Request):
        return (req.width, req.height, req.bitdepth)

    def _sizes(self, req: Request):
        n_params = (-(-req.height // 64)) * (-(-req.width // 64)) * 8
        _, in_b = self.cdef.packed_layout(req.width, req.height, req.bitdepth, n_params)
        _, out_b = self.cdef.packed_layout(req.width, req.height, req.bitdepth)
        return n_params, in_b, out_b

    def need_bytes(self, req: Request) -> int:
        _, in_b, out_b = self._sizes(req)
        return in_b + out_b

    def prewarm(self, shapes, count: int, fill: float = 0.0) -> None:
        """Allocate device and pinned host buffer sets up front, so that no
        allocation (a pinned host allocation of a 4K frame takes tens of
        milliseconds) happens while serving: `count` sets of each (width,
        height, bitdepth), then more, one of each shape in turn, until
        `fill` of the budget is held."""
        dummy = []

        def take(w, h, bd):
            rows, cols = -(-h // 64), -(-w // 64)
            r = Request(-1, w, h, bd, None, np.zeros((rows, cols, 8), np.uint8))
            r.need = self.need_bytes(r)
            if self.held_bytes + r.need > self.budget:
                return False
            self.reserve(r)
            dummy.append(r)
            return True

        for w, h, bd in shapes:
            for _ in range(count):
                if not take(w, h, bd):
                    break
        grew = True
        while grew and self.held_bytes < fill * self.budget:
            grew = False
            for w, h, bd in shapes:
                if self.held_bytes < fill * self.budget and take(w, h, bd):
                    grew = True
        for r in dummy:
            self.release(r)
        self.allocs = 0

    def reserve(self, req: Request) -> None:
        k = self.key(req)
        if self.free[k]:
            req.slot = self.free[k].pop()
            self.free_bytes -= req.need
        else:
            # drop cached buffers of other sizes until the new one fits
            for kk in list(self.free):
                while self.held_bytes + req.need > self.budget and self.free[kk]:
                    s = self.free[kk].pop()
                    self.held_bytes -= s["bytes"]
                    self.free_bytes -= s["bytes"]
            n_params, _, _ = self._sizes(req)
            self.allocs += 1
            flat_in, f_in, prm = self.cdef.alloc_packed(req.width, req.height, req.bitdepth,
                                                        device=self.device, extra_bytes=n_params)
            flat_out, f_out, _ = self.cdef.alloc_packed(req.width, req.height, req.bitdepth,
                                                        device=self.device)
            planes, _ = self.cdef.packed_layout(req.width, req.height, req.bitdepth)
            req.slot = {"flat_in": flat_in, "in": f_in, "params": prm, "flat_out": flat_out,
                        "out": f_out, "bytes": req.need,
                        "in_planes": flat_in[:planes[3]]}   # the planes, without parameters
            self.held_bytes += req.need
        hk = self.host_out[k]
        req.slot["host_out"] = hk.pop() if hk else self.cdef.alloc_packed(
            req.width, req.height, req.bitdepth, device="cpu", pin=True)

    def release(self, req: Request) -> None:
        s = req.slot
        self.host_out[self.key(req)].append(s.pop("host_out"))
        self.free[self.key(req)].append(s)
        self.free_bytes += s["bytes"]

    def launch(self, reqs: list):
        torch = self.torch
        for r in reqs:
            if r.params_host is None:
                r.params_host = torch.from_numpy(
                    np.ascontiguousarray(r.params, dtype=np.uint8).reshape(-1)).pin_memory()
        evs = self.events[self.next_word]
        ev_up, ev_c, ev_d = evs[:3]
        word = self.status_words[self.next_word:self.next_word + 1]
        self.next_word = (self.next_word + 1) % self.status_words.numel()
        if self.timing:
            evs[3].record(self.up)
        with torch.cuda.stream(self.up):
            for r in reqs:
                r.slot["in_planes"].copy_(r.frame, non_blocking=True)
                r.slot["params"].copy_(r.params_host, non_blocking=True)
        ev_up.record(self.up)
        self.comp.wait_event(ev_up)
        if self.timing:
            evs[4].record(self.comp)
        self.cdef.cdef_filter_frames(self.ctx, [r.slot["in"] for r in reqs],
                                     [r.slot["params"] for r in reqs],
                                     [r.slot["out"] for r in reqs], stream=self.comp)
        ev_c.record(self.comp)
        down = self.down
        down.wait_event(ev_c)
        if self.timing:
            evs[5].record(down)
        with torch.cuda.stream(down):
            for r in reqs:
                r.slot["host_out"][0].copy_(r.slot["flat_out"], non_blocking=True)
        if self.timing:
            evs[6].record(down)
        self.ctx.status_async(word, stream=down)
        ev_d.record(down)
        # keep the host output reachable from the request once it is done
        for r in reqs:
            r.out = r.slot["host_out"]
        return (ev_d, len(reqs), word, evs, sum(r.need for r in reqs))

    def poll(self, handle):
        ev, n, word, evs, nbytes = handle
        if not ev.query():
            return None
        if self.timing:
            up, c, d, s0, k0, d0, d1 = evs
            self.batch_times.append((n, nbytes, s0.elapsed_time(up), up.elapsed_time(k0),
                                     k0.elapsed_time(c), c.elapsed_time(d), c.elapsed_time(d0),
                                     d0.elapsed_time(d1), d1.elapsed_time(d)))
        # The context's status word collects device-side parameter errors.
        # Requests are validated on the host before they are queued, so it
        # stays 0; if it is ever set, the batch that saw it fails (and the
        # word is read and cleared synchronously).
        if int(word[0]) == 0:
            return ["ok"] * n
        st = self.ctx.status()
        return [f"device status {st}"] * n


def pack_frame(cdef, frame_planes, bitdepth: int):
    """A frame's planes (uint16 numpy y, u, v) in one pinned host buffer in
    the packed layout :class:`CudaBackend` copies."""
    import torch
    h, w = frame_planes[0].shape
    flat, f, _ = cdef.alloc_packed(w, h, bitdepth, device="cpu")
    flat.zero_()
    for t, a in zip(f.planes(), frame_planes):
        a = np.asarray(a)
        if bitdepth == 8:
            t[:, :a.shape[1]] = torch.from_numpy(a.astype(np.uint8))
        else:
            t[:, :a.shape[1]] = torch.from_numpy(a.astype(np.uint16).view(np.int16))
    return flat.pin_memory()


def unpack_frame(out) -> tuple:
    """Copies of the visible planes of a CudaBackend output as uint16 arrays."""
    return tuple(np.array(p, dtype=np.uint16) for p in out[1].to_numpy())
