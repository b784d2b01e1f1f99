"""Throughput benchmark of the CDEF hot path on GB300.

Default workload: 3840x2160 10-bit 4:2:0, 8 frames, direction search +
filter, one fused launch per frame, streamed on one CUDA stream (the 4K
10-bit case the HBM-roofline target is stated for).  A step filters all 8
frames.  Metric: luma megapixels per second (chroma work included).

Prints ONE JSON line (rank 0).  Keys beyond the metric:
  roofline      HBM roofline of the dominant kernel (the fused filter):
                algorithmic bytes per launch (every input sample read once,
                every output sample written once) / mean launch time from
                CUDA events on the launching stream, against the measured
                copy bandwidth
  cpu_baseline  the C oracle timed on this host's cores on a bounded sample
                of the same frames
  e2e           same metric through the C ABI with host buffers: pinned
                host -> device copy, filter, device -> host copy per frame,
                all inside the timed region
  clocks        nvidia-smi samples taken during the timed region

--impl reference times the oracle (the reference arm of this benchmark).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpixel/s (find_dir+filter)"
UNIT = "Mpixel/s"
KERNEL_SOURCES = ["paper_1602_05975_gb300/csrc/filter.cu",
                  "paper_1602_05975_gb300/csrc/tile.cuh",
                  "paper_1602_05975_gb300/csrc/tma.cuh",
                  "paper_1602_05975_gb300/csrc/cdef_device.cuh"]


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:  # noqa: BLE001
        return None


def ncu_traffic(kernel: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.txt")))
    except Exception:  # noqa: BLE001
        return None
    e = d.get(kernel)
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return e


# ------------------------------------------------------------------ workload
FILTER_WORKLOADS = {
    "filter": dict(name="3840x2160 10-bit 4:2:0, 8 frames, direction search + filter, "
                        "one launch per frame",
                   width=3840, height=2160, bitdepth=10, frames=8, base_seed=2000),
    "filter1080p": dict(name="1920x1080 8-bit 4:2:0, 30 frames, direction search + filter, "
                             "one launch per frame",
                        width=1920, height=1080, bitdepth=8, frames=30, base_seed=1000),
    "filter444": dict(name="1920x1080 8-bit 4:4:4, 30 frames, direction search + filter "
                           "(full-resolution chroma), one launch per frame",
                      width=1920, height=1080, bitdepth=8, frames=30, base_seed=5000, chroma=444),
    "filter12": dict(name="3840x2160 12-bit 4:2:0, 8 frames, direction search + filter, "
                          "one launch per frame",
                     width=3840, height=2160, bitdepth=12, frames=8, base_seed=6000),
}
WORKLOAD = FILTER_WORKLOADS["filter"]


def frame_seeds(rank: int = 0):
    """Seeds of one replica's frames: every rank filters its own frames."""
    return [WORKLOAD["base_seed"] + 100 * rank + f for f in range(WORKLOAD["frames"])]


def make_frames(rank: int = 0):
    from paper_1602_05975_gb300 import synth
    w, h, bd = WORKLOAD["width"], WORKLOAD["height"], WORKLOAD["bitdepth"]
    return [synth.make_frame(w, h, bd, None, s, WORKLOAD.get("chroma", 420))
            for s in frame_seeds(rank)]


def workload_samples() -> int:
    from paper_1602_05975_gb300 import synth
    w, h = WORKLOAD["width"], WORKLOAD["height"]
    cw, ch = synth.chroma_dims(w, h, WORKLOAD.get("chroma", 420))
    return w * h + 2 * cw * ch


def max_over_ranks(x: float, device=None) -> float:
    """The largest of every rank's x (the job's time); x itself on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws: int, units_per_rank: float, ms_per_step: float) -> float:
    """Units per second over all ranks (weak scaling: each rank does its own
    units per step), in millions."""
    return ws * units_per_rank / (ms_per_step * 1e-3) / 1e6


def algorithmic_bytes_per_frame() -> int:
    return workload_samples() * (1 if WORKLOAD["bitdepth"] == 8 else 2) * 2


# The method's integer operations (Eq. 1-12): per filtered sample (luma or
# chroma) 12 taps x 8 (difference, magnitude, shift, subtraction, clamp at 0,
# minimum, sign, weighted accumulation), 24 for the clip range over the taps,
# 4 for the rounding of Eq. 8 and the addition, 2 for the clip; per luma 8x8
# block the direction search's 376 additions, 124 multiplications and 7
# comparisons (section 2's count), 64 or 128 (shift first above 8 bits) for
# the offset of the samples and 1 for the contrast.
OPS_PER_SAMPLE = 12 * 8 + 24 + 4 + 2


def algorithmic_ops_per_frame() -> int:
    w, h, bd = WORKLOAD["width"], WORKLOAD["height"], WORKLOAD["bitdepth"]
    filtered = w * h if WORKLOAD.get("chroma", 420) == 422 else workload_samples()
    search_per_block = 376 + 124 + 7 + 64 * (1 if bd == 8 else 2) + 1
    return filtered * OPS_PER_SAMPLE + (w // 8) * (h // 8) * search_per_block


def alu_peak_gops(bitdepth: int = 8) -> float:
    """152 SMs x 4 schedulers x 32 lanes issue one 32-bit operation each per
    clock at 2070 MHz; every value of the 8/10-bit path fits 16 bits, so a
    lane can carry two of the method's operations (12-bit values do not)."""
    return 152 * 4 * 32 * (2 if bitdepth <= 10 else 1) * 2.07


# ------------------------------------------------------------------ oracle (CPU)
BAND = 120  # rows per oracle task (a multiple of 8)


def _oracle_band(args):
    """Filter one horizontal band of a frame with the oracle (as a frame of
    its own).  Returns (luma pixels, seconds)."""
    planes, bd, params, fmt = args
    from oracle import ref
    t = time.perf_counter()
    if fmt == 420:
        ref.filter_frame(*planes, bd, params)
    else:
        ref.filter_frame_format(*planes, bd, params, fmt)
    return planes[0].shape[0] * planes[0].shape[1], time.perf_counter() - t


def oracle_tasks(frames, nbands):
    tasks = []
    for fr in frames:
        h = fr.height
        for b0 in range(0, h, BAND):
            if len(tasks) >= nbands:
                return tasks
            b1 = min(h, b0 + BAND)
            y = fr.rec[0][b0:b1]
            fmt = WORKLOAD.get("chroma", 420)
            c0, c1 = (b0 // 2, b1 // 2) if fmt == 420 else (b0, b1)
            u = fr.rec[1][c0:c1]
            v = fr.rec[2][c0:c1]
            rows = [(b0 // 64 + k) % fr.params.shape[0] for k in range(-(-(b1 - b0) // 64))]
            prm = np.ascontiguousarray(fr.params[rows])
            tasks.append(((y, u, v), fr.bitdepth, prm, fmt))
    return tasks


def run_oracle(pool, cores, frames, nbands):
    from oracle import ref
    ref.build()
    tasks = oracle_tasks(frames, nbands)
    t = time.perf_counter()
    res = pool.map(_oracle_band, tasks, chunksize=1)
    wall = time.perf_counter() - t
    px = sum(r[0] for r in res)
    return px / wall / 1e6, px, wall, sum(r[1] for r in res)


def oracle_sample(frames, nbands) -> str:
    n = len(oracle_tasks(frames, nbands))
    total = sum(-(-f.height // BAND) for f in frames)
    what = "all" if n == total else f"{n} of the {total}"
    return (f"{what} {WORKLOAD['width']}x{BAND} bands (luma + chroma) of the {len(frames)} "
            f"{WORKLOAD['width']}x{WORKLOAD['height']} {WORKLOAD['bitdepth']}-bit frames, "
            f"one band per task, each filtered as a frame of its own by the oracle")


# ------------------------------------------------------------------ clocks
def _smi_time(stamp: str):
    """nvidia-smi's `YYYY/MM/DD hh:mm:ss.mmm` local time → epoch seconds."""
    try:
        whole, _, frac = stamp.partition(".")
        return time.mktime(time.strptime(whole, "%Y/%m/%d %H:%M:%S")) + float("0." + (frac or "0"))
    except Exception:  # noqa: BLE001
        return None


class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        if getattr(self, "disabled", False):
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:  # noqa: BLE001
            self.proc = None

    def mark(self, which: str):
        """Host wall-clock bounds of the timed region."""
        setattr(self, which, time.time())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:  # noqa: BLE001
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 10:
                parts[0] = _smi_time(parts[0])
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        # samples taken while the timed region ran (the nearest one if the
        # region was shorter than the sampling period)
        t0, t1 = getattr(self, "begin", None), getattr(self, "end", None)
        inside = rows
        if t0 is not None and t1 is not None and all(r[0] is not None for r in rows):
            inside = [r for r in rows if t0 - 0.05 <= r[0] <= t1 + 0.05]
            if not inside:
                mid = 0.5 * (t0 + t1)
                inside = [min(rows, key=lambda r: abs(r[0] - mid))]
        sm = [float(r[2]) for r in inside if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in inside for n, v in zip(names, r[6:10])
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(inside)}


# ------------------------------------------------------------------ main arms
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_1602_05975_gb300 import synth  # noqa: F401
    cores = min(os.cpu_count() or 1, 16)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        frames = make_frames()
        nb = args.cpu_bands or 10**9
        for _ in range(args.warmup):
            run_oracle(pool, cores, frames, nb)
        pxs, walls = 0, 0.0
        for _ in range(args.steps):
            v, px, wall, _ = run_oracle(pool, cores, frames, nb)
            pxs += px
            walls += wall
    value = pxs / walls / 1e6
    sample = f"per step, {oracle_sample(frames, nb)}"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": walls / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD["name"], "sample": "bounded oracle sample",
                   "inputs_sha256": synth.digest_of(frames)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_ours(args):
    ws, rank, local = dist_env()
    pool = None
    cores = 0
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # spawn the oracle pool before any CUDA work
        cores = min(os.cpu_count() or 1, 16)
        pool = mp.get_context("spawn").Pool(cores)

    import torch
    from paper_1602_05975_gb300 import build, cdef
    build.build()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = cdef.Context(local)
    # the frames of a sequence are filtered independently: consecutive calls
    # on the stream may overlap (programmatic dependent launch, no wait)
    ctx.set_overlap(not args.no_overlap)

    frames = make_frames(rank)
    nf = len(frames)
    from paper_1602_05975_gb300 import synth
    inputs_sha = synth.digest_of(frames)   # SHA-256 over the frames' digests
    ins = [cdef.frame_from_numpy(f.rec, f.bitdepth, device=dev) for f in frames]
    # two output sets, alternating by step: no two filter calls that may run
    # concurrently (overlapped launches) write the same buffer
    fmt = WORKLOAD.get("chroma", 420)
    out_sets = [[cdef.alloc_frame(f.width, f.height, f.bitdepth, device=dev, fill=0, chroma=fmt)
                 for f in frames] for _ in range(2)]
    outs = out_sets[0]
    prms = [cdef.params_tensor(f.params, device=dev) for f in frames]
    stream = torch.cuda.Stream(device=dev)
    px_per_frame = WORKLOAD["width"] * WORKLOAD["height"]

    parity = [0]

    def step(evs=None):
        o = out_sets[parity[0]]
        parity[0] ^= 1
        for i in range(nf):
            if evs is not None:
                evs[i][0].record(stream)
            cdef.cdef_filter_frame(ctx, ins[i], prms[i], o[i], stream=stream)
            if evs is not None:
                evs[i][1].record(stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()

    # parity spot check of the benchmark's own launch configuration
    got = outs[0].to_numpy()
    if args.check:
        from oracle import ref
        exp = (ref.filter_frame(*frames[0].rec, frames[0].bitdepth, frames[0].params) if fmt == 420
               else ref.filter_frame_format(*frames[0].rec, frames[0].bitdepth, frames[0].params,
                                            fmt))
        for g, e in zip(got, exp):
            assert np.array_equal(g, e), "bench output differs from the oracle"

    # isolated launches (events around each, calls not overlapped): the
    # kernel's own duration, untimed for the headline
    ctx.set_overlap(False)
    evs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(nf)] for _ in range(min(args.steps, 10))]
    with torch.cuda.stream(stream):
        for row in evs:
            step(row)
    torch.cuda.synchronize()
    isolated_ms = [a.elapsed_time(b) for row in evs for (a, b) in row]
    ctx.set_overlap(not args.no_overlap)
    with torch.cuda.stream(stream):
        step()

    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    clocks.mark("begin")
    t0.record(stream)
    for k in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    clocks.mark("end")
    clk = clocks.stop()
    ms = t0.elapsed_time(t1)
    ms = max_over_ranks(ms, dev)
    ms_per_step = ms / args.steps
    value = whole_job_rate(ws, nf * px_per_frame, ms_per_step)
    assert ctx.status() == 0

    # e2e: host buffers, copies inside the timed region, 3 streams in flight
    e2e = None
    if not args.no_e2e:
        hin = [cdef.frame_from_numpy(f.rec, f.bitdepth, device="cpu", pin=True) for f in frames]
        hout = [cdef.alloc_frame(f.width, f.height, f.bitdepth, device="cpu", chroma=fmt)
                for f in frames]
        hout = [cdef.Frame(*(t.pin_memory() for t in h.planes()), h.width, h.height, h.bitdepth,
                           h.chroma) for h in hout]
        streams = [torch.cuda.Stream(device=dev) for _ in range(3)]
        h2d = sum(t.numel() * t.element_size() for h in hin for t in h.planes())
        d2h = sum(t.numel() * t.element_size() for h in hout for t in h.planes())

        def e2e_step():
            for i in range(nf):
                s = streams[i % len(streams)]
                with torch.cuda.stream(s):
                    for dt, st in zip(ins[i].planes(), hin[i].planes()):
                        dt.copy_(st, non_blocking=True)
                    cdef.cdef_filter_frame(ctx, ins[i], prms[i], outs[i], stream=s)
                    for st, dt in zip(hout[i].planes(), outs[i].planes()):
                        st.copy_(dt, non_blocking=True)

        for _ in range(args.warmup):
            e2e_step()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        tt0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        e_ms = (time.perf_counter() - tt0) * 1e3
        e_ms = max_over_ranks(e_ms, dev)
        e2e = {"value": whole_job_rate(ws, nf * px_per_frame, e_ms / args.steps), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

        # the same copies without the filter: the ceiling the link sets
        def copy_step():
            for i in range(nf):
                s = streams[i % len(streams)]
                with torch.cuda.stream(s):
                    for dt, st in zip(ins[i].planes(), hin[i].planes()):
                        dt.copy_(st, non_blocking=True)
                    for st, dt in zip(hout[i].planes(), outs[i].planes()):
                        st.copy_(dt, non_blocking=True)

        for _ in range(args.warmup):
            copy_step()
        torch.cuda.synchronize()
        tt0 = time.perf_counter()
        for _ in range(args.steps):
            copy_step()
        torch.cuda.synchronize()
        c_ms = max_over_ranks((time.perf_counter() - tt0) * 1e3, dev)
        e2e["copies_only"] = {
            "value": whole_job_rate(ws, nf * px_per_frame, c_ms / args.steps), "unit": UNIT,
            "gb_per_s": (h2d + d2h) / (c_ms / args.steps * 1e-3) / 1e9,
            "what": "the same host-device copies per step without the filter"}
        for h, o in zip(hout[:1], outs[:1]):
            assert all(np.array_equal(a, b) for a, b in zip(h.to_numpy(), o.to_numpy()))

    peaks = measured_peaks()
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    # the kernel's own duration: CUDA events around each launch, launches
    # not overlapped; beside it the share of the timed region per launch
    # (consecutive frames' launches overlap there: a throughput figure)
    launch_ms = statistics.mean(isolated_ms)
    share_ms = ms_per_step / nf
    ops_b = algorithmic_ops_per_frame()
    bytes_b = algorithmic_bytes_per_frame()
    peak_ops = alu_peak_gops(WORKLOAD["bitdepth"])
    traffic = ncu_traffic("filter_kernel") if WORKLOAD is FILTER_WORKLOADS["filter"] else None
    ops = ops_b / (launch_ms * 1e-3) / 1e9
    achieved = bytes_b / (launch_ms * 1e-3) / 1e9
    roofline = {"bound": "alu", "achieved": ops, "peak": peak_ops, "unit": "Gop/s",
                "frac": ops / peak_ops,
                "traffic": (traffic or {}).get("dram_bytes_per_launch"),
                "traffic_note": (traffic or {}).get("note"),
                "kernel": "filter_kernel (fused find_dir + filter)",
                "ops_per_launch": ops_b,
                "peak_source": "derived: 152 SMs x 128 lanes x 2 (16-bit pairs) x 2070 MHz"
                if WORKLOAD["bitdepth"] <= 10 else "derived: 152 SMs x 128 lanes x 2070 MHz",
                "hbm": {"achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                        "peak_source": "measured" if peaks else "fallback"},
                "bytes_per_launch": bytes_b,
                "launch_us": launch_ms * 1e3,
                "launch_time": "mean of CUDA events around each launch, launches not overlapped",
                "overlapped": {
                    "share_us": share_ms * 1e3,
                    "achieved": ops_b / (share_ms * 1e-3) / 1e9,
                    "frac": ops_b / (share_ms * 1e-3) / 1e9 / peak_ops,
                    "hbm_frac": bytes_b / (share_ms * 1e-3) / 1e9 / hbm,
                    "what": "timed region / launches: consecutive frames' launches overlap "
                            "(programmatic dependent launch), the tail of one filling the SMs "
                            "the next starts on" if not args.no_overlap
                            else "timed region / launches"}}
    # beside the derived ceiling, the measured one: the integer issue rate
    # of the filter's tap instruction mix on this GPU (probe kernel)
    if WORKLOAD["bitdepth"] <= 10:
        mix = cdef.probe_int_mix(ctx, 0)
        alu_only = cdef.probe_int_mix(ctx, 1)
        peak_mix = 2 * mix / 1e9   # two 16-bit lanes per lane instruction, Gop/s
        roofline["measured_int_ceiling"] = {
            "peak": peak_mix, "unit": "Gop/s",
            "frac": ops / peak_mix, "frac_overlapped": ops_b / (share_ms * 1e-3) / 1e9 / peak_mix,
            "tap_mix_lane_instr_per_s": mix, "alu_only_lane_instr_per_s": alu_only,
            "what": "cdef_probe_int_mix: the tap's 6 ALU operations and 2 multiply-adds "
                    "in independent chains, 4 CTAs of 256 threads per SM, CUDA events"}

    cpu = None
    if pool is not None:
        nb = args.cpu_bands or 10**9
        v, px, wall, cpu_s = run_oracle(pool, cores, frames, nb)
        reps = 1
        while not args.cpu_bands and cpu_s < 10.0 and reps < 3:
            # fast host: the whole step again, so that the sample is >= 10 s of CPU work
            _, px2, wall2, cpu2 = run_oracle(pool, cores, frames, nb)
            px, wall, cpu_s, reps = px + px2, wall + wall2, cpu_s + cpu2, reps + 1
        v = px / wall / 1e6
        pool.close()
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{oracle_sample(frames, nb)}" + (f", {reps} times" if reps > 1 else "") +
                         f": {px / 1e6:.1f} Mpixel, "
                         f"{cpu_s:.1f} s of CPU work in {wall:.1f} s wall"}

    # the other headline workloads (strength search, serving) on one GPU,
    # after the filter's timed region, each with its own clock record
    extra = None
    if ws == 1 and not args.no_extras and WORKLOAD is FILTER_WORKLOADS["filter"]:
        extra = {"search": search_extra(args), "serve": serve_extra(args)}

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "frames_per_step": nf,
                       "width": WORKLOAD["width"], "height": WORKLOAD["height"],
                       "bitdepth": WORKLOAD["bitdepth"], "parallelism": f"replicas x{ws}",
                       "inputs_sha256": inputs_sha,
                       "l2": f"each frame's buffers are touched once per step and "
                             f"{(nf - 1) * algorithmic_bytes_per_frame() / 1e6:.0f} MB of "
                             f"other frames' traffic (L2: 129 MB) passes between two uses"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": args.steps * nf,
            "extra": extra,
        }))
    if ws > 1:
        dist.destroy_process_group()
    ctx.close()


SEARCH_WORKLOAD = dict(
    name="strength search: 16 frames 8-bit 4:2:0, 640x360 / 1280x720 / 1920x1080 (6/5/5), "
         "64 luma + 64 chroma strength pairs per 64x64 block, greedy presets, one call",
    sizes=[(640, 360), (1280, 720), (1920, 1080)], frames=16, base_seed=3000)


# The strength search's operations per sample and plane group (section 5 on
# Eq. 7-12, evaluated the factored way: every candidate's filter sum is a
# primary sum plus a secondary sum): 16 primary strengths x 4 taps x 8 and
# 3 non-zero secondary strengths x 8 taps x 8 constraint operations, 24 for
# the clip range, then per candidate 8 (sum of the two sets, rounding of
# Eq. 8, clip, error, square and accumulation).  Eq. 14 adds the filtered
# sum and sum of squares per candidate (3); the 128-combination search adds
# the (19, 7) preset's 12 taps and the uncoded part's accumulation per
# candidate (1).  Per luma 8x8 block: the direction search as in the filter.
def search_ops_per_sample(variant: str) -> int:
    per_cand = {"sse": 8, "eq14": 11, "coded": 9, "444": 8, "12bit": 8, "444coded": 9,
                "444eq14": 11, "12biteq14": 11}[variant]
    extra = 12 * 8 if variant in ("coded", "444coded") else 0
    return 16 * 4 * 8 + 3 * 8 * 8 + 24 + 64 * per_cand + extra


def search_ops(frames, variant: str) -> int:
    ops = 0
    for f in frames:
        cw, ch = (f.width, f.height) if variant.startswith("444") else (f.width // 2, f.height // 2)
        samples = f.width * f.height + 2 * cw * ch
        ops += samples * search_ops_per_sample(variant) + (f.width // 8) * (f.height // 8) * (
            376 + 124 + 7 + 64 + 1)
    return ops


def _oracle_search(task):
    """One frame's strength search by the oracle (a worker process).
    Returns (candidate evaluations, CPU seconds)."""
    w, h, seed, damping, lam, variant, passes, coded = task
    from oracle import ref
    from paper_1602_05975_gb300 import synth
    bd, fmt = search_variant_format(variant)
    f = synth.make_frame(w, h, bd, None, seed, fmt)
    t = time.process_time()
    if variant in ("444eq14", "12biteq14"):
        dl, dc = ref.distortion_eq14_format(f.rec, f.src, bd, damping, fmt)
        ref.select_presets_general(dl, dc, 64, None, lam, passes)
    elif variant == "444coded":
        ref.search_strengths_coded_format(f.rec, f.src, bd, damping, lam, fmt, coded, passes)
    elif variant in ("444", "12bit"):
        ref.search_strengths_format(f.rec, f.src, bd, damping, lam, fmt, passes)
    elif variant == "eq14":
        ref.search_strengths_eq14(f.rec, f.src, 8, damping, lam, passes)
    elif variant == "coded":
        ref.search_strengths_coded(f.rec, f.src, 8, damping, lam, coded, passes)
    else:
        ref.search_strengths(f.rec, f.src, 8, damping, lam, passes)
    blocks = -(-w // 64) * -(-h // 64)
    return blocks * 2 * (128 if variant.endswith("coded") else 64), time.process_time() - t


def search_variant_format(variant: str):
    """(bit depth, chroma format) of the search workload's frames."""
    return {"444": (8, 444), "444coded": (8, 444), "12bit": (12, 420), "444eq14": (8, 444),
            "12biteq14": (12, 420)}.get(variant, (8, 420))


def run_search(args):
    """Batched strength search over 16 mixed-size frames in one call;
    metric: candidate (block, strength combination, plane group) evaluations
    per second, 128 per 64x64 block (256 in the search over coded-residual
    maps, where the skip-condition bit doubles the combinations)."""
    pool = None
    if not args.no_cpu_baseline:
        # spawn the oracle pool before any CUDA work
        from oracle import ref
        ref.build()
        pool = mp.get_context("spawn").Pool(min(os.cpu_count() or 1, 16))
    print(json.dumps(measure_search(args, args.search_variant, args.steps, args.warmup, pool)))


def measure_search(args, variant, steps, warmup, pool=None):
    """The search workload's measurement (see run_search): the batched call
    timed with the L2 flushed before each call, its stages by CUDA events
    inside the search graph, and the one-call-per-frame path on the same
    frames; returns the bench line as a dict."""
    import torch
    from paper_1602_05975_gb300 import build, cdef, synth
    build.build()
    ctx = cdef.Context(0)
    ctx.set_search_refine(args.refine)
    if variant.endswith("eq14"):
        ctx.set_search_metric("eq14")
    bd, fmt = search_variant_format(variant)
    frames = []
    for f in range(SEARCH_WORKLOAD["frames"]):
        w, h = SEARCH_WORKLOAD["sizes"][f % 3]
        frames.append(synth.make_frame(w, h, bd, None, SEARCH_WORKLOAD["base_seed"] + f, fmt))
    recs = [cdef.frame_from_numpy(fr.rec, bd) for fr in frames]
    srcs = [cdef.frame_from_numpy(fr.src, bd) for fr in frames]
    nb = sum(fr.params.shape[0] * fr.params.shape[1] for fr in frames)
    damping = [4 + (fr.q > 16) + (fr.q > 32) for fr in frames]   # larger damping for larger Q
    lambdas = [fr.q * fr.q for fr in frames]
    coded_variant = variant.endswith("coded")
    width = 128 if coded_variant else 64               # table entries per block and group
    ids = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    dl = torch.zeros(nb * width, dtype=torch.int64, device="cuda")
    dc = torch.zeros(nb * width, dtype=torch.int64, device="cuda")
    maps = []
    if coded_variant:
        # coded-residual flags: 60% of the 8x8 blocks, one in eight filter blocks fully skipped
        rng = np.random.default_rng(SEARCH_WORKLOAD["base_seed"])
        for fr in frames:
            m = (rng.random((fr.height // 8, fr.width // 8)) < 0.6).astype(np.uint8)
            m[::16, ::16] = 0
            fb = (m.shape[0] + 7) // 8, (m.shape[1] + 7) // 8
            for by in range(fb[0]):
                for bx in range(fb[1]):
                    if (by * fb[1] + bx) % 8 == 3:
                        m[by * 8:by * 8 + 8, bx * 8:bx * 8 + 8] = 0
            maps.append(torch.from_numpy(m.reshape(-1)).cuda())
    stream = torch.cuda.Stream()

    def call(sl=slice(None)):
        a = int(starts[sl.start or 0])
        b = int(starts[len(frames) if sl.stop is None else sl.stop])
        args_ = (recs[sl], srcs[sl])
        if coded_variant:
            args_ += (maps[sl],)
        return (cdef.cdef_search_strengths_coded if coded_variant
                else cdef.cdef_search_strengths)(
            ctx, *args_, damping[sl], lambdas[sl], ids[a:b], dl[a * width:b * width],
            dc[a * width:b * width], stream=stream)

    starts = np.cumsum([0] + [fr.params.shape[0] * fr.params.shape[1] for fr in frames])
    for _ in range(warmup):
        call()
    if args.check and variant == "sse":
        from oracle import ref
        o = ref.search_strengths(frames[0].rec, frames[0].src, 8, damping[0], lambdas[0])
        n0 = frames[0].params.shape[0] * frames[0].params.shape[1]
        assert (dl[:n0 * 64].cpu().numpy().reshape(n0, 64) == o["dist_luma"]).all()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    # inputs (49 MB) fit in L2: flush it (write 256 MB) before every timed call
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed(fn):
        flush.fill_(1)
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t, r

    clocks.mark("begin")
    call_s = [timed(call)[0] for _ in range(steps)]
    sec = sum(call_s) / steps
    clocks.mark("end")
    clk = clocks.stop()
    tune = ctx.tuning()
    # the distortion kernel's own time: events around it in the search graph
    ctx.set_stage_timing(True)
    stage = []
    for _ in range(steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        call()
        stage.append(ctx.stage_times())
    ctx.set_stage_timing(False)
    dist_ms = statistics.mean(t[0] for t in stage)
    pre_ms = statistics.mean(t[1] for t in stage)
    batched = [dl.clone(), dc.clone(), ids.clone()]
    res_b = call()

    # the plain path: one call (one frame) at a time, same outputs
    def plain():
        out = []
        for i in range(len(frames)):
            out += call(slice(i, i + 1))
        return out

    for _ in range(warmup):
        plain()
    plain_sec = 0.0
    plain_s = []
    for _ in range(steps):
        dt, res_p = timed(plain)
        plain_sec += dt / steps
        plain_s.append(dt)
    same = (res_p == res_b and torch.equal(batched[0], dl) and torch.equal(batched[1], dc)
            and torch.equal(batched[2], ids))
    assert same, "batched and one-frame-at-a-time searches differ"
    assert ctx.status() == 0
    ops = search_ops(frames, variant)
    peak_ops = alu_peak_gops(bd)
    roofline = {"bound": "alu", "achieved": ops / (dist_ms * 1e-3) / 1e9, "peak": peak_ops,
                "unit": "Gop/s", "frac": ops / (dist_ms * 1e-3) / 1e9 / peak_ops,
                "traffic": None,
                "kernel": "dist_kernel, one plane per work unit (4:4:4 planes in the packed "
                          "layout) + find_dir_kernel (distortion tables)"
                if variant == "444"
                else "dist_kernel<1, coded>, one plane per work unit (4:4:4 planes in the "
                     "packed layout) + find_dir_kernel (128-combination tables)"
                if variant == "444coded"
                else "dist_wide_kernel + find_dir_kernel (distortion tables, 32-bit lanes)"
                if variant == "12bit"
                else "dist_kernel<8, eq. 14>, one plane per work unit (4:4:4 planes in the "
                     "packed layout) + find_dir_kernel (eq. 14 tables)"
                if variant == "444eq14"
                else "dist_wide_eq14_kernel + find_dir_kernel (eq. 14 tables, 32-bit lanes)"
                if variant == "12biteq14" else "dist_kernel (distortion tables)",
                "ops_per_launch": ops, "mean_launch_us": dist_ms * 1e3,
                "launch_time": "CUDA events around the kernel inside the search graph",
                "preset_kernel_us": pre_ms * 1e3,
                "peak_source": "derived: 152 SMs x 128 lanes x 2 (16-bit pairs) x 2070 MHz"
                if bd <= 10 else "derived: 152 SMs x 128 lanes x 2070 MHz"}
    if bd <= 10:   # the measured ceiling of the tap instruction mix (as for the filter)
        peak_mix = 2 * cdef.probe_int_mix(ctx, 0) / 1e9
        roofline["measured_int_ceiling"] = {
            "peak": peak_mix, "unit": "Gop/s", "frac": roofline["achieved"] / peak_mix,
            "what": "cdef_probe_int_mix: the filter tap's 6 ALU operations and 2 "
                    "multiply-adds in independent chains"}
    cpu = None
    if pool is not None:
        sample = [i for i in range(len(frames)) if (frames[i].width, frames[i].height) == (640, 360)]
        tasks = [(frames[i].width, frames[i].height, SEARCH_WORKLOAD["base_seed"] + i, damping[i],
                  lambdas[i], variant, args.refine,
                  maps[i].cpu().numpy().reshape(frames[i].height // 8, frames[i].width // 8)
                  if maps else None) for i in sample]
        t0 = time.perf_counter()
        res = pool.map(_oracle_search, tasks, chunksize=1)
        wall = time.perf_counter() - t0
        pool.close()
        cand = sum(r[0] for r in res)
        cpu = {"value": cand / wall, "unit": "candidates/s", "cores": min(len(tasks), pool._processes),
               "kind": "oracle",
               "sample": f"the {len(tasks)} 640x360 frames of the workload, one process per frame: "
                         f"{cand} candidates, {sum(r[1] for r in res):.1f} s of CPU work in "
                         f"{wall:.1f} s wall"}
    ctx.close()
    return {
        "metric": "strength-search candidates/s", "value": nb * 2 * width / sec,
        "unit": "candidates/s",
        "n_gpus": 1, "steps": steps, "warmup": warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": {"workload": SEARCH_WORKLOAD["name"], "blocks": nb,
                                        "inputs_sha256": synth.digest_of(frames),
                                        "luma_pixels": sum(f.width * f.height for f in frames),
                                        "l2": "L2 flushed (256 MB write) before each call"},
        "tuning": dict(zip(("search_groups", "search_ctas_per_sm"), tune)),
        "roofline": roofline, "cpu_baseline": cpu,
        "refine_passes": args.refine, "variant": variant,
        "plain": {"ms_per_step": plain_sec * 1e3, "value": nb * 2 * width / plain_sec,
                  "what": "one cdef_search_strengths call per frame, identical outputs",
                  "spread_ms": spread_ms(plain_s)},
        "spread_ms": spread_ms(call_s),
        "clocks": clk}


def spread_ms(secs) -> dict:
    """Minimum, median and maximum of the timed calls (ms) and their count."""
    v = sorted(x * 1e3 for x in secs)
    return {"min": v[0], "median": statistics.median(v), "max": v[-1], "calls": len(v)}


def search_extra(args):
    """The strength-search workload (16 mixed frames, 64 + 64 pairs) for the
    default line: candidates/s of the batched call, its stages, and the
    one-call-per-frame path on the same frames."""
    r = measure_search(args, "sse", 5, 3)
    rl = r["roofline"]
    return {"metric": r["metric"], "value": r["value"], "unit": r["unit"],
            "workload": r["config"]["workload"], "ms_per_call": r["ms_per_step"],
            "distortion_kernel_us": rl["mean_launch_us"], "preset_kernel_us": rl["preset_kernel_us"],
            "plain_ms_per_call": r["plain"]["ms_per_step"],
            "batched_over_plain": r["plain"]["ms_per_step"] / r["ms_per_step"],
            "spread_ms": r["spread_ms"], "plain_spread_ms": r["plain"]["spread_ms"],
            "roofline": {k: rl[k] for k in ("bound", "achieved", "peak", "unit", "frac", "kernel",
                                            "peak_source", "measured_int_ceiling") if k in rl},
            "tuning": r["tuning"], "l2": r["config"]["l2"], "calls": 5, "clocks": r["clocks"]}


def serve_extra(args):
    """The serving workload for the default line: Poisson arrivals at the
    one-frame-at-a-time capacity (2000 requests), batched against one frame
    at a time, plus both capacities."""
    r = measure_serve(args, 2000, (1.0,), 100, 1000)
    cfg = r["config"]
    at = cfg["rates"]["1.0"]
    keys = ("frames_per_s", "p50_ms", "p99_ms", "mean_ms", "mean_batch")
    return {"metric": "served frames/s and latency at the one-frame-at-a-time capacity",
            "workload": cfg["workload"], "requests": 2000,
            "batched": {k: at["batched"][k] for k in keys},
            "one_at_a_time": {k: at["one_at_a_time"][k] for k in keys},
            "saturation_fps": {"batched": cfg["batched_capacity"]["frames_per_s"],
                               "one_at_a_time": cfg["one_at_a_time_capacity"]["frames_per_s"]},
            "verified": cfg["verified"], "clocks": r["clocks"]}


SERVE_WORKLOAD = dict(
    name="serving loop: Poisson arrivals, resolutions uniform over 640x360 / 1280x720 / "
         "1920x1080 / 3840x2160, 8/10-bit 50/50, random per-block strengths, HBM budget "
         "8 GiB; continuous batching against one frame at a time",
    sizes=[(640, 360), (1280, 720), (1920, 1080), (3840, 2160)], bitdepths=(8, 10),
    requests=10000, rates=(0.5, 0.8, 1.0, 1.5), budget=8 << 30, contents=2, seed=0,
    base_seed=4000, verify_requests=400, batch_bytes=256 << 20, inflight=3)


def run_serve(args):
    """The serving loop at Poisson arrival rates of 0.5-1.5x the measured
    one-frame-at-a-time capacity; both servers see the same arrivals."""
    W = SERVE_WORKLOAD
    print(json.dumps(measure_serve(args, args.requests or W["requests"], W["rates"],
                                   W["verify_requests"], min(args.requests or W["requests"], 2000))))


def host_settings() -> dict:
    """Kernel settings of the host that bear on serving-loop stalls (read
    only): automatic NUMA balancing and transparent huge pages."""
    out = {}
    for key, path in (("numa_balancing", "/proc/sys/kernel/numa_balancing"),
                      ("transparent_hugepage", "/sys/kernel/mm/transparent_hugepage/enabled"),
                      ("cpus", None)):
        try:
            out[key] = os.cpu_count() if path is None else open(path).read().strip()
        except OSError:
            out[key] = None
    return out


def measure_serve(args, n, rate_fracs, nv, ncap):
    """The serving measurement (see run_serve) with n requests per arrival
    rate, nv verified requests and ncap requests for the capacities;
    returns the bench line as a dict."""
    import torch
    from paper_1602_05975_gb300 import build, cdef, serve, synth
    build.build()
    ctx = cdef.Context(0)
    W = SERVE_WORKLOAD
    rng = np.random.default_rng(W["seed"])
    contents = {}
    for si, (w, h) in enumerate(W["sizes"]):
        for bd in W["bitdepths"]:
            contents[(w, h, bd)] = [
                serve.pack_frame(cdef, synth.make_frame(w, h, bd, None,
                                                        W["base_seed"] + 100 * si + 10 * bd + k).rec,
                                 bd) for k in range(W["contents"])]
    specs = []
    for i in range(max(n, nv, ncap)):
        w, h = W["sizes"][rng.integers(len(W["sizes"]))]
        bd = W["bitdepths"][rng.integers(len(W["bitdepths"]))]
        specs.append((w, h, bd, int(rng.integers(W["contents"])), synth.random_params(rng, w, h)))
    arena = torch.empty(sum(p.size for *_, p in specs), dtype=torch.uint8).pin_memory()
    views, o = [], 0
    for *_, prm in specs:
        v = arena[o:o + prm.size]
        v.copy_(torch.from_numpy(prm.reshape(-1)))
        views.append(v)
        o += prm.size

    def requests(arrivals, count):
        return [serve.Request(i, w, h, bd, contents[(w, h, bd)][k], prm, float(arrivals[i]),
                              params_host=views[i])
                for i, (w, h, bd, k, prm) in enumerate(specs[:count])]

    budget = W["budget"]
    timing = bool(getattr(args, "serve_timing", False))
    batched_be = serve.CudaBackend(ctx, budget, timing=timing)
    single_be = serve.CudaBackend(ctx, budget, timing=timing)
    shapes = [(w, h, bd) for (w, h) in W["sizes"] for bd in W["bitdepths"]]
    # buffers for every burst the budget admits: no allocation while serving
    batched_be.prewarm(shapes, 24, fill=0.9)
    single_be.prewarm(shapes, 2)

    def batched(on_done=None):
        return serve.Server(batched_be, budget, max_batch=cdef.MAX_BATCH,
                            max_inflight=args.inflight or W["inflight"], on_done=on_done,
                            max_batch_bytes=(args.batch_mib << 20) if args.batch_mib
                            else W["batch_bytes"])

    def one_at_a_time(on_done=None):
        return serve.Server(single_be, budget, max_batch=1, max_inflight=1, on_done=on_done)

    # 1. verification (untimed): every output of a mixed run equals the same
    #    frame filtered alone through the single-frame entry point
    served = {}

    def keep(r):
        if r.status == "ok":
            served[r.rid] = serve.unpack_frame(r.out)

    vreq = requests(np.zeros(nv), nv)
    batched(on_done=keep).run(vreq, timeout=600)
    mismatches = 0
    for r in vreq:
        w, h, bd, k, prm = specs[r.rid]
        flat_in, fin, _ = cdef.alloc_packed(w, h, bd, device="cuda")
        flat_in.copy_(contents[(w, h, bd)][k])
        _, fout, _ = cdef.alloc_packed(w, h, bd, device="cuda")
        cdef.cdef_filter_frame(ctx, fin, views[r.rid].to("cuda"), fout)
        exp = fout.to_numpy()
        if r.status != "ok" or not all(np.array_equal(a, b) for a, b in zip(served[r.rid], exp)):
            mismatches += 1
    assert mismatches == 0, f"{mismatches} served results differ from the single-frame path"

    keys = ("frames_per_s", "mpixel_per_s", "p50_ms", "p99_ms", "mean_ms", "batches",
            "mean_batch", "peak_device_bytes", "wall_s", "ok", "p99_tail", "buffer_allocs",
            "host_calls") + (("device_stages",) if timing else ())
    # 2. capacities: all requests present at t = 0 (after a warm-up run)
    one_at_a_time().run(requests(np.zeros(400), 400), timeout=600)
    cap = one_at_a_time().run(requests(np.zeros(ncap), ncap), timeout=600)
    capacity = cap["frames_per_s"]
    bcap = batched().run(requests(np.zeros(ncap), ncap), timeout=600)

    # 3. Poisson arrivals at fractions of the one-at-a-time capacity
    clocks = ClockSampler(0)
    clocks.disabled = args.no_clocks
    clocks.start()
    rates = {}
    for k, frac in enumerate(rate_fracs):
        arr = serve.poisson_arrivals(n, frac * capacity, seed=W["seed"] + 1 + k)
        if frac == 1.0:
            clocks.mark("begin")
        b = batched().run(requests(arr, n), timeout=900)
        if frac == 1.0:
            clocks.mark("end")
        o = one_at_a_time().run(requests(arr, n), timeout=900)
        rates[str(frac)] = {"batched": {q: b[q] for q in keys},
                            "one_at_a_time": {q: o[q] for q in keys}}
        assert b["ok"] == n and o["ok"] == n
    clk = clocks.stop()
    head = rates["1.0"]["batched"]
    ctx.close()
    return {
        "metric": "served frames/s at saturation (continuous batching)",
        "value": bcap["frames_per_s"], "unit": "frames/s", "n_gpus": 1, "steps": 1,
        "warmup": 1, "ms_per_step": bcap["wall_s"] * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"],
        "latency_at": "Poisson arrivals at the one-frame-at-a-time capacity",
        "config": {"workload": W["name"], "requests": n, "saturation_requests": ncap,
                   "batched_capacity": {q: bcap[q] for q in keys},
                   "one_at_a_time_capacity": {q: cap[q] for q in keys},
                   "one_at_a_time_capacity_fps": capacity, "budget_bytes": budget,
                   "batch_bytes": (args.batch_mib << 20) if args.batch_mib else W["batch_bytes"],
                   "inflight": args.inflight or W["inflight"],
                   "verified": f"{nv} requests served in mixed batches equal the "
                               f"single-frame path bit for bit",
                   "host_settings": host_settings(),
                   "rates": rates},
        "clocks": clk}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="filter only: leave out the search and serving figures")
    ap.add_argument("--no-overlap", action="store_true",
                    help="filter: keep stream order between frames (no overlapped launches)")
    ap.add_argument("--cpu-bands", type=int, default=0,
                    help="oracle sample: number of 120-row bands (0 = the whole step)")
    ap.add_argument("--check", action="store_true", help="oracle check of frame 0")
    ap.add_argument("--workload", default="filter",
                    choices=["filter", "filter1080p", "filter444", "filter12", "search", "serve"],
                    help="filter: the 4K 10-bit filter (default line); filter1080p: 30 "
                         "1080p 8-bit frames; filter444: 30 1080p 8-bit 4:4:4 frames; "
                         "filter12: 8 4K 12-bit frames; search: batched strength search over "
                         "16 mixed frames; serve: the serving loop")
    ap.add_argument("--requests", type=int, default=0, help="serve: requests per rate")
    ap.add_argument("--batch-mib", type=int, default=0,
                    help="serve: byte cap of one batch in MiB (0: the workload's)")
    ap.add_argument("--inflight", type=int, default=0,
                    help="serve: batches on the device at once (0: the workload's)")
    ap.add_argument("--serve-timing", action="store_true",
                    help="serve: time every batch's copy, kernel and read-back stages "
                         "with CUDA events and report them")
    ap.add_argument("--refine", type=int, default=0,
                    help="search: preset re-optimisation passes after the greedy search")
    ap.add_argument("--search-variant", default="sse",
                    choices=["sse", "eq14", "coded", "444", "12bit", "444coded", "444eq14",
                             "12biteq14"],
                    help="search: squared error (64 pairs), eq. 14 distortion, the "
                         "128-combination search with coded-residual maps, or the squared-error "
                         "search over 8-bit 4:4:4 or 12-bit 4:2:0 frames")
    ap.add_argument("--no-clocks", action="store_true",
                    help="do not sample nvidia-smi clocks during the run")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.workload == "search" and args.impl == "ours":
        run_search(args)
        return
    if args.workload == "serve" and args.impl == "ours":
        run_serve(args)
        return
    global WORKLOAD
    if args.workload in FILTER_WORKLOADS:
        WORKLOAD = FILTER_WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
