"""Host logic of the serving loop (admission, continuous batching, faults),
driven by a fake backend: no GPU, no CUDA library."""
import numpy as np
import pytest

from paper_1602_05975_gb300 import serve


class FakeBackend(serve.Backend):
    """Batches finish after `latency` polls; launches listed in `fail_launch`
    raise, batches listed in `fail_batch` finish with an error."""

    def __init__(self, latency=2, fail_launch=(), fail_batch=()):
        self.latency = latency
        self.fail_launch = set(fail_launch)
        self.fail_batch = set(fail_batch)
        self.launches = []
        self.held = 0
        self.peak_held = 0
        self.n_launch = 0

    def need_bytes(self, req):
        return req.width * req.height * 3

    def reserve(self, req):
        req.slot = object()
        self.held += req.need
        self.peak_held = max(self.peak_held, self.held)

    def release(self, req):
        self.held -= req.need

    def launch(self, reqs):
        k = self.n_launch
        self.n_launch += 1
        if k in self.fail_launch:
            raise RuntimeError("injected launch error")
        self.launches.append([r.rid for r in reqs])
        return {"k": k, "left": self.latency, "n": len(reqs)}

    def poll(self, h):
        h["left"] -= 1
        if h["left"] > 0:
            return None
        return ["injected device error"] * h["n"] if h["k"] in self.fail_batch else ["ok"] * h["n"]


def params_for(w, h, pri=3, sec=1, damping=4):
    p = np.zeros((-(-h // 64), -(-w // 64), 8), np.uint8)
    p[..., 0], p[..., 1], p[..., 2], p[..., 3], p[..., 4] = pri, sec, pri, sec, damping
    return p


def req(rid, w=64, h=64, bd=8, arrival=0.0, **kw):
    return serve.Request(rid, w, h, bd, None, params_for(w, h, **kw), arrival)


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


def drain(s, clock, limit=10000):
    n = 0
    while not s.idle():
        clock.t += 1e-3
        s.step()
        n += 1
        assert n < limit
    return n


def test_all_requests_complete_in_order_of_admission():
    fb, clk = FakeBackend(), Clock()
    s = serve.Server(fb, budget_bytes=1 << 30, clock=clk)
    rs = [req(i) for i in range(50)]
    for r in rs:
        assert s.submit(r)
    drain(s, clk)
    assert all(r.status == "ok" for r in rs)
    assert [rid for b in fb.launches for rid in b] == list(range(50))
    assert s.in_use == 0 and fb.held == 0
    assert all(r.latency >= 0 for r in rs)


def test_budget_bounds_device_memory():
    fb, clk = FakeBackend(latency=3), Clock()
    budget = 3 * 64 * 64 * 3
    s = serve.Server(fb, budget_bytes=budget, clock=clk)
    rs = [req(i) for i in range(20)]
    for r in rs:
        s.submit(r)
    drain(s, clk)
    assert all(r.status == "ok" for r in rs)
    assert s.peak_in_use <= budget and fb.peak_held <= budget
    assert max(len(b) for b in fb.launches) <= 3


def test_requests_arriving_during_a_batch_join_the_next_one():
    fb, clk = FakeBackend(latency=10), Clock()
    s = serve.Server(fb, budget_bytes=1 << 30, max_inflight=1, clock=clk)
    s.submit(req(0))
    s.step()
    assert fb.launches == [[0]]
    for i in range(1, 6):
        s.submit(req(i))
        s.step()                      # the device is busy: they wait together
    assert len(fb.launches) == 1
    drain(s, clk)
    assert fb.launches == [[0], [1, 2, 3, 4, 5]]


def test_two_batches_in_flight_overlap():
    fb, clk = FakeBackend(latency=5), Clock()
    s = serve.Server(fb, budget_bytes=1 << 30, max_inflight=2, clock=clk)
    s.submit(req(0))
    s.step()
    s.submit(req(1))
    s.step()
    assert fb.launches == [[0], [1]] and len(s.inflight) == 2
    drain(s, clk)


def test_one_at_a_time_mode():
    fb, clk = FakeBackend(), Clock()
    s = serve.Server(fb, budget_bytes=1 << 30, max_batch=1, max_inflight=1, clock=clk)
    for i in range(7):
        s.submit(req(i))
    drain(s, clk)
    assert fb.launches == [[i] for i in range(7)]


def test_max_batch_splits_large_queues():
    fb, clk = FakeBackend(), Clock()
    s = serve.Server(fb, budget_bytes=1 << 30, max_batch=4, max_inflight=2, clock=clk)
    for i in range(10):
        s.submit(req(i))
    drain(s, clk)
    assert all(len(b) <= 4 for b in fb.launches)
    assert sorted(r for b in fb.launches for r in b) == list(range(10))


@pytest.mark.parametrize("bad", [dict(pri=16), dict(sec=3), dict(damping=2), dict(damping=7)])
def test_bad_parameters_rejected_without_touching_others(bad):
    fb, clk = FakeBackend(), Clock()
    s = serve.Server(fb, budget_bytes=1 << 30, clock=clk)
    good = [req(i) for i in range(3)]
    b = req(99, **bad)
    s.submit(good[0])
    assert not s.submit(b)
    s.submit(good[1])
    s.submit(good[2])
    drain(s, clk)
    assert b.status == "rejected" and "range" in b.error
    assert all(r.status == "ok" for r in good)
    assert all(99 not in l for l in fb.launches)


def test_skip_mapping_strengths_accepted():
    fb, clk = FakeBackend(), Clock()
    s = serve.Server(fb, budget_bytes=1 << 30, clock=clk)
    assert s.submit(req(0, pri=19, sec=7))
    drain(s, clk)


def test_wrong_shapes_rejected():
    fb, clk = FakeBackend(), Clock()
    s = serve.Server(fb, budget_bytes=1 << 30, clock=clk)
    r = serve.Request(0, 64, 64, 8, None, params_for(128, 64), 0.0)
    assert not s.submit(r) and "shape" in r.error
    r = serve.Request(1, 60, 64, 8, None, params_for(60, 64), 0.0)
    assert not s.submit(r) and "multiple of 8" in r.error
    r = serve.Request(2, 64, 64, 9, None, params_for(64, 64), 0.0)
    assert not s.submit(r) and "bit depth" in r.error


def test_request_larger_than_budget_rejected():
    fb, clk = FakeBackend(), Clock()
    s = serve.Server(fb, budget_bytes=64 * 64 * 3, clock=clk)
    big = req(0, w=128, h=128)
    assert not s.submit(big)
    assert big.status == "rejected" and "budget" in big.error
    small = req(1)
    assert s.submit(small)
    drain(s, clk)
    assert small.status == "ok"


def test_cancel_before_launch_only():
    fb, clk = FakeBackend(latency=4), Clock()
    s = serve.Server(fb, budget_bytes=64 * 64 * 3, max_inflight=1, clock=clk)
    a, b, c = req(0), req(1), req(2)
    for r in (a, b, c):
        s.submit(r)
    s.step()                                     # a admitted and launched
    assert a.status == "launched"
    assert not s.cancel(0)                       # already on the device
    assert s.cancel(2)                           # still queued
    drain(s, clk)
    assert (a.status, b.status, c.status) == ("ok", "ok", "cancelled")
    assert [l for l in fb.launches] == [[0], [1]]
    assert s.in_use == 0 and fb.held == 0


def test_cancel_admitted_frees_budget():
    fb, clk = FakeBackend(latency=4), Clock()
    s = serve.Server(fb, budget_bytes=1 << 30, max_inflight=1, clock=clk)
    a, b = req(0), req(1)
    s.submit(a)
    s.step()
    s.submit(b)
    s.step()                                     # b admitted, waiting for the device
    assert b.status == "admitted" and s.in_use == 2 * a.need
    assert s.cancel(1)
    assert s.in_use == a.need and fb.held == a.need
    drain(s, clk)
    assert b.status == "cancelled" and a.status == "ok"


def test_launch_error_fails_that_batch_only():
    fb, clk = FakeBackend(fail_launch={1}), Clock()
    s = serve.Server(fb, budget_bytes=1 << 30, max_inflight=1, clock=clk)
    s.submit(req(0))
    s.step()
    s.submit(req(1))
    s.submit(req(2))
    drain(s, clk)
    s.submit(req(3))
    drain(s, clk)
    st = {r.rid: r.status for r in s.finished}
    assert st == {0: "ok", 1: "failed", 2: "failed", 3: "ok"}
    assert "injected launch error" in [r for r in s.finished if r.rid == 1][0].error
    assert s.in_use == 0 and fb.held == 0


def test_device_error_fails_that_batch_only():
    fb, clk = FakeBackend(fail_batch={0}), Clock()
    s = serve.Server(fb, budget_bytes=1 << 30, max_inflight=1, clock=clk)
    s.submit(req(0))
    s.step()
    s.submit(req(1))
    drain(s, clk)
    st = {r.rid: (r.status, r.error) for r in s.finished}
    assert st[0] == ("failed", "injected device error") and st[1] == ("ok", "")


def test_realtime_run_with_poisson_arrivals():
    fb = FakeBackend(latency=3)
    s = serve.Server(fb, budget_bytes=1 << 30)
    t = serve.poisson_arrivals(300, rate=20000.0, seed=0)
    rs = [req(i, arrival=float(t[i])) for i in range(300)]
    st = s.run(rs, timeout=60)
    assert st["ok"] == 300 and st["requests"] == 300
    assert st["p50_ms"] <= st["p99_ms"]
    assert all(r.t_done >= r.arrival and r.t_launch >= r.t_admit >= r.t_submit for r in rs)
    assert st["batches"] <= 300


def test_poisson_arrivals_rate():
    t = serve.poisson_arrivals(20000, rate=1000.0, seed=1)
    assert np.all(np.diff(t) > 0)
    assert abs(20000 / t[-1] - 1000.0) < 30.0


def test_admission_window_is_one_batch():
    fb, clk = FakeBackend(latency=50), Clock()
    s = serve.Server(fb, budget_bytes=1 << 40, max_batch=4, max_inflight=1, clock=clk)
    for i in range(20):
        s.submit(req(i))
    s.step()
    s.step()
    # one batch on the device, at most one more admitted, the rest queued
    assert len(s.inflight) == 1 and len(s.ready) == 4 and len(s.queue) == 12
    assert s.in_use == 8 * req(0).width * req(0).height * 3
    drain(s, clk)
    assert len(s.finished) == 20


def test_batches_cut_by_bytes():
    fb, clk = FakeBackend(), Clock()
    one = 64 * 64 * 3
    s = serve.Server(fb, budget_bytes=1 << 40, max_batch=48, max_inflight=1, clock=clk,
                     max_batch_bytes=3 * one)
    for i in range(10):
        s.submit(req(i))
    drain(s, clk)
    assert [len(b) for b in fb.launches] == [3, 3, 3, 1]
    big = serve.Server(fb, budget_bytes=1 << 40, max_batch_bytes=one // 2, clock=clk)
    big.submit(req(99))                 # larger than the cap: still launched alone
    drain(big, clk)
    assert fb.launches[-1] == [99]
