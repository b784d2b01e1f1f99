"""Serving loop on the GPU: every request's result is the same whether it is
filtered alone or inside a mixed continuous batch, and equals the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cdef():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1602_05975_gb300 import build, cdef as _c
    build.build()
    _c.load()
    return _c


@pytest.fixture(scope="module")
def ctx(cdef):
    c = cdef.Context(0)
    yield c
    c.close()


SIZES = [(64, 64, 8), (128, 72, 10), (352, 288, 8), (200, 136, 10), (96, 40, 8),
         (320, 184, 10), (72, 264, 8), (256, 128, 10)]


@pytest.fixture(scope="module")
def setup(cdef, ctx):
    from paper_1602_05975_gb300 import serve, synth
    rng = np.random.default_rng(7)
    reqs, frames = [], []
    for i in range(24):
        w, h, bd = SIZES[i % len(SIZES)]
        fr = synth.make_frame(w, h, bd, None, 500 + i)
        params = synth.random_params(rng, w, h)
        frames.append((fr, params))
        reqs.append(serve.Request(i, w, h, bd, serve.pack_frame(cdef, fr.rec, bd), params,
                                  arrival=0.0 if i < 12 else 0.002 * (i - 11)))
    return torch, serve, reqs, frames


def alone(cdef, ctx, torch, fr, params):
    src = cdef.frame_from_numpy(fr.rec, fr.bitdepth)
    out = cdef.alloc_frame(fr.width, fr.height, fr.bitdepth, fill=0)
    cdef.cdef_filter_frame(ctx, src, cdef.params_tensor(params), out)
    torch.cuda.synchronize()
    return out.to_numpy()


@pytest.mark.parametrize("budget_frames", [100, 3])
def test_mix_equals_alone_and_oracle(cdef, ctx, ref, setup, budget_frames):
    torch, serve, reqs, frames = setup
    for r in reqs:
        r.status, r.slot, r.out = "new", None, None
    results = {}

    def on_done(r):
        if r.status == "ok":
            results[r.rid] = serve.unpack_frame(r.out)

    largest = max(serve.CudaBackend(ctx, 1 << 40).need_bytes(r) for r in reqs)
    budget = budget_frames * largest
    be = serve.CudaBackend(ctx, budget)
    srv = serve.Server(be, budget, max_batch=48, max_inflight=2, on_done=on_done)
    st = srv.run(reqs, timeout=120)
    assert st["ok"] == len(reqs), st
    assert srv.peak_in_use <= budget and be.held_bytes <= budget
    if budget_frames == 100:
        assert st["mean_batch"] > 1.0       # requests really shared launches
    for r, (fr, params) in zip(reqs, frames):
        a = alone(cdef, ctx, torch, fr, params)
        o = ref.filter_frame(*fr.rec, fr.bitdepth, params)
        for got, al, ex in zip(results[r.rid], a, o):
            assert np.array_equal(got, al), f"request {r.rid}: batched != alone"
            assert np.array_equal(got, ex), f"request {r.rid}: != oracle"
    assert ctx.status() == 0


def test_one_at_a_time_server_matches(cdef, ctx, ref, setup):
    torch, serve, reqs, frames = setup
    sub = [serve.Request(r.rid, r.width, r.height, r.bitdepth, r.frame, r.params, 0.0)
           for r in reqs[:8]]
    results = {}
    be = serve.CudaBackend(ctx, 1 << 30)
    srv = serve.Server(be, 1 << 30, max_batch=1, max_inflight=1,
                       on_done=lambda r: results.__setitem__(r.rid, serve.unpack_frame(r.out)))
    st = srv.run(sub, timeout=60)
    assert st["ok"] == 8 and st["mean_batch"] == 1.0
    for r in sub:
        fr, params = frames[r.rid]
        for got, ex in zip(results[r.rid], ref.filter_frame(*fr.rec, fr.bitdepth, params)):
            assert np.array_equal(got, ex)
