"""Bounded device-side waits that run out.

Every tile-load wait of the filter and distortion kernels has an iteration
limit.  cdef_debug_set_waits shortens the limit and adds to every load's
expected transaction count bytes that no copy delivers, so each wait gives
up: no fault, no trap, no endless loop.  The kernel then sets the timeout
status, takes the undelivered bytes back, waits (bounded) for the loads it
did issue and leaves.  These tests check that the call reports
CDEF_ERR_TIMEOUT and that the next normal call on the same context is
bit-exact against the oracle (the work counters were reset)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHORT = 1 << 16      # SM cycles (~32 us at 2 GHz)
UNDELIVERED = 16     # bytes no copy delivers


@pytest.fixture(scope="module")
def cdef():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1602_05975_gb300 import build, cdef as _c
    build.build()
    _c.load()
    yield _c
    _c.debug_set_waits(0, 0)


def test_debug_waits_rejects_out_of_range(cdef):
    with pytest.raises(cdef.CdefError):
        cdef.debug_set_waits(-1, 0)
    with pytest.raises(cdef.CdefError):
        cdef.debug_set_waits(0, (1 << 16) + 1)


@pytest.mark.parametrize("bd", [8, 10, 12])
def test_filter_wait_runs_out_then_recovers(cdef, ref, bd):
    from paper_1602_05975_gb300 import synth
    ctx = cdef.Context(0)
    f = synth.make_frame(200, 136, bd, 32, seed=7000 + bd)
    inp = cdef.frame_from_numpy(f.rec, bd)
    prm = cdef.params_tensor(f.params)
    out = cdef.alloc_frame(200, 136, bd, fill=0)
    cdef.debug_set_waits(SHORT, UNDELIVERED)
    try:
        cdef.cdef_filter_frame(ctx, inp, prm, out)
        torch.cuda.synchronize()
    finally:
        cdef.debug_set_waits(0, 0)
    assert ctx.status(clear=True) == -6          # CDEF_ERR_TIMEOUT
    assert ctx.status() == 0                     # cleared
    # every CTA left before filtering: the output was never written
    assert all(int(p.abs().sum()) == 0 for p in out.planes())
    # the same context, limits restored: bit-exact, repeatedly
    exp = ref.filter_frame(*f.rec, bd, f.params)
    for _ in range(2):
        out2 = cdef.alloc_frame(200, 136, bd, fill=0)
        cdef.cdef_filter_frame(ctx, inp, prm, out2)
        torch.cuda.synchronize()
        assert ctx.status() == 0
        for g, e in zip(out2.to_numpy(), exp):
            assert np.array_equal(g, e)
    ctx.close()


def test_filter_batch_wait_runs_out_then_recovers(cdef, ref):
    from paper_1602_05975_gb300 import synth
    ctx = cdef.Context(0)
    frames = [synth.make_frame(w, h, bd, 32, seed=7010 + k)
              for k, (w, h, bd) in enumerate(((136, 72, 8), (64, 64, 10), (200, 136, 8)))]
    ins = [cdef.frame_from_numpy(f.rec, f.bitdepth) for f in frames]
    prms = [cdef.params_tensor(f.params) for f in frames]
    outs = [cdef.alloc_frame(f.width, f.height, f.bitdepth, fill=0) for f in frames]
    cdef.debug_set_waits(SHORT, UNDELIVERED)
    try:
        cdef.cdef_filter_frames(ctx, ins, prms, outs)
        torch.cuda.synchronize()
    finally:
        cdef.debug_set_waits(0, 0)
    assert ctx.status(clear=True) == -6
    cdef.cdef_filter_frames(ctx, ins, prms, outs)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    for f, o in zip(frames, outs):
        for g, e in zip(o.to_numpy(), ref.filter_frame(*f.rec, f.bitdepth, f.params)):
            assert np.array_equal(g, e)
    ctx.close()


@pytest.mark.parametrize("grid", [0, 1])
def test_search_wait_runs_out_then_recovers(cdef, ref, grid):
    """The distortion kernel's waits give up (both of a CTA's tile buffers
    are drained); the search graph recorded with the short limits is
    replaced by one with the default limits on the next call."""
    from paper_1602_05975_gb300 import synth
    ctx = cdef.Context(0)
    ctx.set_tuning(1, 2, preset_kernel=grid)
    frames = [synth.make_frame(w, h, 8, 32, seed=7020 + k)
              for k, (w, h) in enumerate(((200, 136), (136, 72)))]
    recs = [cdef.frame_from_numpy(f.rec, 8) for f in frames]
    srcs = [cdef.frame_from_numpy(f.src, 8) for f in frames]
    nb = sum(f.params.shape[0] * f.params.shape[1] for f in frames)
    ids = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    dl = torch.zeros(nb * 64, dtype=torch.int64, device="cuda")
    dc = torch.zeros(nb * 64, dtype=torch.int64, device="cuda")
    args = (recs, srcs, [5, 4], [900, 256], ids, dl, dc)
    cdef.debug_set_waits(SHORT, UNDELIVERED)
    try:
        cdef.cdef_search_strengths(ctx, *args)
    finally:
        cdef.debug_set_waits(0, 0)
    assert ctx.status(clear=True) == -6
    res = cdef.cdef_search_strengths(ctx, *args)
    assert ctx.status() == 0
    o0 = 0
    for f, r, d, lam in zip(frames, res, [5, 4], [900, 256]):
        b = f.params.shape[0] * f.params.shape[1]
        o = ref.search_strengths(f.rec, f.src, 8, d, lam)
        assert np.array_equal(dl[o0 * 64:(o0 + b) * 64].cpu().numpy().reshape(b, 64), o["dist_luma"])
        assert np.array_equal(dc[o0 * 64:(o0 + b) * 64].cpu().numpy().reshape(b, 64), o["dist_chroma"])
        assert r["npresets"] == o["npresets"] and r["cost"] == o["cost"]
        assert np.array_equal(ids[o0:o0 + b].cpu().numpy(), o["block_ids"])
        o0 += b
    ctx.close()
