"""The allocation-free strength search (cdef_search_strengths_noalloc).

Callers that may not allocate device memory after start-up (a codec given a
fixed memory budget by its host application, a real-time loop that cannot
take the synchronisation cudaMalloc/cudaFree may cause) use this entry
point: no context, scratch in a fixed array inside the library.  These tests
call it through the C ABI: twice in a row on different frames against both
cdef_search_strengths and the oracle (the search is integer arithmetic, so
the tolerance is zero, as in the other parity tests), near the array's
capacity, with a bounded wait that runs out, and with frames it refuses.
The device's free memory must not change across a call.  The file name
makes pytest collect it last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MAX_BLOCKS = 16384   # CDEF_NOALLOC_MAX_BLOCKS


@pytest.fixture(scope="module")
def cdef():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1602_05975_gb300 import build, cdef as _c
    build.build()
    _c.load()
    torch.cuda.set_device(0)
    # The first call on a device loads the library's fixed array (held
    # until the process exits); the free-memory checks start after it.
    f = _c.alloc_frame(8, 8, 8, fill=0)
    ids, dl, dc = _outputs(1)
    _c.cdef_search_strengths_noalloc([f], [f], [4], [0], ids, dl, dc)
    torch.cuda.synchronize()
    return _c


def _outputs(tot, fill_ids=0, fill_tab=0):
    return (torch.full((tot,), fill_ids, dtype=torch.uint8, device="cuda"),
            torch.full((tot * 64,), fill_tab, dtype=torch.int64, device="cuda"),
            torch.full((tot * 64,), fill_tab, dtype=torch.int64, device="cuda"))


def _noalloc(cdef, recs, srcs, damping, lambdas, tot):
    """One call with garbage-filled outputs; the device's free memory is
    the same before and after it."""
    ids, dl, dc = _outputs(tot, 77, -5)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    res = cdef.cdef_search_strengths_noalloc(recs, srcs, damping, lambdas, ids, dl, dc)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    return res, ids, dl, dc


def _run_both(cdef, ref, specs, seed, oracle=True):
    from paper_1602_05975_gb300 import synth
    frames = [synth.make_frame(w, h, bd, None, seed=seed + k) for k, (w, h, bd) in enumerate(specs)]
    recs = [cdef.frame_from_numpy(f.rec, f.bitdepth) for f in frames]
    srcs = [cdef.frame_from_numpy(f.src, f.bitdepth) for f in frames]
    tot = sum(f.params.shape[0] * f.params.shape[1] for f in frames)
    damping = [3 + (k % 4) for k in range(len(frames))]
    lambdas = [int(f.q) ** 2 << (2 * (f.bitdepth - 8)) for f in frames]

    # existing entry point (context scratch)
    ctx = cdef.Context(0)
    ids_a, dl_a, dc_a = _outputs(tot)
    res_a = cdef.cdef_search_strengths(ctx, recs, srcs, damping, lambdas, ids_a, dl_a, dc_a)
    ctx.close()

    res_b, ids_b, dl_b, dc_b = _noalloc(cdef, recs, srcs, damping, lambdas, tot)
    assert torch.equal(dl_a, dl_b) and torch.equal(dc_a, dc_b)
    assert torch.equal(ids_a, ids_b)
    for a, b in zip(res_a, res_b):
        assert a["npresets"] == b["npresets"] and a["cost"] == b["cost"]
        assert a["presets"] == b["presets"]
    if oracle:
        o0 = 0
        for f, r, d, lam in zip(frames, res_b, damping, lambdas):
            b = f.params.shape[0] * f.params.shape[1]
            o = ref.search_strengths(f.rec, f.src, f.bitdepth, d, lam)
            assert np.array_equal(dl_b[o0 * 64:(o0 + b) * 64].cpu().numpy().reshape(b, 64),
                                  o["dist_luma"])
            assert np.array_equal(dc_b[o0 * 64:(o0 + b) * 64].cpu().numpy().reshape(b, 64),
                                  o["dist_chroma"])
            assert r["npresets"] == o["npresets"] and r["cost"] == o["cost"]
            assert [cdef.preset_index(p) for p in r["presets"][:r["npresets"]]] == \
                [int(t) for t in o["presets"][:o["npresets"]]]
            assert np.array_equal(ids_b[o0:o0 + b].cpu().numpy(), o["block_ids"])
            o0 += b
    return res_b


def test_noalloc_matches_search_strengths_twice(cdef, ref):
    r1 = _run_both(cdef, ref, [(136, 72, 8), (64, 64, 10)], seed=500)
    r2 = _run_both(cdef, ref, [(200, 136, 8), (80, 64, 10), (8, 8, 8)], seed=600)
    assert len(r1) == 2 and len(r2) == 3


def test_noalloc_48_frames(cdef, ref):
    """The frame limit: 48 frames in one call, against the oracle."""
    sizes = [(64, 64, 8), (72, 40, 10), (128, 64, 8), (8, 16, 10)]
    _run_both(cdef, ref, [sizes[k % 4] for k in range(48)], seed=700)


def test_noalloc_near_capacity(cdef):
    """8 frames of 3840x2160 (16320 filter blocks of the 16384 the array
    holds): the minima, the preset totals behind them and the result records
    fill the array up to its end; bit-exact against cdef_search_strengths."""
    from paper_1602_05975_gb300 import synth
    f = synth.make_frame(3840, 2160, 8, 32, seed=800)
    rec, src = cdef.frame_from_numpy(f.rec, 8), cdef.frame_from_numpy(f.src, 8)
    n = 8
    tot = n * f.params.shape[0] * f.params.shape[1]
    assert MAX_BLOCKS - 64 <= tot <= MAX_BLOCKS
    damping, lambdas = [3, 4, 5, 6] * 2, [64 << k for k in range(n)]
    ctx = cdef.Context(0)
    ids_a, dl_a, dc_a = _outputs(tot)
    res_a = cdef.cdef_search_strengths(ctx, [rec] * n, [src] * n, damping, lambdas, ids_a, dl_a, dc_a)
    ctx.close()
    res_b, ids_b, dl_b, dc_b = _noalloc(cdef, [rec] * n, [src] * n, damping, lambdas, tot)
    assert torch.equal(dl_a, dl_b) and torch.equal(dc_a, dc_b) and torch.equal(ids_a, ids_b)
    assert res_a == res_b


def test_noalloc_rejects_over_capacity(cdef):
    # 8192 x 8256 luma = 128 x 129 = 16512 filter blocks > 16384
    w, h = 8192, 8256
    f = cdef.alloc_frame(w, h, 8, fill=0)
    ids = torch.zeros(1, dtype=torch.uint8, device="cuda")
    d = torch.zeros(64, dtype=torch.int64, device="cuda")
    with pytest.raises(cdef.CdefError) as e:
        cdef.cdef_search_strengths_noalloc([f], [f], [4], [0], ids, d, d)
    assert e.value.status == -4
    assert np.all(ids.cpu().numpy() == 0)


@pytest.mark.parametrize("bd,chroma,status", [(12, 420, -3), (8, 444, -2), (10, 422, -2)])
def test_noalloc_rejects_other_formats(cdef, bd, chroma, status):
    """Only 8- and 10-bit 4:2:0 frames: 12-bit frames get CDEF_ERR_BITDEPTH,
    4:4:4 and 4:2:2 frames CDEF_ERR_SIZE, before any work."""
    f = cdef.alloc_frame(64, 64, bd, fill=0, chroma=chroma)
    ids, dl, dc = _outputs(1, 9, 9)
    with pytest.raises(cdef.CdefError) as e:
        cdef.cdef_search_strengths_noalloc([f], [f], [4], [0], ids, dl, dc)
    assert e.value.status == status
    assert int(ids[0]) == 9 and int(dl[0]) == 9


def test_noalloc_reports_a_wait_that_runs_out(cdef, ref):
    """A bounded tile-load wait that gives up (cdef_debug_set_waits: a short
    limit, bytes no copy delivers) comes back as CDEF_ERR_TIMEOUT from the
    call itself; the next call (default limits) is bit-exact again: the
    status word is cleared per call and the work counters were reset."""
    from paper_1602_05975_gb300 import synth
    f = synth.make_frame(200, 136, 8, 32, seed=900)
    rec, src = cdef.frame_from_numpy(f.rec, 8), cdef.frame_from_numpy(f.src, 8)
    tot = f.params.shape[0] * f.params.shape[1]
    ids, dl, dc = _outputs(tot)
    cdef.debug_set_waits(1 << 16, 16)
    try:
        with pytest.raises(cdef.CdefError) as e:
            cdef.cdef_search_strengths_noalloc([rec], [src], [5], [900], ids, dl, dc)
    finally:
        cdef.debug_set_waits(0, 0)
    assert e.value.status == -6
    for _ in range(2):
        res, ids, dl, dc = _noalloc(cdef, [rec], [src], [5], [900], tot)
        o = ref.search_strengths(f.rec, f.src, 8, 5, 900)
        assert np.array_equal(dl.cpu().numpy().reshape(tot, 64), o["dist_luma"])
        assert np.array_equal(dc.cpu().numpy().reshape(tot, 64), o["dist_chroma"])
        assert res[0]["cost"] == o["cost"] and res[0]["npresets"] == o["npresets"]
        assert np.array_equal(ids.cpu().numpy(), o["block_ids"])
