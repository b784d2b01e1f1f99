"""The allocation-free strength search (cdef_search_strengths_noalloc).

Callers that may not allocate device memory after start-up (a codec given a
fixed memory budget by its host application, a real-time loop that cannot
take the synchronisation cudaMalloc/cudaFree may cause) use this entry
point: no context, scratch in a fixed array inside the library.  This test
calls it through the C ABI twice in a row, each time on different frames,
and checks every output against cdef_search_strengths; the search is integer
arithmetic, so the tolerance is zero, as in the other parity tests.  The
file name makes pytest collect it last.
"""
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
    torch.cuda.set_device(0)
    return _c


def _run_both(cdef, specs, seed):
    from paper_1602_05975_gb300 import synth
    frames = [synth.make_frame(w, h, bd, None, seed=seed + k) for k, (w, h, bd) in enumerate(specs)]
    recs = [cdef.frame_from_numpy(f.rec, f.bitdepth) for f in frames]
    srcs = [cdef.frame_from_numpy(f.src, f.bitdepth) for f in frames]
    tot = sum(f.params.shape[0] * f.params.shape[1] for f in frames)
    damping = [3 + (k % 4) for k in range(len(frames))]
    lambdas = [int(f.q) ** 2 << (2 * (f.bitdepth - 8)) for f in frames]

    # existing entry point (context scratch)
    ctx = cdef.Context(0)
    ids_a = torch.zeros(tot, dtype=torch.uint8, device="cuda")
    dl_a = torch.zeros(tot * 64, dtype=torch.int64, device="cuda")
    dc_a = torch.zeros(tot * 64, dtype=torch.int64, device="cuda")
    res_a = cdef.cdef_search_strengths(ctx, recs, srcs, damping, lambdas, ids_a, dl_a, dc_a)
    ctx.close()

    # allocation-free entry point; outputs pre-filled with garbage
    ids_b = torch.full((tot,), 77, dtype=torch.uint8, device="cuda")
    dl_b = torch.full((tot * 64,), -5, dtype=torch.int64, device="cuda")
    dc_b = torch.full((tot * 64,), -5, dtype=torch.int64, device="cuda")
    res_b = cdef.cdef_search_strengths_noalloc(recs, srcs, damping, lambdas, ids_b, dl_b, dc_b)
    torch.cuda.synchronize()

    assert torch.equal(dl_a, dl_b) and torch.equal(dc_a, dc_b)
    assert torch.equal(ids_a, ids_b)
    for a, b in zip(res_a, res_b):
        assert a["npresets"] == b["npresets"] and a["cost"] == b["cost"]
        assert a["presets"] == b["presets"]
    return res_b


def test_noalloc_matches_search_strengths_twice(cdef):
    r1 = _run_both(cdef, [(136, 72, 8), (64, 64, 10)], seed=500)
    r2 = _run_both(cdef, [(200, 136, 8), (80, 64, 10), (8, 8, 8)], seed=600)
    assert len(r1) == 2 and len(r2) == 3


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
