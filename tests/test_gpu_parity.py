"""GPU parity: the CUDA path (through the C ABI) against the oracle, bit for
bit on every direction, contrast, output sample and int64 distortion.  All
integer work: the tolerance is zero."""
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


def _gpu_filter(cdef, ctx, planes, bd, params, with_maps=False):
    h, w = planes[0].shape
    inp = cdef.frame_from_numpy(planes, bd)
    out = cdef.alloc_frame(w, h, bd, fill=0)
    prm = cdef.params_tensor(params)
    if with_maps:
        dirs = torch.zeros((h // 8) * (w // 8), dtype=torch.uint8, device="cuda")
        var = torch.zeros((h // 8) * (w // 8), dtype=torch.int32, device="cuda")
        cdef.cdef_find_dir(ctx, inp.y, w, h, bd, dirs, var)
        cdef.cdef_filter_frame(ctx, inp, prm, out, dirs, var)
    else:
        cdef.cdef_filter_frame(ctx, inp, prm, out)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    return out.to_numpy()


def _assert_frames_equal(got, exp):
    for g, e, name in zip(got, exp, "yuv"):
        bad = np.argwhere(g != e)
        assert bad.size == 0, f"plane {name}: {len(bad)} mismatches, first at {bad[:5].tolist()}"


# --------------------------------------------------------------- direction search
@pytest.mark.parametrize("w,h,bd,kind", [
    (8, 8, 8, "rand"), (352, 288, 8, "synth"), (136, 72, 10, "rand"),
    (200, 96, 10, "synth"), (64, 48, 12, "rand"), (1024, 8, 8, "rand")])
def test_find_dir_parity(cdef, ctx, ref, w, h, bd, kind):
    from paper_1602_05975_gb300 import synth
    rng = np.random.default_rng(w + h + bd)
    if kind == "rand":
        y = synth.random_frame_planes(rng, w, h, bd)[0]
    else:
        y = synth.make_frame(w, h, bd, 32, seed=5).rec[0]
    inp = cdef.frame_from_numpy((y, y[::2, ::2], y[::2, ::2]), bd)
    dirs = torch.zeros((h // 8) * (w // 8), dtype=torch.uint8, device="cuda")
    var = torch.zeros_like(dirs, dtype=torch.int32)
    cdef.cdef_find_dir(ctx, inp.y, w, h, bd, dirs, var)
    torch.cuda.synchronize()
    ed, ev = ref.find_dir(y, bd)
    assert np.array_equal(dirs.cpu().numpy().reshape(ed.shape), ed)
    assert np.array_equal(var.cpu().numpy().reshape(ev.shape), ev)


def test_find_dir_extremes(cdef, ctx, ref):
    """Constant, perfectly directional and maximum-contrast blocks."""
    blocks = [np.full((8, 8), 0), np.full((8, 8), 255),
              np.where(np.indices((8, 8)).sum(0) % 2 == 0, 255, 0)]
    ii, jj = np.indices((8, 8))
    for key in (ii + jj, ii, jj, ii - jj + 7, ii + jj // 2, ii // 2 + jj):
        blocks.append((key * 37) % 256)
    y = np.concatenate(blocks, axis=1).astype(np.uint16)
    h, w = y.shape
    inp = cdef.frame_from_numpy((y, y[::2, ::2], y[::2, ::2]), 8)
    dirs = torch.zeros(w // 8, dtype=torch.uint8, device="cuda")
    var = torch.zeros(w // 8, dtype=torch.int32, device="cuda")
    cdef.cdef_find_dir(ctx, inp.y, w, h, 8, dirs, var)
    torch.cuda.synchronize()
    ed, ev = ref.find_dir(y, 8)
    assert np.array_equal(dirs.cpu().numpy(), ed.reshape(-1))
    assert np.array_equal(var.cpu().numpy(), ev.reshape(-1))


# --------------------------------------------------------------- filter
FILTER_CASES = [
    (8, 8, 8, "rand"), (16, 8, 8, "rand"), (72, 72, 8, "rand"), (72, 72, 10, "rand"),
    (352, 288, 8, "synth"), (136, 80, 10, "synth"), (200, 136, 8, "synth"),
    (64, 64, 10, "rand"), (120, 16, 12, "rand"), (8, 200, 8, "synth"),
]


@pytest.mark.parametrize("w,h,bd,kind", FILTER_CASES)
@pytest.mark.parametrize("with_maps", [False, True])
def test_filter_parity(cdef, ctx, ref, w, h, bd, kind, with_maps):
    from paper_1602_05975_gb300 import synth
    rng = np.random.default_rng(w * 7 + h * 3 + bd)
    if kind == "rand":
        planes = synth.random_frame_planes(rng, w, h, bd)
    else:
        planes = synth.make_frame(w, h, min(bd, 10), 32, seed=w + h).rec
        if bd == 12:
            planes = tuple(p << 2 for p in planes)
    prm = synth.random_params(rng, w, h)
    got = _gpu_filter(cdef, ctx, planes, bd, prm, with_maps)
    exp = ref.filter_frame(*planes, bd, prm)
    _assert_frames_equal(got, exp)


@pytest.mark.parametrize("bd", [8, 10])
def test_filter_every_strength(cdef, ctx, ref, bd):
    """Every (primary, secondary, damping) combination, one per filter block,
    including the special values 19 and 7."""
    from paper_1602_05975_gb300 import synth
    combos = [(p, s, d) for p in list(range(16)) + [19] for s in (0, 1, 2, 4, 7) for d in (3, 4, 5, 6)]
    fbc = 20
    fbr = -(-len(combos) // fbc)
    w, h = fbc * 64, fbr * 64
    fr = synth.make_frame(w, h, bd, 64, seed=bd)
    prm = np.zeros((fbr, fbc, 8), np.uint8)
    rng = np.random.default_rng(bd)
    for k, (p, s, d) in enumerate(combos):
        prm[k // fbc, k % fbc, :5] = (p, s, combos[-1 - k][0], combos[-1 - k][1], d)
    got = _gpu_filter(cdef, ctx, fr.rec, bd, prm)
    exp = ref.filter_frame(*fr.rec, bd, prm)
    _assert_frames_equal(got, exp)
    del rng


def test_filter_extreme_planes(cdef, ctx, ref):
    from paper_1602_05975_gb300 import synth
    rng = np.random.default_rng(99)
    for bd in (8, 10):
        mx = (1 << bd) - 1
        for planes in (
            tuple(np.zeros(s, np.uint16) for s in ((40, 48), (20, 24), (20, 24))),
            tuple(np.full(s, mx, np.uint16) for s in ((40, 48), (20, 24), (20, 24))),
            tuple((rng.integers(0, 2, s) * mx).astype(np.uint16) for s in ((40, 48), (20, 24), (20, 24))),
        ):
            prm = synth.random_params(rng, 48, 40)
            prm[..., 0] = 15
            prm[..., 1] = 4
            got = _gpu_filter(cdef, ctx, planes, bd, prm)
            exp = ref.filter_frame(*planes, bd, prm)
            _assert_frames_equal(got, exp)


def test_filter_batch_mixed(cdef, ctx, ref):
    """One launch over frames of different sizes and bit depths equals each
    frame filtered alone."""
    from paper_1602_05975_gb300 import synth
    specs = [(136, 72, 8), (64, 64, 10), (352, 288, 8), (8, 8, 10), (200, 136, 10)]
    frames, ins, outs, prms = [], [], [], []
    for k, (w, h, bd) in enumerate(specs):
        fr = synth.make_frame(w, h, bd, 32, seed=100 + k)
        frames.append(fr)
        ins.append(cdef.frame_from_numpy(fr.rec, bd))
        outs.append(cdef.alloc_frame(w, h, bd, fill=0))
        prms.append(cdef.params_tensor(fr.params))
    cdef.cdef_filter_frames(ctx, ins, prms, outs)
    torch.cuda.synchronize()
    for fr, o in zip(frames, outs):
        _assert_frames_equal(o.to_numpy(), ref.filter_frame(*fr.rec, fr.bitdepth, fr.params))


# Launches with more filter blocks than one round of persistent CTAs (4 per
# SM), so that CTAs take several blocks from the work counter and the last
# round is partial: frames with ragged right and bottom edges, coded maps,
# 4:2:2 and 12-bit frames, against the oracle.
@pytest.mark.parametrize("w,h,bd,fmt,with_map", [
    (2600, 1096, 10, 420, False), (2600, 1096, 8, 420, True), (2600, 1096, 8, 422, False),
    (2600, 1096, 12, 420, False)])
def test_filter_rounds_parity(cdef, ctx, ref, w, h, bd, fmt, with_map):
    from paper_1602_05975_gb300 import synth
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert -(-w // 64) * -(-h // 64) > 4 * sms   # more blocks than one round
    rng = np.random.default_rng(w + h + bd + fmt)
    planes = synth.make_frame(w, h, bd, 32, seed=990 + bd + fmt, chroma=fmt).rec
    params = synth.random_params(rng, w, h)
    params[..., 5] = rng.integers(0, 4, params.shape[:2])
    coded = (rng.random((h // 8, w // 8)) < 0.6).astype(np.uint8) if with_map else None
    ctx.set_overlap(False)
    inp = cdef.frame_from_numpy(planes, bd)
    out = cdef.alloc_frame(w, h, bd, fill=0, chroma=fmt)
    prm = cdef.params_tensor(params)
    if with_map:
        cdef.cdef_filter_frame_coded(ctx, inp, prm, torch.from_numpy(coded.reshape(-1)).cuda(), out)
    else:
        cdef.cdef_filter_frame(ctx, inp, prm, out)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    _assert_frames_equal(out.to_numpy(), ref.filter_frame_format(*planes, bd, params, fmt, coded))


def test_filter_rounds_batch(cdef, ctx, ref):
    """One launch over frames whose blocks together exceed one round of CTAs:
    the partial last round falls in the last frames of the batch."""
    from paper_1602_05975_gb300 import synth
    specs = [(1280, 720, 10), (1288, 728, 8), (1280, 720, 10), (648, 360, 8)]
    frames, ins, outs, prms = [], [], [], []
    for k, (w, h, bd) in enumerate(specs):
        fr = synth.make_frame(w, h, bd, 32, seed=1000 + k)
        frames.append(fr)
        ins.append(cdef.frame_from_numpy(fr.rec, bd))
        outs.append(cdef.alloc_frame(w, h, bd, fill=0))
        prms.append(cdef.params_tensor(fr.params))
    ctx.set_overlap(False)
    cdef.cdef_filter_frames(ctx, ins, prms, outs)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    for fr, o in zip(frames, outs):
        _assert_frames_equal(o.to_numpy(), ref.filter_frame(*fr.rec, fr.bitdepth, fr.params))


def test_invalid_params_flagged(cdef, ctx):
    from paper_1602_05975_gb300 import synth
    fr = synth.make_frame(128, 64, 8, 32, seed=7)
    prm = fr.params.copy()
    prm[0, 1, 0] = 16  # primary strength out of range
    inp = cdef.frame_from_numpy(fr.rec, 8)
    out = cdef.alloc_frame(128, 64, 8, fill=0)
    ctx.status(clear=True)
    word = torch.full((1,), -7, dtype=torch.int32).pin_memory()
    ctx.status_async(word)                                    # before: clean
    torch.cuda.synchronize()
    assert int(word[0]) == 0
    cdef.cdef_filter_frame(ctx, inp, cdef.params_tensor(prm), out)
    ctx.status_async(word)                                    # after, in stream order
    torch.cuda.synchronize()
    assert int(word[0]) != 0
    assert ctx.status(clear=True) == -1
    y = out.to_numpy()[0]
    assert np.array_equal(y[:, 64:128], fr.rec[0][:, 64:128])  # block left unfiltered
    assert ctx.status() == 0


def test_argument_errors(cdef, ctx):
    f = cdef.alloc_frame(64, 64, 8)
    o = cdef.alloc_frame(64, 64, 8)
    prm = torch.zeros(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(cdef.CdefError) as e:
        cdef.cdef_filter_frame(ctx, f, prm, f)  # in-place
    assert e.value.status == -1
    bad = cdef.Frame(f.y, f.u, f.v, 60, 64, 8)  # width not a multiple of 8
    with pytest.raises(cdef.CdefError) as e:
        cdef.cdef_filter_frame(ctx, bad, prm, o)
    assert e.value.status == -2
    o10 = cdef.alloc_frame(64, 64, 10)
    with pytest.raises(cdef.CdefError) as e:
        cdef.cdef_filter_frame(ctx, f, prm, o10)  # bit depth mismatch
    assert e.value.status == -2
    odd = cdef.Frame(f.y[:, 1:], f.u, f.v, 56, 64, 8)  # misaligned data pointer
    with pytest.raises(cdef.CdefError) as e:
        cdef.cdef_filter_frame(ctx, odd, prm, o)
    assert e.value.status == -1
    b7 = cdef.Frame(f.y, f.u, f.v, 64, 64, 7)
    with pytest.raises(cdef.CdefError) as e:
        cdef.cdef_filter_frame(ctx, b7, prm, o)
    assert e.value.status == -3


# --------------------------------------------------------------- strength search
SEARCH_CASES = [
    [(128, 72, 8)],
    [(80, 64, 10)],
    [(64, 64, 8), (136, 72, 8), (72, 136, 10)],
    [(8, 8, 8)],
]


@pytest.mark.parametrize("specs", SEARCH_CASES)
def test_search_parity(cdef, ctx, ref, specs):
    from paper_1602_05975_gb300 import synth
    frames = [synth.make_frame(w, h, bd, None, seed=200 + k) for k, (w, h, bd) in enumerate(specs)]
    recs = [cdef.frame_from_numpy(f.rec, f.bitdepth) for f in frames]
    srcs = [cdef.frame_from_numpy(f.src, f.bitdepth) for f in frames]
    nbs = [f.params.shape[0] * f.params.shape[1] for f in frames]
    tot = sum(nbs)
    damping = [3 + (k % 4) for k in range(len(frames))]
    lambdas = [int(f.q) ** 2 * (1 << (2 * (f.bitdepth - 8))) for f in frames]
    ids = torch.zeros(tot, dtype=torch.uint8, device="cuda")
    dl = torch.zeros(tot * 64, dtype=torch.int64, device="cuda")
    dc = torch.zeros(tot * 64, dtype=torch.int64, device="cuda")
    res = cdef.cdef_search_strengths(ctx, recs, srcs, damping, lambdas, ids, dl, dc)
    dl, dc, ids = dl.cpu().numpy(), dc.cpu().numpy(), ids.cpu().numpy()
    off = 0
    for k, f in enumerate(frames):
        o = ref.search_strengths(f.rec, f.src, f.bitdepth, damping[k], lambdas[k])
        nb = nbs[k]
        assert np.array_equal(dl[off * 64:(off + nb) * 64].reshape(nb, 64), o["dist_luma"])
        assert np.array_equal(dc[off * 64:(off + nb) * 64].reshape(nb, 64), o["dist_chroma"])
        assert res[k]["npresets"] == o["npresets"]
        assert res[k]["cost"] == o["cost"]
        got_t = [cdef.preset_index(p) for p in res[k]["presets"]]
        assert got_t == list(o["presets"])
        assert np.array_equal(ids[off:off + nb], o["block_ids"])
        off += nb


def test_search_scratch_tables(cdef, ctx, ref):
    """With no caller tables the context's scratch is used; presets equal."""
    from paper_1602_05975_gb300 import synth
    f = synth.make_frame(136, 72, 8, 16, seed=300)
    ids = torch.zeros(6, dtype=torch.uint8, device="cuda")
    res = cdef.cdef_search_strengths(ctx, [cdef.frame_from_numpy(f.rec, 8)],
                                     [cdef.frame_from_numpy(f.src, 8)], [5], [256], ids)[0]
    o = ref.search_strengths(f.rec, f.src, 8, 5, 256)
    assert res["cost"] == o["cost"] and res["npresets"] == o["npresets"]
    assert np.array_equal(ids.cpu().numpy(), o["block_ids"])


@pytest.mark.parametrize("groups,ctas", [(1, 2), (1, 1), (2, 2), (4, 2), (0, 0)])
def test_search_every_launch_configuration(cdef, ctx, ref, groups, ctas):
    """Every configuration the autotuner may pick (and the autotuner itself)
    gives the oracle's tables, presets, ids and J, on a mixed 8/10-bit batch
    whose frames have ragged edges."""
    from paper_1602_05975_gb300 import synth
    specs = [(200, 136, 8, 16, 600), (136, 72, 10, 32, 601), (72, 264, 8, 64, 602)]
    frames = [synth.make_frame(w, h, bd, q, seed=s) for w, h, bd, q, s in specs]
    nb = sum(f.params.shape[0] * f.params.shape[1] for f in frames)
    ids = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    dl = torch.zeros(nb * 64, dtype=torch.int64, device="cuda")
    dc = torch.zeros(nb * 64, dtype=torch.int64, device="cuda")
    ctx.set_tuning(groups, ctas)
    try:
        res = cdef.cdef_search_strengths(ctx, [cdef.frame_from_numpy(f.rec, f.bitdepth) for f in frames],
                                         [cdef.frame_from_numpy(f.src, f.bitdepth) for f in frames],
                                         [5, 4, 6], [256, 1024, 4096], ids, dl, dc)
        used = ctx.tuning()
    finally:
        ctx.set_tuning(0, 0)
    if groups:
        assert used == (groups, ctas)
    else:
        assert used in [(1, 2), (1, 1), (2, 2), (4, 2)]
    o0 = 0
    for f, r, d, lam in zip(frames, res, [5, 4, 6], [256, 1024, 4096]):
        b = f.params.shape[0] * f.params.shape[1]
        o = ref.search_strengths(f.rec, f.src, f.bitdepth, d, lam)
        assert np.array_equal(dl[o0 * 64:(o0 + b) * 64].cpu().numpy().reshape(b, 64), o["dist_luma"])
        assert np.array_equal(dc[o0 * 64:(o0 + b) * 64].cpu().numpy().reshape(b, 64), o["dist_chroma"])
        assert np.array_equal(ids[o0:o0 + b].cpu().numpy(), o["block_ids"])
        assert r["cost"] == o["cost"] and r["npresets"] == o["npresets"]
        o0 += b


def test_tuning_rejects_unknown_configurations(cdef, ctx):
    for g, c, k in [(3, 1, 0), (8, 1, 0), (1, 3, 0), (-1, 0, 0), (0, 0, 2), (0, 0, -1)]:
        with pytest.raises(cdef.CdefError):
            ctx.set_tuning(g, c, preset_kernel=k)
    ctx.set_tuning(0, 0)


# --------------------------------------------------------------- full-size frames
@pytest.mark.parametrize("w,h,bd,seed", [(3840, 2160, 10, 2000), (1920, 1080, 8, 1000)])
def test_benchmark_frames_full(cdef, ctx, ref, w, h, bd, seed):
    """The benchmark's own frames and launch (fused direction search), every
    output sample and the standalone direction maps against the oracle."""
    from paper_1602_05975_gb300 import synth
    f = synth.make_frame(w, h, bd, None, seed)
    _assert_frames_equal(_gpu_filter(cdef, ctx, f.rec, bd, f.params),
                         ref.filter_frame(*f.rec, bd, f.params))
    inp = cdef.frame_from_numpy(f.rec, bd)
    dirs = torch.zeros((h // 8) * (w // 8), dtype=torch.uint8, device="cuda")
    var = torch.zeros_like(dirs, dtype=torch.int32)
    cdef.cdef_find_dir(ctx, inp.y, w, h, bd, dirs, var)
    torch.cuda.synchronize()
    ed, ev = ref.find_dir(f.rec[0], bd)
    assert np.array_equal(dirs.cpu().numpy().reshape(ed.shape), ed)
    assert np.array_equal(var.cpu().numpy().reshape(ev.shape), ev)


@pytest.mark.parametrize("bd", [8, 10])
def test_largest_frame_sampled(cdef, ctx, ref, bd):
    """7680x4320 (8K): the whole frame on the GPU; sampled 64x64 blocks
    (corners, edges, interior) against the oracle run on the 3x3-block
    neighbourhood with the full frame's direction maps.  A block's output
    depends only on its pixels, a 2-pixel halo, its parameters and its 8x8
    directions, so the centre block of such a crop is exact."""
    from paper_1602_05975_gb300 import synth
    w, h = 7680, 4320
    rng = np.random.default_rng(bd)
    planes = synth.random_frame_planes(rng, w, h, bd)
    # smooth the random planes a little so that directions and strengths vary
    planes = tuple(((p.astype(np.int64) + np.roll(p, 1, 0) + np.roll(p, 1, 1)) // 3).astype(np.uint16)
                   for p in planes)
    params = synth.random_params(rng, w, h)
    got = _gpu_filter(cdef, ctx, planes, bd, params)
    dirs, var = ref.find_dir(planes[0], bd)
    rows, cols = params.shape[:2]
    picks = [(0, 0), (0, cols - 1), (rows - 1, 0), (rows - 1, cols - 1), (0, cols // 2),
             (rows // 2, 0), (rows - 1, cols // 3)] + \
            [(int(rng.integers(1, rows - 1)), int(rng.integers(1, cols - 1))) for _ in range(5)]
    for by, bx in picks:
        r0, r1 = max(by - 1, 0), min(by + 2, rows)
        c0, c1 = max(bx - 1, 0), min(bx + 2, cols)
        y0, y1, x0, x1 = r0 * 64, min(r1 * 64, h), c0 * 64, min(c1 * 64, w)
        crop = (planes[0][y0:y1, x0:x1], planes[1][y0 // 2:y1 // 2, x0 // 2:x1 // 2],
                planes[2][y0 // 2:y1 // 2, x0 // 2:x1 // 2])
        exp = ref.filter_frame(*crop, bd, params[r0:r1, c0:c1],
                               dirs[y0 // 8:y1 // 8, x0 // 8:x1 // 8],
                               var[y0 // 8:y1 // 8, x0 // 8:x1 // 8])
        ly, lx = by * 64, bx * 64
        ey, ex = min(ly + 64, h), min(lx + 64, w)
        assert np.array_equal(got[0][ly:ey, lx:ex], exp[0][ly - y0:ey - y0, lx - x0:ex - x0]), (by, bx)
        for k in (1, 2):
            assert np.array_equal(got[k][ly // 2:ey // 2, lx // 2:ex // 2],
                                  exp[k][(ly - y0) // 2:(ey - y0) // 2,
                                         (lx - x0) // 2:(ex - x0) // 2]), (by, bx, k)


@pytest.mark.parametrize("overlap", [False, True])
def test_consecutive_frames_on_one_stream(cdef, ctx, ref, overlap):
    """A run of filter calls on one stream, launched as programmatic
    dependents of each other, with and without the independence promise:
    every frame equals the oracle."""
    from paper_1602_05975_gb300 import synth
    frames = [synth.make_frame(w, h, bd, None, 700 + i)
              for i, (w, h, bd) in enumerate([(352, 288, 8), (640, 360, 10), (200, 136, 8),
                                              (640, 360, 10), (1280, 720, 8), (96, 64, 10)])]
    ins = [cdef.frame_from_numpy(f.rec, f.bitdepth) for f in frames]
    outs = [cdef.alloc_frame(f.width, f.height, f.bitdepth, fill=0) for f in frames]
    prms = [cdef.params_tensor(f.params) for f in frames]
    stream = torch.cuda.Stream()
    ctx.set_overlap(overlap)
    try:
        for _ in range(3):
            for i, o, p in zip(ins, outs, prms):
                cdef.cdef_filter_frame(ctx, i, p, o, stream=stream)
        stream.synchronize()
    finally:
        ctx.set_overlap(False)
    assert ctx.status() == 0
    for f, o in zip(frames, outs):
        _assert_frames_equal(o.to_numpy(), ref.filter_frame(*f.rec, f.bitdepth, f.params))


def test_stream_order_kept_without_overlap(cdef, ctx, ref):
    """Without the promise a filter call reads what the kernel just before
    it on the stream wrote: filter a frame, then filter that output again."""
    from paper_1602_05975_gb300 import synth
    f = synth.make_frame(640, 360, 10, 32, seed=720)
    a = cdef.frame_from_numpy(f.rec, 10)
    b = cdef.alloc_frame(640, 360, 10, fill=0)
    c = cdef.alloc_frame(640, 360, 10, fill=0)
    p = cdef.params_tensor(f.params)
    stream = torch.cuda.Stream()
    cdef.cdef_filter_frame(ctx, a, p, b, stream=stream)
    cdef.cdef_filter_frame(ctx, b, p, c, stream=stream)
    stream.synchronize()
    once = ref.filter_frame(*f.rec, 10, f.params)
    _assert_frames_equal(c.to_numpy(), ref.filter_frame(*once, 10, f.params))


@pytest.mark.parametrize("passes,grid", [(1, 0), (4, 0), (16, 0), (1, 1), (4, 1)])
def test_search_preset_refinement(cdef, ctx, ref, passes, grid):
    """Section 5's one-at-a-time re-optimisation of the presets after the
    greedy search: presets, N, J and block ids equal the oracle's, with the
    cluster-per-frame and with the grid-wide preset kernel."""
    from paper_1602_05975_gb300 import synth
    specs = [(200, 136, 8, 16, 610), (136, 72, 10, 32, 611), (320, 192, 8, 64, 612)]
    frames = [synth.make_frame(w, h, bd, q, seed=s) for w, h, bd, q, s in specs]
    damping, lambdas = [5, 4, 6], [64, 512, 4096]
    nb = sum(f.params.shape[0] * f.params.shape[1] for f in frames)
    ids = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    ctx.set_search_refine(passes)
    ctx.set_tuning(0, 0, preset_kernel=grid)
    try:
        res = cdef.cdef_search_strengths(ctx, [cdef.frame_from_numpy(f.rec, f.bitdepth) for f in frames],
                                         [cdef.frame_from_numpy(f.src, f.bitdepth) for f in frames],
                                         damping, lambdas, ids)
    finally:
        ctx.set_search_refine(0)
        ctx.set_tuning(0, 0)
    assert ctx.status() == 0
    o0 = 0
    for f, r, d, lam in zip(frames, res, damping, lambdas):
        b = f.params.shape[0] * f.params.shape[1]
        o = ref.search_strengths(f.rec, f.src, f.bitdepth, d, lam, refine_passes=passes)
        g = ref.search_strengths(f.rec, f.src, f.bitdepth, d, lam)
        assert r["npresets"] == o["npresets"] and r["cost"] == o["cost"] <= g["cost"]
        assert ([cdef.preset_index(p) for p in r["presets"][:r["npresets"]]] ==
                [int(t) for t in o["presets"][:o["npresets"]]])
        assert np.array_equal(ids[o0:o0 + b].cpu().numpy(), o["block_ids"])
        o0 += b


def test_search_refine_rejects_bad_pass_counts(cdef, ctx):
    for p in (-1, 17):
        with pytest.raises(cdef.CdefError):
            ctx.set_search_refine(p)


# --------------------------------------------------------------- section 4 skip semantics
@pytest.mark.parametrize("w,h,bd,density", [(200, 136, 8, 0.5), (352, 288, 10, 0.2),
                                            (136, 72, 12, 0.7), (640, 360, 8, 0.0),
                                            (64, 64, 10, 1.0)])
def test_filter_coded_parity(cdef, ctx, ref, w, h, bd, density):
    """Coded-residual maps, skip-condition bits and the (0,0)+skip mapping:
    every output sample equals the oracle's."""
    from paper_1602_05975_gb300 import synth
    rng = np.random.default_rng(w * 3 + h + bd)
    f = synth.make_frame(w, h, bd, 32, seed=800 + w)
    params = synth.random_params(rng, w, h)
    params[..., 5] = rng.integers(0, 4, params.shape[:2])
    zero = rng.random(params.shape[:2]) < 0.3                 # some (0, 0) presets
    params[zero, 0] = 0
    params[zero, 1] = 0
    coded = (rng.random((h // 8, w // 8)) < density).astype(np.uint8)
    coded[:8, :8] = 0                                          # a skipped filter block
    inp = cdef.frame_from_numpy(f.rec, bd)
    out = cdef.alloc_frame(w, h, bd, fill=0)
    cmap = torch.from_numpy(coded.reshape(-1)).cuda()
    cdef.cdef_filter_frame_coded(ctx, inp, cdef.params_tensor(params), cmap, out)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    _assert_frames_equal(out.to_numpy(), ref.filter_frame(*f.rec, bd, params, coded=coded))


def test_filter_skip_bits_without_map(cdef, ctx, ref):
    """cdef_filter_frame (every block coded) honours the (0,0)+skip mapping."""
    from paper_1602_05975_gb300 import synth
    rng = np.random.default_rng(5)
    f = synth.make_frame(200, 136, 10, 32, seed=830)
    params = synth.random_params(rng, 200, 136)
    params[..., 0:4] = 0
    params[..., 5] = rng.integers(0, 4, params.shape[:2])
    _assert_frames_equal(_gpu_filter(cdef, ctx, f.rec, 10, params),
                         ref.filter_frame(*f.rec, 10, params))


def test_filter_bad_skip_bits_flagged(cdef, ctx):
    from paper_1602_05975_gb300 import synth
    f = synth.make_frame(64, 64, 8, 32, seed=831)
    params = f.params.copy()
    params[..., 5] = 4
    inp = cdef.frame_from_numpy(f.rec, 8)
    out = cdef.alloc_frame(64, 64, 8, fill=0)
    cdef.cdef_filter_frame(ctx, inp, cdef.params_tensor(params), out)
    torch.cuda.synchronize()
    assert ctx.status() != 0
    assert ctx.status() == 0          # cleared by the read
    got = out.to_numpy()
    assert all(np.array_equal(g, e) for g, e in zip(got, f.rec))


# --------------------------------------------------------------- 128-combination search
@pytest.mark.parametrize("groups,passes,grid", [(0, 0, 0), (1, 0, 0), (2, 0, 0), (4, 0, 0), (0, 4, 0),
                                               (0, 0, 1), (0, 4, 1)])
def test_search_coded_parity(cdef, ctx, ref, groups, passes, grid):
    """Section 5 with section 4's skip bits: 128-entry tables, skipped filter
    blocks, presets, N, J and ids equal the oracle's, for every launch
    configuration and with re-optimisation."""
    from paper_1602_05975_gb300 import synth
    specs = [(200, 136, 8, 16, 900), (136, 72, 10, 32, 901), (192, 128, 8, 64, 902)]
    frames = [synth.make_frame(w, h, bd, q, seed=s) for w, h, bd, q, s in specs]
    rng = np.random.default_rng(77)
    maps = []
    for f in frames:
        m = (rng.random((f.height // 8, f.width // 8)) < 0.6).astype(np.uint8)
        m[:8, :8] = 0                                          # first filter block skipped
        maps.append(m)
    damping, lambdas = [5, 4, 6], [64, 512, 4096]
    nb = sum(f.params.shape[0] * f.params.shape[1] for f in frames)
    ids = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    dl = torch.zeros(nb * 128, dtype=torch.int64, device="cuda")
    dc = torch.zeros(nb * 128, dtype=torch.int64, device="cuda")
    ctx.set_tuning(groups, 2 if groups else 0, preset_kernel=grid)
    ctx.set_search_refine(passes)
    try:
        res = cdef.cdef_search_strengths_coded(
            ctx, [cdef.frame_from_numpy(f.rec, f.bitdepth) for f in frames],
            [cdef.frame_from_numpy(f.src, f.bitdepth) for f in frames],
            [torch.from_numpy(m.reshape(-1)).cuda() for m in maps], damping, lambdas, ids, dl, dc)
    finally:
        ctx.set_tuning(0, 0)
        ctx.set_search_refine(0)
    assert ctx.status() == 0
    o0 = 0
    for f, m, r, d, lam in zip(frames, maps, res, damping, lambdas):
        b = f.params.shape[0] * f.params.shape[1]
        o = ref.search_strengths_coded(f.rec, f.src, f.bitdepth, d, lam, m, passes)
        assert np.array_equal(dl[o0 * 128:(o0 + b) * 128].cpu().numpy().reshape(b, 128),
                              o["dist_luma"])
        assert np.array_equal(dc[o0 * 128:(o0 + b) * 128].cpu().numpy().reshape(b, 128),
                              o["dist_chroma"])
        assert r["npresets"] == o["npresets"] and r["cost"] == o["cost"]
        assert ([cdef.preset_index_coded(p) for p in r["presets"][:r["npresets"]]] ==
                [int(t) for t in o["presets"][:o["npresets"]]])
        assert np.array_equal(ids[o0:o0 + b].cpu().numpy(), o["block_ids"])
        o0 += b


# --------------------------------------------------------------- chroma formats
@pytest.mark.parametrize("fmt,w,h,bd", [(422, 200, 136, 8), (444, 200, 136, 10),
                                        (444, 352, 288, 8), (422, 136, 72, 12),
                                        (444, 72, 64, 12)])
@pytest.mark.parametrize("with_map", [False, True])
def test_filter_chroma_formats(cdef, ctx, ref, fmt, w, h, bd, with_map):
    """4:2:2 (chroma copied, section 4) and 4:4:4 (full-resolution chroma)
    frames: every output sample equals the oracle's."""
    from paper_1602_05975_gb300 import synth
    rng = np.random.default_rng(fmt + w + bd)
    f = synth.make_frame(w, h, bd, 32, seed=950 + w)
    cw, ch = cdef.chroma_size(w, h, fmt)
    mx = (1 << bd) - 1
    u = np.clip(f.rec[0][:ch, :cw].astype(np.int64) // 2 + rng.integers(0, 60, (ch, cw)), 0, mx)
    v = np.clip(mx - f.rec[0][:ch, :cw].astype(np.int64) + rng.integers(0, 60, (ch, cw)), 0, mx)
    planes = (f.rec[0], u.astype(np.uint16), v.astype(np.uint16))
    params = synth.random_params(rng, w, h)
    params[..., 5] = rng.integers(0, 4, params.shape[:2])
    coded = (rng.random((h // 8, w // 8)) < 0.6).astype(np.uint8) if with_map else None
    inp = cdef.frame_from_numpy(planes, bd)
    out = cdef.alloc_frame(w, h, bd, fill=0, chroma=fmt)
    prm = cdef.params_tensor(params)
    if with_map:
        cdef.cdef_filter_frame_coded(ctx, inp, prm, torch.from_numpy(coded.reshape(-1)).cuda(), out)
    else:
        cdef.cdef_filter_frame(ctx, inp, prm, out)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    _assert_frames_equal(out.to_numpy(), ref.filter_frame_format(*planes, bd, params, fmt, coded))


@pytest.mark.parametrize("bd", [8, 10])
def test_filter_444_consecutive_and_given_maps(cdef, ctx, ref, bd):
    """8/10-bit 4:4:4 frames filtered by the three-plane launch: four frames
    back to back on one stream with overlapped launches (each its own
    output), then the same frames with caller-supplied direction maps; every
    output sample equals the oracle's."""
    from paper_1602_05975_gb300 import synth
    rng = np.random.default_rng(960 + bd)
    sizes = [(136, 72), (200, 136), (64, 64), (72, 40)]
    frames, exps, prms = [], [], []
    for k, (w, h) in enumerate(sizes):
        f = synth.make_frame(w, h, bd, 32, seed=970 + k, chroma=444)
        params = synth.random_params(rng, w, h)
        frames.append(f)
        prms.append(params)
        exps.append(ref.filter_frame_format(*f.rec, bd, params, 444))
    ins = [cdef.frame_from_numpy(f.rec, bd) for f in frames]
    s = torch.cuda.Stream()
    for given in (False, True):
        outs = [cdef.alloc_frame(f.width, f.height, bd, fill=0, chroma=444) for f in frames]
        maps = []
        ctx.set_overlap(not given)
        try:
            with torch.cuda.stream(s):
                for i, (f, inp) in enumerate(zip(frames, ins)):
                    if given:
                        d = torch.zeros((f.height // 8) * (f.width // 8), dtype=torch.uint8, device="cuda")
                        v = torch.zeros_like(d, dtype=torch.int32)
                        cdef.cdef_find_dir(ctx, inp.y, f.width, f.height, bd, d, v, stream=s)
                        maps.append((d, v))
                        cdef.cdef_filter_frame(ctx, inp, cdef.params_tensor(prms[i]), outs[i], d, v,
                                               stream=s)
                    else:
                        cdef.cdef_filter_frame(ctx, inp, cdef.params_tensor(prms[i]), outs[i], stream=s)
            torch.cuda.synchronize()
        finally:
            ctx.set_overlap(False)
        assert ctx.status() == 0
        for o, e in zip(outs, exps):
            _assert_frames_equal(o.to_numpy(), e)


def test_chroma_formats_rejected_where_unsupported(cdef, ctx):
    from paper_1602_05975_gb300 import synth
    f = synth.make_frame(64, 64, 8, 32, seed=960)
    y = f.rec[0]
    inp = cdef.frame_from_numpy((y, y, y), 8)                       # 4:4:4
    out = cdef.alloc_frame(64, 64, 8, fill=0, chroma=444)
    with pytest.raises(cdef.CdefError):
        cdef.cdef_filter_frames(ctx, [inp], [cdef.params_tensor(f.params)], [out])
    with pytest.raises(cdef.CdefError):     # the packed search of the no-allocation entry
        cdef.cdef_search_strengths_noalloc([inp], [inp], [4], [16],
                                           torch.zeros(1, dtype=torch.uint8, device="cuda"),
                                           torch.zeros(64, dtype=torch.int64, device="cuda"),
                                           torch.zeros(64, dtype=torch.int64, device="cuda"))


# --------------------------------------------------------------- eq. 14 distortion
def _eq14_term_counts(w, h, chroma=420):
    """Per filter block: how many 8x8 terms the luma entry and the chroma
    (U + V) entry sum (blocks cut by the frame edge count once)."""
    fr, fc = (h + 63) // 64, (w + 63) // 64
    cw, ch = {420: (w // 2, h // 2), 422: (w // 2, h), 444: (w, h)}[chroma]
    sx, sy = 64 * cw // w, 64 * ch // h          # chroma filter-block size
    nl = np.zeros(fr * fc, np.int64)
    nc = np.zeros(fr * fc, np.int64)
    for by in range(fr):
        for bx in range(fc):
            ly = min(64, h - by * 64)
            lx = min(64, w - bx * 64)
            nl[by * fc + bx] = -(-ly // 8) * -(-lx // 8)
            cy = min(sy, ch - by * sy)
            cx = min(sx, cw - bx * sx)
            nc[by * fc + bx] = 2 * (-(-cy // 8)) * (-(-cx // 8))
    return nl, nc


def _assert_eq14_tables_close(got, exp, nterms, cols=None):
    """The GPU's eq. 14 tables against the oracle's.  Per 8x8 term the GPU
    rounds an IEEE single-precision evaluation, within 0.5 + 2^-20 * value
    of the exact 256 * D (six correctly rounded operations); the oracle
    rounds a double-precision one, within 0.5 (plus a few double ulps) of
    it.  So an entry that sums n terms may differ by at most
    n + 2^-20 * (entry + n)."""
    got = np.asarray(got, np.int64)
    exp = np.asarray(exp, np.int64)
    if cols is not None:
        got, exp = got[:, cols], exp[:, cols]
    bound = nterms[:, None] + np.ceil((exp + nterms[:, None]) * 2.0 ** -20).astype(np.int64)
    diff = np.abs(got - exp)
    bad = np.argwhere(diff > bound)
    assert bad.size == 0, (f"{len(bad)} entries beyond the bound, first {bad[:3].tolist()}: "
                           f"got {got[tuple(bad[0])]}, oracle {exp[tuple(bad[0])]}")
    # and on average the two evaluations are well inside it
    assert diff.sum() <= bound.sum() // 2


@pytest.mark.parametrize("passes", [0, 2])
def test_search_eq14_parity(cdef, ctx, ref, passes):
    """Section 5's eq. 14 tables (8x8 SSIM weighting, 1/256 units): every
    GPU entry lies within the bound the two evaluations' precisions allow of
    the double-precision oracle's (4:2:0 chroma 8x8 blocks cut by the frame
    edge included), and the presets, N, J and ids the GPU returns are
    exactly the oracle's selection (greedy, re-optimised) on the GPU's own
    tables."""
    from paper_1602_05975_gb300 import synth
    specs = [(200, 136, 8, 16, 1100), (136, 72, 10, 32, 1101), (192, 120, 8, 64, 1102)]
    frames = [synth.make_frame(w, h, bd, q, seed=s) for w, h, bd, q, s in specs]
    damping, lambdas = [5, 4, 6], [64 * 256, 512 * 256, 4096 * 256]
    nb = sum(f.params.shape[0] * f.params.shape[1] for f in frames)
    ids = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    dl = torch.zeros(nb * 64, dtype=torch.int64, device="cuda")
    dc = torch.zeros(nb * 64, dtype=torch.int64, device="cuda")
    ctx.set_search_metric("eq14")
    ctx.set_search_refine(passes)
    try:
        res = cdef.cdef_search_strengths(ctx, [cdef.frame_from_numpy(f.rec, f.bitdepth) for f in frames],
                                         [cdef.frame_from_numpy(f.src, f.bitdepth) for f in frames],
                                         damping, lambdas, ids, dl, dc)
    finally:
        ctx.set_search_metric("sse")
        ctx.set_search_refine(0)
    assert ctx.status() == 0
    o0 = 0
    for f, r, d, lam in zip(frames, res, damping, lambdas):
        b = f.params.shape[0] * f.params.shape[1]
        gl = dl[o0 * 64:(o0 + b) * 64].cpu().numpy().reshape(b, 64)
        gc = dc[o0 * 64:(o0 + b) * 64].cpu().numpy().reshape(b, 64)
        el, ec = ref.distortion_eq14(f.rec, f.src, f.bitdepth, d)
        nl, nc = _eq14_term_counts(f.width, f.height)
        _assert_eq14_tables_close(gl, el, nl)
        _assert_eq14_tables_close(gc, ec, nc)
        o = ref.select_presets_general(gl, gc, 64, None, lam, passes)
        assert r["npresets"] == o["npresets"] and r["cost"] == o["cost"]
        assert ([cdef.preset_index(p) for p in r["presets"][:r["npresets"]]] ==
                [int(t) for t in o["presets"][:o["npresets"]]])
        assert np.array_equal(ids[o0:o0 + b].cpu().numpy(), o["block_ids"])
        o0 += b


def test_search_metric_rejections(cdef, ctx):
    assert ctx._lib.cdef_ctx_set_search_metric(ctx.handle, 2) != 0


@pytest.mark.parametrize("passes", [0, 2])
def test_search_eq14_coded_parity(cdef, ctx, ref, passes):
    """Eq. 14 over the 128 combinations (section 5 with section 4's skip
    semantics): 8/10-bit 4:2:0, 4:4:4 and 12-bit frames with coded-residual
    maps (one filter block without residual) in one call; tables and
    skipped flags within the precision bound of / equal to the oracle's,
    presets, N, J and ids exactly the oracle's selection on the GPU's
    tables."""
    from paper_1602_05975_gb300 import synth
    specs = [(420, 200, 136, 8, 1180), (444, 136, 72, 10, 1181), (420, 136, 72, 12, 1182),
             (420, 192, 128, 10, 1183)]
    rng = np.random.default_rng(1184)
    frames, maps = [], []
    for fmt, w, h, bd, sd in specs:
        frames.append(synth.make_frame(w, h, bd, 32, seed=sd, chroma=fmt))
        m = (rng.random((h // 8, w // 8)) < 0.55).astype(np.uint8)
        m[:8, 8:16] = 0
        maps.append(m)
    damping, lambdas = [5, 4, 6, 3], [64 << 8, 512 << 8, 4096 << 8, 900 << 8]
    nb = sum(f.params.shape[0] * f.params.shape[1] for f in frames)
    ids = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    dl = torch.full((nb * 128,), -1, dtype=torch.int64, device="cuda")
    dc = torch.full((nb * 128,), -1, dtype=torch.int64, device="cuda")
    ctx.set_search_metric("eq14")
    ctx.set_search_refine(passes)
    try:
        res = cdef.cdef_search_strengths_coded(
            ctx, [cdef.frame_from_numpy(f.rec, f.bitdepth) for f in frames],
            [cdef.frame_from_numpy(f.src, f.bitdepth) for f in frames],
            [torch.from_numpy(m.reshape(-1)).cuda() for m in maps], damping, lambdas, ids, dl, dc)
    finally:
        ctx.set_search_metric("sse")
        ctx.set_search_refine(0)
    assert ctx.status() == 0
    o0 = 0
    for f, sp, m, r, d, lam in zip(frames, specs, maps, res, damping, lambdas):
        b = f.params.shape[0] * f.params.shape[1]
        gl = dl[o0 * 128:(o0 + b) * 128].cpu().numpy().reshape(b, 128)
        gc = dc[o0 * 128:(o0 + b) * 128].cpu().numpy().reshape(b, 128)
        el, ec, sk = ref.distortion_eq14_coded_format(f.rec, f.src, f.bitdepth, d, sp[0], m)
        nl, nc = _eq14_term_counts(f.width, f.height, sp[0])
        _assert_eq14_tables_close(gl, el, nl)
        _assert_eq14_tables_close(gc, ec, nc)
        assert sk[1] == 1
        o = ref.select_presets_general(gl, gc, 128, sk, lam, passes)
        assert r["npresets"] == o["npresets"] and r["cost"] == o["cost"]
        assert [cdef.preset_index_coded(p) for p in r["presets"][:r["npresets"]]] == \
            [int(t) for t in o["presets"][:o["npresets"]]]
        assert np.array_equal(ids[o0:o0 + b].cpu().numpy(), o["block_ids"])
        o0 += b


@pytest.mark.gpu
def test_search_stage_timing(cdef, ctx):
    """Stage events in the search graph: positive stage times, results equal
    with and without them, and no times before a timed search."""
    from paper_1602_05975_gb300 import synth
    frames = [synth.make_frame(w, h, 8, 32, seed=s) for w, h, s in ((192, 128, 1120), (136, 72, 1121))]
    recs = [cdef.frame_from_numpy(f.rec, 8) for f in frames]
    srcs = [cdef.frame_from_numpy(f.src, 8) for f in frames]
    nb = sum(f.params.shape[0] * f.params.shape[1] for f in frames)

    def run():
        ids = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        dl = torch.zeros(nb * 64, dtype=torch.int64, device="cuda")
        dc = torch.zeros(nb * 64, dtype=torch.int64, device="cuda")
        res = cdef.cdef_search_strengths(ctx, recs, srcs, [5, 4], [256, 1024], ids, dl, dc)
        return res, ids.cpu(), dl.cpu(), dc.cpu()

    plain = run()
    ctx.set_stage_timing(True)
    try:
        with pytest.raises(cdef.CdefError):
            ctx.stage_times()
        for metric in ("sse", "eq14"):
            ctx.set_search_metric(metric)
            timed = run()
            t_dist, t_pre = ctx.stage_times()
            assert t_dist > 0 and t_pre > 0
            if metric == "sse":
                assert timed[0] == plain[0]
                assert all(torch.equal(a, b) for a, b in zip(timed[1:], plain[1:]))
    finally:
        ctx.set_search_metric("sse")
        ctx.set_stage_timing(False)
    assert ctx.status() == 0
    assert run()[0] == plain[0]


@pytest.mark.gpu
@pytest.mark.parametrize("variant,passes", [("sse", 0), ("sse", 3), ("eq14", 2), ("coded", 0),
                                            ("coded", 2)])
def test_search_subset_parity(cdef, ctx, ref, variant, passes):
    """Section 5's low-complexity search (reading R26): tables of allowed
    pairs equal the oracle's, the others are 0; presets, N, J and ids equal
    the oracle's selection over the subset, for every launch configuration."""
    from paper_1602_05975_gb300 import synth
    specs = [(200, 136, 8, 16, 1130), (136, 72, 10, 32, 1131), (192, 128, 8, 64, 1132)]
    frames = [synth.make_frame(w, h, bd, q, seed=s) for w, h, bd, q, s in specs]
    rng = np.random.default_rng(1133)
    lq = sorted(set(rng.integers(0, 64, 12).tolist()) | {0})
    cq = sorted(set(rng.integers(0, 64, 6).tolist()))
    lmask = sum(1 << q for q in lq)
    cmask = sum(1 << q for q in cq)
    width = 128 if variant == "coded" else 64
    maps = []
    if variant == "coded":
        for f in frames:
            m = (rng.random((f.height // 8, f.width // 8)) < 0.6).astype(np.uint8)
            m[:8, :8] = 0
            maps.append(m)
    damping, lambdas = [5, 4, 6], [64, 512, 4096]
    nb = sum(f.params.shape[0] * f.params.shape[1] for f in frames)
    recs = [cdef.frame_from_numpy(f.rec, f.bitdepth) for f in frames]
    srcs = [cdef.frame_from_numpy(f.src, f.bitdepth) for f in frames]
    # (groups, CTAs per SM, preset kernel)
    configs = [(0, 0, 0), (0, 0, 1)] if variant == "eq14" else [(0, 0, 0), (1, 2, 0), (4, 2, 0),
                                                                 (0, 0, 1)]
    ctx.set_search_subset(lmask, cmask)
    ctx.set_search_refine(passes)
    if variant == "eq14":
        ctx.set_search_metric("eq14")
    try:
        for groups, per_sm, grid in configs:
            ctx.set_tuning(groups, per_sm, preset_kernel=grid)
            ids = torch.zeros(nb, dtype=torch.uint8, device="cuda")
            dl = torch.full((nb * width,), -1, dtype=torch.int64, device="cuda")
            dc = torch.full((nb * width,), -1, dtype=torch.int64, device="cuda")
            if variant == "coded":
                res = cdef.cdef_search_strengths_coded(
                    ctx, recs, srcs, [torch.from_numpy(m.reshape(-1)).cuda() for m in maps],
                    damping, lambdas, ids, dl, dc)
            else:
                res = cdef.cdef_search_strengths(ctx, recs, srcs, damping, lambdas, ids, dl, dc)
            assert ctx.status() == 0
            o0 = 0
            for i, (f, r, d, lam) in enumerate(zip(frames, res, damping, lambdas)):
                b = f.params.shape[0] * f.params.shape[1]
                o = ref.search_strengths_subset(f.rec, f.src, f.bitdepth, d, lam, lmask, cmask,
                                                passes, maps[i] if maps else None, variant)
                gl = dl[o0 * width:(o0 + b) * width].cpu().numpy().reshape(b, width)
                gc = dc[o0 * width:(o0 + b) * width].cpu().numpy().reshape(b, width)
                cols_l = np.array([((lmask >> (q % 64)) & 1) == 1 for q in range(width)])
                cols_c = np.array([((cmask >> (q % 64)) & 1) == 1 for q in range(width)])
                if variant == "eq14":
                    # tables within the precision bound; the selection is
                    # the oracle's on the GPU's own tables
                    nl, nc = _eq14_term_counts(f.width, f.height)
                    _assert_eq14_tables_close(gl, o["dist_luma"], nl, cols_l)
                    _assert_eq14_tables_close(gc, o["dist_chroma"], nc, cols_c)
                    o = ref.select_presets_subset(gl, gc, 64, None, lmask, cmask, lam, passes)
                else:
                    assert np.array_equal(gl[:, cols_l], o["dist_luma"][:, cols_l])
                    assert np.array_equal(gc[:, cols_c], o["dist_chroma"][:, cols_c])
                assert (gl[:, ~cols_l] == 0).all() and (gc[:, ~cols_c] == 0).all()
                assert r["npresets"] == o["npresets"] and r["cost"] == o["cost"]
                idx = cdef.preset_index_coded if variant == "coded" else cdef.preset_index
                assert [idx(p) for p in r["presets"][:r["npresets"]]] == \
                    [int(t) for t in o["presets"][:o["npresets"]]]
                assert np.array_equal(ids[o0:o0 + b].cpu().numpy(), o["block_ids"])
                o0 += b
    finally:
        ctx.set_tuning(0, 0)
        ctx.set_search_refine(0)
        ctx.set_search_metric("sse")
        ctx.set_search_subset()


@pytest.mark.gpu
def test_search_subset_rejections(cdef, ctx):
    assert ctx._lib.cdef_ctx_set_search_subset(ctx.handle, 0, 1) != 0
    assert ctx._lib.cdef_ctx_set_search_subset(ctx.handle, 1, 0) != 0


def _format_search_frame(cdef, fmt, w, h, bd, seed):
    """A (rec, src) pair of chroma format `fmt`: the synthetic recipe at the
    format's chroma resolution; the source chroma planes near the decoded
    ones."""
    from paper_1602_05975_gb300 import synth
    f = synth.make_frame(w, h, bd, 32, seed=seed, chroma=fmt)
    return f, f.rec, f.src


@pytest.mark.gpu
@pytest.mark.parametrize("passes,grid", [(0, 0), (2, 0), (2, 1)])
def test_search_formats_parity(cdef, ctx, ref, passes, grid):
    """Section 5 over 4:4:4, 4:2:2 and 12-bit frames (reading R25), mixed
    with an 8-bit 4:2:0 frame in one call: tables, presets, N, J and ids
    equal the oracle's."""
    specs = [(444, 136, 72, 8, 1140), (422, 200, 136, 10, 1141), (420, 136, 72, 12, 1142),
             (420, 192, 128, 8, 1143), (444, 64, 64, 10, 1144)]
    frames = [_format_search_frame(cdef, *sp) for sp in specs]
    damping, lambdas = [5, 4, 6, 3, 5], [64, 512, 4096, 900, 0]
    nb = sum(f.params.shape[0] * f.params.shape[1] for f, _, _ in frames)
    ids = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    dl = torch.full((nb * 64,), -1, dtype=torch.int64, device="cuda")
    dc = torch.full((nb * 64,), -1, dtype=torch.int64, device="cuda")
    ctx.set_search_refine(passes)
    ctx.set_tuning(0, 0, preset_kernel=grid)
    try:
        res = cdef.cdef_search_strengths(ctx, [cdef.frame_from_numpy(r, f.bitdepth) for f, r, _ in frames],
                                         [cdef.frame_from_numpy(s_, f.bitdepth) for f, _, s_ in frames],
                                         damping, lambdas, ids, dl, dc)
    finally:
        ctx.set_tuning(0, 0)
        ctx.set_search_refine(0)
    assert ctx.status() == 0
    o0 = 0
    for (f, r, s_), sp, rr, d, lam in zip(frames, specs, res, damping, lambdas):
        b = f.params.shape[0] * f.params.shape[1]
        o = ref.search_strengths_format(r, s_, f.bitdepth, d, lam, sp[0], passes)
        assert np.array_equal(dl[o0 * 64:(o0 + b) * 64].cpu().numpy().reshape(b, 64), o["dist_luma"])
        assert np.array_equal(dc[o0 * 64:(o0 + b) * 64].cpu().numpy().reshape(b, 64), o["dist_chroma"])
        assert rr["npresets"] == o["npresets"] and rr["cost"] == o["cost"]
        assert [cdef.preset_index(p) for p in rr["presets"][:rr["npresets"]]] == \
            [int(t) for t in o["presets"][:o["npresets"]]]
        assert np.array_equal(ids[o0:o0 + b].cpu().numpy(), o["block_ids"])
        o0 += b


@pytest.mark.gpu
def test_search_formats_subset_and_rejections(cdef, ctx, ref):
    """The low-complexity subset in the wide tables."""
    f, r, s_ = _format_search_frame(cdef, 444, 136, 72, 8, 1150)
    rec, src = cdef.frame_from_numpy(r, 8), cdef.frame_from_numpy(s_, 8)
    nb = f.params.shape[0] * f.params.shape[1]
    lmask, cmask = sum(1 << q for q in (0, 5, 9, 33, 62)), sum(1 << q for q in (1, 2, 40))
    ids = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    dl = torch.zeros(nb * 64, dtype=torch.int64, device="cuda")
    dc = torch.zeros(nb * 64, dtype=torch.int64, device="cuda")
    ctx.set_search_subset(lmask, cmask)
    try:
        res = cdef.cdef_search_strengths(ctx, [rec], [src], [5], [300], ids, dl, dc)
    finally:
        ctx.set_search_subset()
    dlo, dco = ref.distortion_format(r, s_, 8, 5, 444)
    o = ref.select_presets_subset(dlo, dco, 64, None, lmask, cmask, 300)
    gl = dl.cpu().numpy().reshape(nb, 64)
    gc = dc.cpu().numpy().reshape(nb, 64)
    cl = np.array([(lmask >> q) & 1 for q in range(64)], bool)
    cc = np.array([(cmask >> q) & 1 for q in range(64)], bool)
    assert np.array_equal(gl[:, cl], dlo[:, cl]) and (gl[:, ~cl] == 0).all()
    assert np.array_equal(gc[:, cc], dco[:, cc]) and (gc[:, ~cc] == 0).all()
    assert res[0]["cost"] == o["cost"] and res[0]["npresets"] == o["npresets"]
    assert ctx.status() == 0


@pytest.mark.gpu
@pytest.mark.parametrize("passes,grid", [(0, 0), (2, 0), (2, 1)])
def test_search_444_planes_parity(cdef, ctx, ref, passes, grid):
    """8/10-bit 4:4:4 calls (every frame 4:4:4: one plane per work unit in
    the packed layout, U and V added into the chroma table): ragged, 8x8 and
    one-block frames; tables, presets, N, J and ids equal the oracle's."""
    specs = [(444, 136, 72, 8, 1160), (444, 64, 64, 10, 1161), (444, 200, 136, 8, 1162),
             (444, 8, 8, 10, 1163), (444, 72, 40, 8, 1164)]
    frames = [_format_search_frame(cdef, *sp) for sp in specs]
    damping, lambdas = [5, 3, 6, 4, 5], [64, 0, 4096, 900, 300]
    nb = sum(f.params.shape[0] * f.params.shape[1] for f, _, _ in frames)
    ids = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    dl = torch.full((nb * 64,), -1, dtype=torch.int64, device="cuda")
    dc = torch.full((nb * 64,), -1, dtype=torch.int64, device="cuda")
    ctx.set_search_refine(passes)
    ctx.set_tuning(0, 0, preset_kernel=grid)
    try:
        res = cdef.cdef_search_strengths(ctx, [cdef.frame_from_numpy(r, f.bitdepth) for f, r, _ in frames],
                                         [cdef.frame_from_numpy(s_, f.bitdepth) for f, _, s_ in frames],
                                         damping, lambdas, ids, dl, dc)
    finally:
        ctx.set_tuning(0, 0)
        ctx.set_search_refine(0)
    assert ctx.status() == 0
    o0 = 0
    for (f, r, s_), sp, rr, d, lam in zip(frames, specs, res, damping, lambdas):
        b = f.params.shape[0] * f.params.shape[1]
        o = ref.search_strengths_format(r, s_, f.bitdepth, d, lam, sp[0], passes)
        assert np.array_equal(dl[o0 * 64:(o0 + b) * 64].cpu().numpy().reshape(b, 64), o["dist_luma"])
        assert np.array_equal(dc[o0 * 64:(o0 + b) * 64].cpu().numpy().reshape(b, 64), o["dist_chroma"])
        assert rr["npresets"] == o["npresets"] and rr["cost"] == o["cost"]
        assert [cdef.preset_index(p) for p in rr["presets"][:rr["npresets"]]] == \
            [int(t) for t in o["presets"][:o["npresets"]]]
        assert np.array_equal(ids[o0:o0 + b].cpu().numpy(), o["block_ids"])
        o0 += b


@pytest.mark.parametrize("passes", [0, 2])
def test_search_eq14_formats_parity(cdef, ctx, ref, passes):
    """Eq. 14 tables of 4:4:4, 4:2:2 and 12-bit frames (and an 8-bit 4:2:0
    frame in the same call, which then takes the same 32-bit path) within
    the precision bound of the double-precision oracle's; presets, N, J and
    ids exactly the oracle's selection on the GPU's own tables."""
    specs = [(444, 136, 72, 8, 1190), (422, 200, 136, 10, 1191), (420, 136, 72, 12, 1192),
             (420, 192, 128, 8, 1193), (444, 64, 64, 10, 1194)]
    frames = [_format_search_frame(cdef, *sp) for sp in specs]
    damping, lambdas = [5, 4, 6, 3, 5], [64 << 8, 512 << 8, 4096 << 8, 900 << 8, 0]
    nb = sum(f.params.shape[0] * f.params.shape[1] for f, _, _ in frames)
    ids = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    dl = torch.full((nb * 64,), -1, dtype=torch.int64, device="cuda")
    dc = torch.full((nb * 64,), -1, dtype=torch.int64, device="cuda")
    ctx.set_search_metric("eq14")
    ctx.set_search_refine(passes)
    try:
        res = cdef.cdef_search_strengths(ctx, [cdef.frame_from_numpy(r, f.bitdepth) for f, r, _ in frames],
                                         [cdef.frame_from_numpy(s_, f.bitdepth) for f, _, s_ in frames],
                                         damping, lambdas, ids, dl, dc)
    finally:
        ctx.set_search_metric("sse")
        ctx.set_search_refine(0)
    assert ctx.status() == 0
    o0 = 0
    for (f, r, s_), sp, rr, d, lam in zip(frames, specs, res, damping, lambdas):
        b = f.params.shape[0] * f.params.shape[1]
        gl = dl[o0 * 64:(o0 + b) * 64].cpu().numpy().reshape(b, 64)
        gc = dc[o0 * 64:(o0 + b) * 64].cpu().numpy().reshape(b, 64)
        el, ec = ref.distortion_eq14_format(r, s_, f.bitdepth, d, sp[0])
        nl, nc = _eq14_term_counts(f.width, f.height, sp[0])
        _assert_eq14_tables_close(gl, el, nl)
        _assert_eq14_tables_close(gc, ec, nc)
        if sp[0] == 422:
            assert (gc == gc[:, :1]).all()          # chroma not filtered: one value per block
        o = ref.select_presets_general(gl, gc, 64, None, lam, passes)
        assert rr["npresets"] == o["npresets"] and rr["cost"] == o["cost"]
        assert [cdef.preset_index(p) for p in rr["presets"][:rr["npresets"]]] == \
            [int(t) for t in o["presets"][:o["npresets"]]]
        assert np.array_equal(ids[o0:o0 + b].cpu().numpy(), o["block_ids"])
        o0 += b


@pytest.mark.gpu
@pytest.mark.parametrize("passes,subset", [(0, False), (2, False), (0, True)])
def test_search_444_planes_eq14_parity(cdef, ctx, ref, passes, subset):
    """Eq. 14 over 8/10-bit 4:4:4 calls (one plane per work unit, each plane's
    8x8 values in the luma layout, U and V added into the chroma table):
    tables within the precision bound of the double-precision oracle's;
    presets, N, J and ids exactly the oracle's selection on the GPU's own
    tables; with a subset, the entries outside it are 0."""
    specs = [(444, 136, 72, 8, 1200), (444, 64, 64, 10, 1201), (444, 72, 40, 8, 1202)]
    frames = [_format_search_frame(cdef, *sp) for sp in specs]
    damping, lambdas = [5, 3, 6], [64 << 8, 0, 900 << 8]
    nb = sum(f.params.shape[0] * f.params.shape[1] for f, _, _ in frames)
    ids = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    dl = torch.full((nb * 64,), -1, dtype=torch.int64, device="cuda")
    dc = torch.full((nb * 64,), -1, dtype=torch.int64, device="cuda")
    lmask, cmask = sum(1 << q for q in (0, 5, 9, 33, 62)), sum(1 << q for q in (1, 2, 40, 63))
    ctx.set_search_metric("eq14")
    ctx.set_search_refine(passes)
    if subset:
        ctx.set_search_subset(lmask, cmask)
    try:
        res = cdef.cdef_search_strengths(ctx, [cdef.frame_from_numpy(r, f.bitdepth) for f, r, _ in frames],
                                         [cdef.frame_from_numpy(s_, f.bitdepth) for f, _, s_ in frames],
                                         damping, lambdas, ids, dl, dc)
    finally:
        ctx.set_search_metric("sse")
        ctx.set_search_refine(0)
        ctx.set_search_subset()
    assert ctx.status() == 0
    cl = np.array([(lmask >> q) & 1 for q in range(64)], bool) if subset else np.ones(64, bool)
    cc = np.array([(cmask >> q) & 1 for q in range(64)], bool) if subset else np.ones(64, bool)
    o0 = 0
    for (f, r, s_), sp, rr, d, lam in zip(frames, specs, res, damping, lambdas):
        b = f.params.shape[0] * f.params.shape[1]
        gl = dl[o0 * 64:(o0 + b) * 64].cpu().numpy().reshape(b, 64)
        gc = dc[o0 * 64:(o0 + b) * 64].cpu().numpy().reshape(b, 64)
        el, ec = ref.distortion_eq14_format(r, s_, f.bitdepth, d, 444)
        nl, nc = _eq14_term_counts(f.width, f.height, 444)
        _assert_eq14_tables_close(gl, el, nl, cols=np.flatnonzero(cl))
        _assert_eq14_tables_close(gc, ec, nc, cols=np.flatnonzero(cc))
        assert (gl[:, ~cl] == 0).all() and (gc[:, ~cc] == 0).all()
        if subset:
            o = ref.select_presets_subset(gl, gc, 64, None, lmask, cmask, lam, passes)
        else:
            o = ref.select_presets_general(gl, gc, 64, None, lam, passes)
        assert rr["npresets"] == o["npresets"] and rr["cost"] == o["cost"]
        if not subset:
            assert [cdef.preset_index(p) for p in rr["presets"][:rr["npresets"]]] == \
                [int(t) for t in o["presets"][:o["npresets"]]]
            assert np.array_equal(ids[o0:o0 + b].cpu().numpy(), o["block_ids"])
        o0 += b


def test_filter_frames_maximum_batch(cdef, ctx, ref):
    """48 frames (the batch limit) of mixed sizes and bit depths in one
    launch each equal the oracle; 49 frames are refused."""
    from paper_1602_05975_gb300 import synth
    rng = np.random.default_rng(1160)
    sizes = [(64, 64), (136, 72), (72, 136), (200, 40), (8, 8), (128, 64)]
    frames, ins, outs, prms = [], [], [], []
    for i in range(48):
        w, h = sizes[i % len(sizes)]
        bd = (8, 10, 12)[i % 3]
        f = synth.make_frame(w, h, bd, 32, seed=1160 + i)
        frames.append(f)
        ins.append(cdef.frame_from_numpy(f.rec, bd))
        outs.append(cdef.alloc_frame(w, h, bd, fill=0))
        prms.append(cdef.params_tensor(f.params))
    cdef.cdef_filter_frames(ctx, ins, prms, outs)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    for f, o in zip(frames, outs):
        _assert_frames_equal(o.to_numpy(), ref.filter_frame(*f.rec, f.bitdepth, f.params))
    with pytest.raises(cdef.CdefError):
        cdef.cdef_filter_frames(ctx, ins + ins[:1], prms + prms[:1], outs + [cdef.alloc_frame(64, 64, 8)])


@pytest.mark.parametrize("sizes,bd", [
    ([(2048, 2176)], 10),                   # 1088 blocks: 64-bit minima, tables staged twice a step
    ([(7680, 4352), (256, 256)], 8),        # 8160 blocks (staged 4 times) with a resident frame
    ([(8192, 8320)], 8),                    # 16640 blocks: beyond the cluster kernel's state
])
def test_search_large_periodic_frames(cdef, ctx, ref, sizes, bd):
    """The search on frames far larger than the oracle's search can take,
    through tables known by construction (`periodic_frames.py`): the
    tables, presets, N, J and every block's id."""
    from periodic_frames import periodic_search_case
    cases = periodic_search_case(ref, sizes, bd, seed=6100 + bd)
    recs = [cdef.frame_from_numpy(c["rec"], bd) for c in cases]
    srcs = [cdef.frame_from_numpy(c["src"], bd) for c in cases]
    nbs = [c["dl"].shape[0] for c in cases]
    tot = sum(nbs)
    ids = torch.zeros(tot, dtype=torch.uint8, device="cuda")
    dl = torch.zeros(tot * 64, dtype=torch.int64, device="cuda")
    dc = torch.zeros(tot * 64, dtype=torch.int64, device="cuda")
    res = cdef.cdef_search_strengths(ctx, recs, srcs, [c["damping"] for c in cases],
                                     [c["lam"] for c in cases], ids, dl, dc)
    assert ctx.status() == 0
    dl, dc, ids = dl.cpu().numpy(), dc.cpu().numpy(), ids.cpu().numpy()
    off = 0
    for k, c in enumerate(cases):
        nb, o = nbs[k], c["exp"]
        assert np.array_equal(dl[off * 64:(off + nb) * 64].reshape(nb, 64), c["dl"])
        assert np.array_equal(dc[off * 64:(off + nb) * 64].reshape(nb, 64), c["dc"])
        assert res[k]["npresets"] == o["npresets"]
        assert res[k]["cost"] == o["cost"]
        assert [cdef.preset_index(p) for p in res[k]["presets"]] == list(o["presets"])
        assert np.array_equal(ids[off:off + nb], o["block_ids"])
        off += nb

@pytest.mark.parametrize("sizes,bd,grid", [
    ([(2048, 2176)], 10, 0),                # 1088 blocks: 64-bit minima, 128-wide rows staged
    ([(4096, 2176), (256, 256)], 8, 0),     # 2176 blocks (staged) with a resident frame
    ([(2048, 2176)], 8, 1),                 # the grid-wide preset kernel
])
def test_search_coded_large_periodic_frames(cdef, ctx, ref, sizes, bd, grid):
    """The 128-combination search (skipped filter blocks) on frames far
    larger than the oracle's search can take, through tables known by
    construction (`periodic_frames.py`): tables, skip-aware presets, N, J
    and every block's id."""
    from periodic_frames import periodic_search_case
    cases = periodic_search_case(ref, sizes, bd, seed=6200 + bd, coded=True)
    recs = [cdef.frame_from_numpy(c["rec"], bd) for c in cases]
    srcs = [cdef.frame_from_numpy(c["src"], bd) for c in cases]
    maps = [torch.from_numpy(c["coded"].reshape(-1)).cuda() for c in cases]
    nbs = [c["dl"].shape[0] for c in cases]
    tot = sum(nbs)
    ids = torch.zeros(tot, dtype=torch.uint8, device="cuda")
    dl = torch.zeros(tot * 128, dtype=torch.int64, device="cuda")
    dc = torch.zeros(tot * 128, dtype=torch.int64, device="cuda")
    ctx.set_tuning(0, 0, preset_kernel=grid)
    try:
        res = cdef.cdef_search_strengths_coded(ctx, recs, srcs, maps, [c["damping"] for c in cases],
                                               [c["lam"] for c in cases], ids, dl, dc)
    finally:
        ctx.set_tuning(0, 0)
    assert ctx.status() == 0
    dl, dc, ids = dl.cpu().numpy(), dc.cpu().numpy(), ids.cpu().numpy()
    off = 0
    for k, c in enumerate(cases):
        nb, o = nbs[k], c["exp"]
        assert np.array_equal(dl[off * 128:(off + nb) * 128].reshape(nb, 128), c["dl"])
        assert np.array_equal(dc[off * 128:(off + nb) * 128].reshape(nb, 128), c["dc"])
        assert res[k]["npresets"] == o["npresets"]
        assert res[k]["cost"] == o["cost"]
        assert ([cdef.preset_index_coded(p) for p in res[k]["presets"][:o["npresets"]]] ==
                [int(t) for t in o["presets"][:o["npresets"]]])
        assert np.array_equal(ids[off:off + nb], o["block_ids"])
        off += nb


def test_search_maximum_batch(cdef, ctx, ref):
    """48 frames in one search call equal 48 oracle searches; 49 are refused."""
    from paper_1602_05975_gb300 import synth
    sizes = [(64, 64), (136, 72), (72, 136), (128, 64)]
    frames = [synth.make_frame(*sizes[i % 4], (8, 10)[i % 2], None, seed=1170 + i) for i in range(48)]
    recs = [cdef.frame_from_numpy(f.rec, f.bitdepth) for f in frames]
    srcs = [cdef.frame_from_numpy(f.src, f.bitdepth) for f in frames]
    nb = sum(f.params.shape[0] * f.params.shape[1] for f in frames)
    damping = [3 + i % 4 for i in range(48)]
    lambdas = [f.q * f.q for f in frames]
    ids = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    dl = torch.zeros(nb * 64, dtype=torch.int64, device="cuda")
    dc = torch.zeros(nb * 64, dtype=torch.int64, device="cuda")
    res = cdef.cdef_search_strengths(ctx, recs, srcs, damping, lambdas, ids, dl, dc)
    assert ctx.status() == 0
    o0 = 0
    for f, r, d, lam in zip(frames, res, damping, lambdas):
        b = f.params.shape[0] * f.params.shape[1]
        o = ref.search_strengths(f.rec, f.src, f.bitdepth, d, lam)
        assert np.array_equal(dl[o0 * 64:(o0 + b) * 64].cpu().numpy().reshape(b, 64), o["dist_luma"])
        assert np.array_equal(dc[o0 * 64:(o0 + b) * 64].cpu().numpy().reshape(b, 64), o["dist_chroma"])
        assert r["npresets"] == o["npresets"] and r["cost"] == o["cost"]
        assert np.array_equal(ids[o0:o0 + b].cpu().numpy(), o["block_ids"])
        o0 += b
    with pytest.raises(cdef.CdefError):
        cdef.cdef_search_strengths(ctx, recs + recs[:1], srcs + srcs[:1], damping + [4],
                                   lambdas + [16], ids)


@pytest.mark.gpu
def test_search_coded_formats_parity(cdef, ctx, ref):
    """The 128-combination search over 4:4:4, 4:2:2 and 12-bit frames (with
    a 4:2:0 frame in the same call, so the whole call takes the 32-bit
    path): tables, skipped blocks, presets, N, J and ids equal the oracle's."""
    specs = [(444, 136, 72, 8, 1180), (422, 200, 136, 10, 1181), (420, 136, 72, 12, 1182),
             (420, 128, 64, 8, 1183)]
    frames = [_format_search_frame(cdef, *sp) for sp in specs]
    rng = np.random.default_rng(1184)
    maps = []
    for f, _, _ in frames:
        m = (rng.random((f.height // 8, f.width // 8)) < 0.5).astype(np.uint8)
        m[:8, :8] = 0                                       # first filter block: no residual
        maps.append(m)
    damping, lambdas = [5, 4, 3, 6], [64, 512, 4096, 0]
    nb = sum(f.params.shape[0] * f.params.shape[1] for f, _, _ in frames)
    ids = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    dl = torch.full((nb * 128,), -1, dtype=torch.int64, device="cuda")
    dc = torch.full((nb * 128,), -1, dtype=torch.int64, device="cuda")
    ctx.set_search_refine(2)
    try:
        res = cdef.cdef_search_strengths_coded(
            ctx, [cdef.frame_from_numpy(r, f.bitdepth) for f, r, _ in frames],
            [cdef.frame_from_numpy(s_, f.bitdepth) for f, _, s_ in frames],
            [torch.from_numpy(m.reshape(-1)).cuda() for m in maps], damping, lambdas, ids, dl, dc)
    finally:
        ctx.set_search_refine(0)
    assert ctx.status() == 0
    o0 = 0
    for (f, r, s_), sp, m, rr, d, lam in zip(frames, specs, maps, res, damping, lambdas):
        b = f.params.shape[0] * f.params.shape[1]
        o = ref.search_strengths_coded_format(r, s_, f.bitdepth, d, lam, sp[0], m, 2)
        assert np.array_equal(dl[o0 * 128:(o0 + b) * 128].cpu().numpy().reshape(b, 128),
                              o["dist_luma"])
        assert np.array_equal(dc[o0 * 128:(o0 + b) * 128].cpu().numpy().reshape(b, 128),
                              o["dist_chroma"])
        assert rr["npresets"] == o["npresets"] and rr["cost"] == o["cost"]
        assert [cdef.preset_index_coded(p) for p in rr["presets"][:rr["npresets"]]] == \
            [int(t) for t in o["presets"][:o["npresets"]]]
        assert np.array_equal(ids[o0:o0 + b].cpu().numpy(), o["block_ids"])
        o0 += b


@pytest.mark.gpu
@pytest.mark.parametrize("passes,grid", [(0, 0), (2, 1)])
def test_search_444_planes_coded_parity(cdef, ctx, ref, passes, grid):
    """The 128-combination search over 8/10-bit 4:4:4 calls (one plane per
    work unit, U and V added into the chroma table, both skip-bit halves):
    tables, skipped blocks, presets, N, J and ids equal the oracle's; a
    filter block without coded residual and ragged frames included."""
    specs = [(444, 136, 72, 8, 1190), (444, 64, 64, 10, 1191), (444, 200, 136, 8, 1192),
             (444, 72, 40, 10, 1193)]
    frames = [_format_search_frame(cdef, *sp) for sp in specs]
    rng = np.random.default_rng(1194)
    maps = []
    for f, _, _ in frames:
        m = (rng.random((f.height // 8, f.width // 8)) < 0.5).astype(np.uint8)
        m[:8, :8] = 0                                       # first filter block: no residual
        maps.append(m)
    damping, lambdas = [5, 4, 3, 6], [64, 512, 4096, 0]
    nb = sum(f.params.shape[0] * f.params.shape[1] for f, _, _ in frames)
    ids = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    dl = torch.full((nb * 128,), -1, dtype=torch.int64, device="cuda")
    dc = torch.full((nb * 128,), -1, dtype=torch.int64, device="cuda")
    ctx.set_search_refine(passes)
    ctx.set_tuning(0, 0, preset_kernel=grid)
    try:
        res = cdef.cdef_search_strengths_coded(
            ctx, [cdef.frame_from_numpy(r, f.bitdepth) for f, r, _ in frames],
            [cdef.frame_from_numpy(s_, f.bitdepth) for f, _, s_ in frames],
            [torch.from_numpy(m.reshape(-1)).cuda() for m in maps], damping, lambdas, ids, dl, dc)
    finally:
        ctx.set_tuning(0, 0)
        ctx.set_search_refine(0)
    assert ctx.status() == 0
    o0 = 0
    for (f, r, s_), sp, m, rr, d, lam in zip(frames, specs, maps, res, damping, lambdas):
        b = f.params.shape[0] * f.params.shape[1]
        o = ref.search_strengths_coded_format(r, s_, f.bitdepth, d, lam, sp[0], m, passes)
        assert np.array_equal(dl[o0 * 128:(o0 + b) * 128].cpu().numpy().reshape(b, 128),
                              o["dist_luma"])
        assert np.array_equal(dc[o0 * 128:(o0 + b) * 128].cpu().numpy().reshape(b, 128),
                              o["dist_chroma"])
        assert rr["npresets"] == o["npresets"] and rr["cost"] == o["cost"]
        assert [cdef.preset_index_coded(p) for p in rr["presets"][:rr["npresets"]]] == \
            [int(t) for t in o["presets"][:o["npresets"]]]
        assert np.array_equal(ids[o0:o0 + b].cpu().numpy(), o["block_ids"])
        o0 += b


@pytest.mark.parametrize("seed", range(6))
def test_filter_random_fuzz(cdef, ctx, ref, seed):
    """Random sizes (multiples of 8 from 8 to 264), bit depths, formats,
    strengths, skip bits and coded maps: every output sample equals the
    oracle's."""
    from paper_1602_05975_gb300 import synth
    rng = np.random.default_rng(5000 + seed)
    for _ in range(10):
        w, h = 8 * int(rng.integers(1, 34)), 8 * int(rng.integers(1, 34))
        bd = int(rng.choice([8, 10, 12]))
        fmt = int(rng.choice([420, 420, 422, 444]))
        f = synth.make_frame(w, h, bd, int(rng.choice([16, 32, 64])), seed=int(rng.integers(1 << 30)),
                             chroma=fmt)
        params = synth.random_params(rng, w, h)
        params[..., 5] = rng.integers(0, 4, params.shape[:2])
        coded = (rng.random((h // 8, w // 8)) < rng.random()).astype(np.uint8)
        inp = cdef.frame_from_numpy(f.rec, bd)
        out = cdef.alloc_frame(w, h, bd, fill=0, chroma=fmt)
        cdef.cdef_filter_frame_coded(ctx, inp, cdef.params_tensor(params),
                                     torch.from_numpy(coded.reshape(-1)).cuda(), out)
        torch.cuda.synchronize()
        exp = ref.filter_frame_format(*f.rec, bd, params, fmt, coded)
        _assert_frames_equal(out.to_numpy(), exp)
    assert ctx.status() == 0


@pytest.mark.parametrize("seed", range(4))
def test_search_random_fuzz(cdef, ctx, ref, seed):
    """Random mixed calls (sizes, bit depths, formats, damping, lambda, with
    or without coded-residual maps): tables, presets, N, J and ids equal
    the oracle's."""
    from paper_1602_05975_gb300 import synth
    rng = np.random.default_rng(6000 + seed)
    with_maps = seed % 2 == 1
    frames, maps = [], []
    for _ in range(5):
        w, h = 8 * int(rng.integers(1, 26)), 8 * int(rng.integers(1, 26))
        bd = int(rng.choice([8, 10] if seed < 2 else [8, 10, 12]))
        fmt = 420 if seed < 2 else int(rng.choice([420, 422, 444]))
        frames.append(synth.make_frame(w, h, bd, None, seed=int(rng.integers(1 << 30)), chroma=fmt))
        maps.append((rng.random((h // 8, w // 8)) < rng.random()).astype(np.uint8))
    damping = [int(d) for d in rng.integers(3, 7, len(frames))]
    lambdas = [int(l) for l in rng.integers(0, 5000, len(frames))]
    width = 128 if with_maps else 64
    nb = sum(f.params.shape[0] * f.params.shape[1] for f in frames)
    ids = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    dl = torch.full((nb * width,), -1, dtype=torch.int64, device="cuda")
    dc = torch.full((nb * width,), -1, dtype=torch.int64, device="cuda")
    recs = [cdef.frame_from_numpy(f.rec, f.bitdepth) for f in frames]
    srcs = [cdef.frame_from_numpy(f.src, f.bitdepth) for f in frames]
    if with_maps:
        res = cdef.cdef_search_strengths_coded(ctx, recs, srcs,
                                               [torch.from_numpy(m.reshape(-1)).cuda() for m in maps],
                                               damping, lambdas, ids, dl, dc)
    else:
        res = cdef.cdef_search_strengths(ctx, recs, srcs, damping, lambdas, ids, dl, dc)
    assert ctx.status() == 0
    o0 = 0
    for f, m, r, d, lam in zip(frames, maps, res, damping, lambdas):
        b = f.params.shape[0] * f.params.shape[1]
        fmt = {(f.width // 2, f.height // 2): 420, (f.width // 2, f.height): 422,
               (f.width, f.height): 444}[(f.rec[1].shape[1], f.rec[1].shape[0])]
        if with_maps:
            o = ref.search_strengths_coded_format(f.rec, f.src, f.bitdepth, d, lam, fmt, m)
            idx = cdef.preset_index_coded
        else:
            o = ref.search_strengths_format(f.rec, f.src, f.bitdepth, d, lam, fmt)
            idx = cdef.preset_index
        assert np.array_equal(dl[o0 * width:(o0 + b) * width].cpu().numpy().reshape(b, width),
                              o["dist_luma"])
        assert np.array_equal(dc[o0 * width:(o0 + b) * width].cpu().numpy().reshape(b, width),
                              o["dist_chroma"])
        assert r["npresets"] == o["npresets"] and r["cost"] == o["cost"]
        assert [idx(p) for p in r["presets"][:r["npresets"]]] == \
            [int(t) for t in o["presets"][:o["npresets"]]]
        assert np.array_equal(ids[o0:o0 + b].cpu().numpy(), o["block_ids"])
        o0 += b


@pytest.mark.parametrize("seed", range(4))
def test_search_444_random_fuzz(cdef, ctx, ref, seed):
    """Random all-4:4:4 calls (the packed plane units): sizes, 8/10-bit,
    damping, lambda, with or without coded-residual maps; tables, presets,
    N, J and ids equal the oracle's."""
    from paper_1602_05975_gb300 import synth
    rng = np.random.default_rng(6100 + seed)
    with_maps = seed % 2 == 1
    frames, maps = [], []
    for _ in range(4):
        w, h = 8 * int(rng.integers(1, 26)), 8 * int(rng.integers(1, 26))
        bd = int(rng.choice([8, 10]))
        frames.append(synth.make_frame(w, h, bd, None, seed=int(rng.integers(1 << 30)), chroma=444))
        maps.append((rng.random((h // 8, w // 8)) < rng.random()).astype(np.uint8))
    damping = [int(d) for d in rng.integers(3, 7, len(frames))]
    lambdas = [int(l) for l in rng.integers(0, 5000, len(frames))]
    width = 128 if with_maps else 64
    nb = sum(f.params.shape[0] * f.params.shape[1] for f in frames)
    ids = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    dl = torch.full((nb * width,), -1, dtype=torch.int64, device="cuda")
    dc = torch.full((nb * width,), -1, dtype=torch.int64, device="cuda")
    recs = [cdef.frame_from_numpy(f.rec, f.bitdepth) for f in frames]
    srcs = [cdef.frame_from_numpy(f.src, f.bitdepth) for f in frames]
    if with_maps:
        res = cdef.cdef_search_strengths_coded(ctx, recs, srcs,
                                               [torch.from_numpy(m.reshape(-1)).cuda() for m in maps],
                                               damping, lambdas, ids, dl, dc)
    else:
        res = cdef.cdef_search_strengths(ctx, recs, srcs, damping, lambdas, ids, dl, dc)
    assert ctx.status() == 0
    o0 = 0
    for f, m, r, d, lam in zip(frames, maps, res, damping, lambdas):
        b = f.params.shape[0] * f.params.shape[1]
        if with_maps:
            o = ref.search_strengths_coded_format(f.rec, f.src, f.bitdepth, d, lam, 444, m)
            idx = cdef.preset_index_coded
        else:
            o = ref.search_strengths_format(f.rec, f.src, f.bitdepth, d, lam, 444)
            idx = cdef.preset_index
        assert np.array_equal(dl[o0 * width:(o0 + b) * width].cpu().numpy().reshape(b, width),
                              o["dist_luma"])
        assert np.array_equal(dc[o0 * width:(o0 + b) * width].cpu().numpy().reshape(b, width),
                              o["dist_chroma"])
        assert r["npresets"] == o["npresets"] and r["cost"] == o["cost"]
        assert [idx(p) for p in r["presets"][:r["npresets"]]] == \
            [int(t) for t in o["presets"][:o["npresets"]]]
        assert np.array_equal(ids[o0:o0 + b].cpu().numpy(), o["block_ids"])
        o0 += b


@pytest.mark.parametrize("seed", range(3))
def test_filter_444_random_fuzz(cdef, ctx, ref, seed):
    """Random 8/10-bit 4:4:4 frames through the three-plane launch: sizes,
    strengths, damping, skip bits, with or without coded maps; every output
    sample equals the oracle's."""
    from paper_1602_05975_gb300 import synth
    rng = np.random.default_rng(6200 + seed)
    for _ in range(3):
        w, h = 8 * int(rng.integers(1, 30)), 8 * int(rng.integers(1, 30))
        bd = int(rng.choice([8, 10]))
        f = synth.make_frame(w, h, bd, None, seed=int(rng.integers(1 << 30)), chroma=444)
        params = synth.random_params(rng, w, h)
        params[..., 5] = rng.integers(0, 4, params.shape[:2])
        coded = (rng.random((h // 8, w // 8)) < rng.random()).astype(np.uint8) if seed % 2 else None
        inp = cdef.frame_from_numpy(f.rec, bd)
        out = cdef.alloc_frame(w, h, bd, fill=0, chroma=444)
        prm = cdef.params_tensor(params)
        if coded is not None:
            cdef.cdef_filter_frame_coded(ctx, inp, prm, torch.from_numpy(coded.reshape(-1)).cuda(), out)
        else:
            cdef.cdef_filter_frame(ctx, inp, prm, out)
        torch.cuda.synchronize()
        assert ctx.status() == 0
        _assert_frames_equal(out.to_numpy(), ref.filter_frame_format(*f.rec, bd, params, 444, coded))
