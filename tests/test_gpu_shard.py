"""The strength search split over devices, on one GPU.

cdef_search_tables computes section 5's tables of a band of filter-block
rows; cdef_preset_totals / cdef_preset_argmin / cdef_preset_assign are the
per-rank steps of the host-driven selection (shard.py).  Checked here:
band tables equal the oracle's rows of the whole frame; the three
reductions equal their definitions on random tables; and ranks emulated as
host threads on one GPU (each its own context, band and driver; the
all-reduce a host barrier that sums the ranks' tensors: no kernel waits on
another) select exactly the oracle's presets, N, J and ids.  Integer work:
tolerance zero (eq. 14 tables: the precision bound of the eq. 14 tests)."""
import threading

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ALL = (1 << 64) - 1


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


def _band_tables(cdef, ctx, frames, bands, width=64, coded=None):
    recs = [cdef.frame_from_numpy(f.rec, f.bitdepth) for f in frames]
    srcs = [cdef.frame_from_numpy(f.src, f.bitdepth) for f in frames]
    nb = sum(rn * -(-f.width // 64) for f, (r0, rn) in zip(frames, bands))
    dl = torch.full((max(nb, 1) * width,), -3, dtype=torch.int64, device="cuda")
    dc = torch.full((max(nb, 1) * width,), -3, dtype=torch.int64, device="cuda")
    sk = None if coded is None else torch.full((max(nb, 1),), 7, dtype=torch.uint8, device="cuda")
    cm = None if coded is None else [torch.from_numpy(c.reshape(-1)).cuda() for c in coded]
    cdef.cdef_search_tables(ctx, recs, srcs, [5] * len(frames), [b[0] for b in bands],
                            [b[1] for b in bands], dl, dc, cm, sk)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    out = (dl[:nb * width].cpu().numpy().reshape(nb, width),
           dc[:nb * width].cpu().numpy().reshape(nb, width))
    return out + ((sk[:nb].cpu().numpy(),) if sk is not None else ())


@pytest.mark.parametrize("kind", ["sse8", "sse10", "coded", "444", "12bit"])
def test_band_tables_equal_rows_of_the_whole_frame(cdef, ctx, ref, kind):
    """Two frames in one call, each a band of its filter-block rows (taps
    and direction search read across the band's edges): the tables equal
    those rows of the oracle's whole-frame tables."""
    from paper_1602_05975_gb300 import synth
    bd = {"sse10": 10, "12bit": 12}.get(kind, 8)
    fmt = 444 if kind == "444" else 420
    frames = [synth.make_frame(w, h, bd, 32, seed=s, chroma=fmt)
              for w, h, s in ((320, 200, 8200), (200, 136, 8201))]
    bands = [(1, 2), (2, 1)]
    coded = None
    if kind == "coded":
        rng = np.random.default_rng(8202)
        coded = [(rng.random((f.height // 8, f.width // 8)) < 0.5).astype(np.uint8) for f in frames]
        coded[0][8:16, 16:24] = 0
    got = _band_tables(cdef, ctx, frames, bands, 128 if coded else 64, coded)
    o = 0
    for i, (f, (r0, rn)) in enumerate(zip(frames, bands)):
        fc = -(-f.width // 64)
        rows = slice(r0 * fc, (r0 + rn) * fc)
        if kind == "coded":
            el, ec, esk = ref.distortion_coded(f.rec, f.src, bd, 5, coded[i])
            assert np.array_equal(got[2][o:o + rn * fc], esk[rows])
        elif fmt != 420 or bd == 12:
            el, ec = ref.distortion_format(f.rec, f.src, bd, 5, fmt)
        else:
            el, ec = ref.distortion(f.rec, f.src, bd, 5)
        w = got[0].shape[1]
        assert np.array_equal(got[0][o:o + rn * fc], el.reshape(-1, w)[rows])
        assert np.array_equal(got[1][o:o + rn * fc], ec.reshape(-1, w)[rows])
        o += rn * fc


def test_band_tables_eq14_and_empty_band(cdef, ctx, ref):
    from test_gpu_parity import _assert_eq14_tables_close, _eq14_term_counts
    from paper_1602_05975_gb300 import synth
    f = synth.make_frame(320, 200, 8, 32, seed=8210)
    ctx.set_search_metric("eq14")
    try:
        dl, dc = _band_tables(cdef, ctx, [f, f], [(2, 2), (0, 0)])
    finally:
        ctx.set_search_metric("sse")
    el, ec = ref.distortion_eq14(f.rec, f.src, 8, 5)
    nl, nc = _eq14_term_counts(320, 200)
    _assert_eq14_tables_close(dl, el[10:20], nl[10:20])
    _assert_eq14_tables_close(dc, ec[10:20], nc[10:20])
    with pytest.raises(cdef.CdefError):    # a band past the frame's rows
        _band_tables(cdef, ctx, [f], [(3, 2)])


def _np_dist(dl, dc, width, t):
    return dl[:, t // width] + dc[:, t % width]


@pytest.mark.parametrize("width", [64, 128])
def test_preset_primitives_equal_their_definitions(cdef, ctx, width):
    """Totals, argmin (subset, keep rule, lowest index on ties) and assign
    (least distortion, first preset attaining it, sums, skipped blocks) on
    random tables with planted ties."""
    rng = np.random.default_rng(8300 + width)
    nb = 300
    dl = rng.integers(0, 1 << 36, (nb, width), dtype=np.int64)
    dc = rng.integers(0, 1 << 36, (nb, width), dtype=np.int64)
    dc[:, 5] = dc[:, 3]                                 # tied presets
    sk = (rng.random(nb) < 0.2).astype(np.uint8)
    g = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    tdl, tdc, tsk = g(dl.reshape(-1)), g(dc.reshape(-1)), g(sk)
    best = torch.zeros(nb, dtype=torch.int64, device="cuda")
    ids = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    sums = torch.zeros(2, dtype=torch.int64, device="cuda")
    tot = torch.zeros(width * width, dtype=torch.int64, device="cuda")
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    keep_sk = ~sk.astype(bool)
    for presets in ([], [7], [3, 5, width * 9 + 2], [1, 2, 3, 4, 5, 6, 7, width * width - 1]):
        cdef.cdef_preset_assign(ctx, nb, width, tdl, tdc, tsk, presets, best, ids, sums)
        d = (np.stack([_np_dist(dl, dc, width, t) for t in presets], 1) if presets
             else np.zeros((nb, 0), np.int64))
        eb = d.min(1) if presets else np.full(nb, -1, np.int64)     # 2^64 - 1 as int64
        ei = np.argmin(d, 1) if presets else np.zeros(nb, np.int64)
        eb[~keep_sk], ei[~keep_sk] = 0, 0
        assert np.array_equal(best.cpu().numpy(), eb)
        assert np.array_equal(ids.cpu().numpy(), ei.astype(np.uint8))
        assert sums.cpu().tolist() == [int(eb[keep_sk].sum()) if presets else 0, int(keep_sk.sum())]
        cdef.cdef_preset_totals(ctx, nb, width, tdl, tdc, tsk, best if presets else None, tot)
        full = (dl[:, :, None] + dc[:, None, :]).reshape(nb, width * width)
        if presets:
            full = np.minimum(full, eb[:, None])
        et = full[keep_sk].sum(0)
        assert np.array_equal(tot.cpu().numpy(), et)
        for lp, cp in ((ALL, ALL), (sum(1 << q for q in (3, 5, 40)), sum(1 << q for q in (0, 3, 5)))):
            ok = np.array([((lp >> ((t // width) % 64)) & 1) and ((cp >> ((t % width) % 64)) & 1)
                           for t in range(width * width)], bool)
            idx = np.flatnonzero(ok)
            v = et[idx].min()
            first = int(idx[np.argmax(et[idx] == v)])
            for keep in (-1, first, int(idx[-1])):
                cdef.cdef_preset_argmin(ctx, width, tot, lp, cp, keep, res)
                want = keep if keep >= 0 and et[keep] == v else first
                assert res.cpu().tolist() == [want, int(et[want])]
    cdef.cdef_preset_totals(ctx, 0, width, None, None, None, None, tot)   # no blocks
    assert int(tot.abs().sum()) == 0
    torch.cuda.synchronize()
    assert ctx.status() == 0


class _HostAllReduce:
    """Ranks emulated as host threads: each call blocks until every rank
    has contributed, then every rank's tensor holds the sum (host-side
    synchronisation only; the ranks' kernels never wait on one another)."""

    def __init__(self, world):
        self.world = world
        self.barrier = threading.Barrier(world, timeout=120)
        self.slots = [None] * world

    def fn(self, rank):
        def allreduce(t):
            torch.cuda.synchronize()
            self.slots[rank] = t
            self.barrier.wait()
            if rank == 0:
                s = sum(x.cpu() for x in self.slots)
                for x in self.slots:
                    x.copy_(s.to(x.device))
                torch.cuda.synchronize()
            self.barrier.wait()
        return allreduce


def _run_ranks(cdef, world, body):
    """Runs body(rank, allreduce) on `world` threads; returns their results."""
    ar = _HostAllReduce(world)
    out, errs = [None] * world, []

    def run(r):
        try:
            out[r] = body(r, ar.fn(r))
        except BaseException as e:  # noqa: BLE001 - re-raised below
            errs.append(e)
            ar.barrier.abort()

    ts = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if errs:
        raise errs[0]
    return out


@pytest.mark.parametrize("world,variant,passes", [(2, "sse", 0), (3, "sse", 2), (3, "coded", 1),
                                                   (2, "subset", 1), (5, "sse", 0)])
def test_sharded_search_equals_oracle(cdef, ref, world, variant, passes):
    """Each emulated rank: its own context, its band's tables
    (cdef_search_tables), the host driver of shard.py with one all-reduce
    of the totals per step.  Every rank returns the oracle's presets, N and
    J; the ranks' ids laid end to end are the oracle's ids (5 ranks over 4
    filter-block rows: one rank holds no blocks)."""
    from paper_1602_05975_gb300 import shard, synth
    f = synth.make_frame(320, 200, 10 if variant == "subset" else 8, 32, seed=8400 + world)
    lp = cp = ALL
    if variant == "subset":
        lp, cp = sum(1 << q for q in (0, 2, 9, 30, 61)), sum(1 << q for q in (0, 1, 33))
    coded = None
    if variant == "coded":
        rng = np.random.default_rng(8401)
        coded = (rng.random((25, 40)) < 0.55).astype(np.uint8)
        coded[8:16, 24:32] = 0
    lam = 900 << (4 if f.bitdepth == 10 else 0)

    def body(rank, allreduce):
        ctx = cdef.Context(0)
        try:
            if variant == "subset":
                ctx.set_search_subset(lp, cp)
            rec, src = cdef.frame_from_numpy(f.rec, f.bitdepth), cdef.frame_from_numpy(f.src, f.bitdepth)
            cm = None if coded is None else torch.from_numpy(coded.reshape(-1)).cuda()
            r = shard.search_strengths_sharded(ctx, rec, src, 5, lam, rank, world, allreduce, cm,
                                               passes)
            torch.cuda.synchronize()
            assert ctx.status() == 0
            return (r["presets"], r["npresets"], r["cost"], r["block_ids"].cpu().numpy(),
                    r["row_begin"], r["row_count"])
        finally:
            ctx.close()

    out = _run_ranks(cdef, world, body)
    if coded is not None:
        dl, dc, sk = ref.distortion_coded(f.rec, f.src, f.bitdepth, 5, coded)
        exp = ref.select_presets_general(dl, dc, 128, sk, lam, passes)
    else:
        exp = ref.search_strengths_subset(f.rec, f.src, f.bitdepth, 5, lam, lp, cp, passes)
    ids, row = [], 0
    for presets, n, cost, bids, r0, rn in out:
        assert presets == [int(t) for t in exp["presets"]]
        assert (n, cost) == (exp["npresets"], exp["cost"])
        assert r0 == row
        row += rn
        ids.append(bids)
    assert row == 4
    assert np.array_equal(np.concatenate(ids), exp["block_ids"])


def test_sharded_search_equals_one_device_search(cdef, ctx):
    """A 1920x1080 frame over 4 emulated ranks against cdef_search_strengths
    on one device (bit-exact presets, N, J, tables and ids)."""
    from paper_1602_05975_gb300 import shard, synth
    f = synth.make_frame(1920, 1080, 8, 32, seed=8500)
    rec, src = cdef.frame_from_numpy(f.rec, 8), cdef.frame_from_numpy(f.src, 8)
    nb = f.params.shape[0] * f.params.shape[1]
    ids = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    dl = torch.zeros(nb * 64, dtype=torch.int64, device="cuda")
    dc = torch.zeros(nb * 64, dtype=torch.int64, device="cuda")
    one = cdef.cdef_search_strengths(ctx, [rec], [src], [5], [1024], ids, dl, dc)[0]

    def body(rank, allreduce):
        c = cdef.Context(0)
        try:
            r = shard.search_strengths_sharded(c, rec, src, 5, 1024, rank, 4, allreduce)
            torch.cuda.synchronize()
            return (r["presets"], r["npresets"], r["cost"], r["block_ids"].cpu(),
                    r["dist_luma"].cpu(), r["dist_chroma"].cpu())
        finally:
            c.close()

    out = _run_ranks(cdef, 4, body)
    for presets, n, cost, *_ in out:
        assert n == one["npresets"] and cost == one["cost"]
        assert presets[:n] == [cdef.preset_index(p) for p in one["presets"][:n]]
    assert torch.equal(torch.cat([o[3] for o in out]), ids.cpu())
    assert torch.equal(torch.cat([o[4] for o in out]), dl.cpu())
    assert torch.equal(torch.cat([o[5] for o in out]), dc.cpu())
