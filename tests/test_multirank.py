"""The benchmark's multi-process path on CPU ranks (gloo, world size 2):
every rank times its own replica, the job's time is the maximum over ranks,
and the whole-job rate counts every rank's frames."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    try:
        t = bench.max_over_ranks(10.0 + 5.0 * rank)
        seeds = bench.frame_seeds(rank)
        dist.barrier()
        out[rank] = (t, tuple(seeds))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_disjoint_replicas():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0          # the slower rank's time
    assert not set(res[0][1]) & set(res[1][1])      # each replica its own frames


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5


def test_whole_job_rate_is_weak_scaling():
    sys.path.insert(0, ROOT)
    import bench
    one = bench.whole_job_rate(1, 8 * 3840 * 2160, 0.5)
    assert bench.whole_job_rate(4, 8 * 3840 * 2160, 0.5) == pytest.approx(4 * one)
    assert one == pytest.approx(8 * 3840 * 2160 / 0.5e-3 / 1e6)


# --------------------------------------------------------------- sharded strength search
class _OracleRowsShard:
    """One rank's part of the sharded preset selection on the CPU: the
    oracle's table rows of the rank's band, reduced with numpy (the GPU
    ranks run the C ABI's kernels instead)."""

    def __init__(self, dl, dc, width, skipped):
        self.dl, self.dc, self.width = dl, dc, width
        self.skip = (np.zeros(dl.shape[0], bool) if skipped is None
                     else np.asarray(skipped, bool))
        self.best = np.full(dl.shape[0], 1 << 62, np.int64)
        self.ids = np.zeros(dl.shape[0], np.uint8)

    def _d(self, t):
        return self.dl[:, t // self.width] + self.dc[:, t % self.width]

    def assign(self, presets):
        n = self.dl.shape[0]
        if presets:
            d = np.stack([self._d(t) for t in presets], axis=1)
            self.ids = np.argmin(d, axis=1).astype(np.uint8)
            self.best = d.min(axis=1)
        else:
            self.ids = np.zeros(n, np.uint8)
            self.best = np.full(n, 1 << 62, np.int64)
        self.best[self.skip] = 0
        self.ids[self.skip] = 0
        tot = int(self.best[~self.skip].sum()) if presets else 0
        return torch.tensor([tot, int((~self.skip).sum())], dtype=torch.int64)

    def totals(self):
        d = (self.dl[:, :, None] + self.dc[:, None, :]).reshape(self.dl.shape[0], self.width ** 2)
        d = np.minimum(d, self.best[:, None])[~self.skip]
        return torch.from_numpy(d.sum(axis=0).astype(np.int64))

    def argmin(self, totals, luma_pairs, chroma_pairs, keep):
        w = self.width
        t = np.arange(w * w)
        ok = np.array([bool((luma_pairs >> ((i // w) % 64)) & 1) and
                       bool((chroma_pairs >> ((i % w) % 64)) & 1) for i in range(w * w)], bool)
        tot = totals.numpy()
        v = tot[ok].min()
        best = int(t[ok][np.argmax(tot[ok] == v)])
        if keep >= 0 and tot[keep] == v:
            best = keep
        return best, int(tot[best])

    def block_ids(self):
        return self.ids


def _shard_rank(rank, world, port, case, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1602_05975_gb300 import shard
    try:
        dl, dc, sk, width, fb_cols = case["dl"], case["dc"], case["skipped"], case["width"], case["fb_cols"]
        r0, rn = shard.band_rows(dl.shape[0] // fb_cols, rank, world)
        rows = slice(r0 * fb_cols, (r0 + rn) * fb_cols)
        part = _OracleRowsShard(dl[rows], dc[rows], width, None if sk is None else sk[rows])
        calls = []

        def allreduce(t):
            calls.append(t.numel())
            dist.all_reduce(t, op=dist.ReduceOp.SUM)

        res = shard.select_presets(part, allreduce, case["lam"], case["passes"],
                                   case["luma_pairs"], case["chroma_pairs"])
        out[rank] = (list(res["presets"]), res["npresets"], res["cost"],
                     np.asarray(res["block_ids"]).tolist(), r0, rn, calls)
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def shard_cases(ref):
    """Oracle tables of a 320x200 frame (5 x 4 filter blocks): squared
    error, and the 128 combinations over a coded-residual map."""
    from paper_1602_05975_gb300 import synth
    f = synth.make_frame(320, 200, 8, 32, seed=8100)
    dl, dc = ref.distortion(f.rec, f.src, 8, 5)
    rng = np.random.default_rng(8101)
    coded = (rng.random((25, 40)) < 0.5).astype(np.uint8)
    coded[:8, 8:16] = 0                       # one filter block without residual
    cl, cc, sk = ref.distortion_coded(f.rec, f.src, 8, 5, coded)
    return dict(sse=(dl.reshape(-1, 64), dc.reshape(-1, 64), None, 64),
                coded=(cl.reshape(-1, 128), cc.reshape(-1, 128), sk, 128))


@pytest.mark.parametrize("world,variant,passes,subset", [
    (2, "sse", 0, False), (2, "sse", 2, True), (3, "coded", 1, False), (5, "sse", 1, False)])
def test_sharded_selection_equals_single_device(ref, shard_cases, world, variant, passes, subset):
    """Section 5 over filter-block rows split across `world` gloo ranks (5
    ranks over 4 rows: one rank holds no blocks): per step every rank sums
    its rows' totals of all presets, one all-reduce, the same argmin on
    every rank.  Presets, N, J and the gathered block ids equal the
    single-device oracle selection bit for bit."""
    dl, dc, sk, width = shard_cases[variant]
    lp = cp = (1 << 64) - 1
    if subset:
        lp = sum(1 << q for q in (0, 3, 9, 22, 41, 63))
        cp = sum(1 << q for q in (0, 5, 17, 30))
    lam = 900
    case = dict(dl=dl, dc=dc, skipped=sk, width=width, fb_cols=5, lam=lam, passes=passes,
                luma_pairs=lp, chroma_pairs=cp)
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_rank, args=(world, port, case, out), nprocs=world, join=True)
        res = dict(out)
    exp = ref.select_presets_subset(dl, dc, width, sk, lp, cp, lam, passes)
    ids = []
    for r in range(world):
        presets, n, cost, bids, r0, rn, calls = res[r]
        assert presets == [int(t) for t in exp["presets"]]
        assert (n, cost) == (exp["npresets"], exp["cost"])
        assert len(bids) == rn * 5
        ids += bids
        # one exchange of width^2 totals per step (8 greedy steps + the
        # re-optimisation's), plus the block count
        assert calls[0] == 2 and all(c == width * width for c in calls[1:])
    assert ids == exp["block_ids"].tolist()
