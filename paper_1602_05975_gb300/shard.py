"""Section 5's strength search split over devices (one process per GPU).

The distortion tables are per filter block, so each rank computes the tables
of its own band of filter-block rows (cdef_search_tables) and keeps them on
its device.  The preset selection (eq. 15: the greedy search, the
one-at-a-time re-optimisation, N by J, the block ids) is then driven from
the host, one step at a time, with one exchange per step: every rank forms
the totals of all width^2 presets over its blocks, the totals are summed
over ranks by a collective (``allreduce``), and every rank takes the same
least total.  Totals over block ranges add up exactly to the totals over
their union, so the result equals the one-device selection bit for bit.

The driver is written against two small interfaces so that the collective
and the per-rank arithmetic stay separate:

- a *shard* (``DeviceShard`` here: the C ABI's cdef_preset_assign /
  cdef_preset_totals / cdef_preset_argmin over the rank's tables) with
  ``assign(presets) -> sums``, ``totals() -> totals`` and
  ``argmin(totals, luma_pairs, chroma_pairs, keep) -> (t, total)``;
- ``allreduce(tensor)``: sums a tensor over the ranks in place
  (``torch.distributed.all_reduce``: NCCL between GPUs).
"""
from __future__ import annotations

import torch

from . import cdef

ALL_PAIRS = (1 << 64) - 1


def band_rows(fb_rows: int, rank: int, world: int):
    """The filter-block rows of `rank`: a contiguous band, the bands of all
    ranks covering the frame once, sizes differing by at most one."""
    r0 = fb_rows * rank // world
    return r0, fb_rows * (rank + 1) // world - r0


class DeviceShard:
    """One rank's part of the selection: its band's tables on its device."""

    def __init__(self, ctx: cdef.Context, dist_luma: torch.Tensor, dist_chroma: torch.Tensor,
                 nblocks: int, width: int = 64, skipped: torch.Tensor | None = None,
                 stream=None):
        dev = dist_luma.device
        self.ctx, self.dl, self.dc, self.nblocks, self.width = ctx, dist_luma, dist_chroma, nblocks, width
        self.skipped, self.stream = skipped, stream
        self.best = torch.empty(max(nblocks, 1), dtype=torch.int64, device=dev)  # uint64 values
        self.ids = torch.zeros(max(nblocks, 1), dtype=torch.uint8, device=dev)
        self.sums = torch.zeros(2, dtype=torch.int64, device=dev)
        self.tot = torch.empty(width * width, dtype=torch.int64, device=dev)
        self.res = torch.zeros(2, dtype=torch.int64, device=dev)

    def assign(self, presets):
        """Per-block least distortion and id over `presets`; returns the
        (total, blocks counted) pair of this rank (device)."""
        cdef.cdef_preset_assign(self.ctx, self.nblocks, self.width, self.dl, self.dc, self.skipped,
                                list(presets), self.best, self.ids, self.sums, self.stream)
        return self.sums

    def totals(self):
        """This rank's totals of every preset under the bound of the last
        assign (device)."""
        cdef.cdef_preset_totals(self.ctx, self.nblocks, self.width, self.dl, self.dc, self.skipped,
                                self.best, self.tot, self.stream)
        return self.tot

    def argmin(self, totals, luma_pairs, chroma_pairs, keep):
        cdef.cdef_preset_argmin(self.ctx, self.width, totals, luma_pairs, chroma_pairs, keep,
                                self.res, self.stream)
        r = self.res.cpu()   # the host driver's decision (synchronises the stream)
        return int(r[0]), int(r[1])

    def block_ids(self):
        return self.ids[:self.nblocks]


def select_presets(shard, allreduce, lam: int, refine_passes: int = 0,
                   luma_pairs: int = ALL_PAIRS, chroma_pairs: int = ALL_PAIRS):
    """Eq. 15 over the union of every rank's blocks: the greedy search (each
    step adds the preset of least total, lowest index on ties), then for
    N = 1, 2, 4, 8 the re-optimisation of slots 1..N in turn (a slot keeps
    its preset when that attains the least total) for at most
    `refine_passes` passes, N by J = total + lam * B * log2 N (B: blocks
    not skipped, ties to the smaller N), and this rank's block ids.
    Every rank calls it with its own shard; all return the same presets."""
    greedy, gtot = [], []
    sums = shard.assign([])
    allreduce(sums)
    nb = int(sums[1])
    for _ in range(8):
        shard.assign(greedy)
        tot = shard.totals()
        allreduce(tot)
        t, v = shard.argmin(tot, luma_pairs, chroma_pairs, -1)
        greedy.append(t)
        gtot.append(v)
    best = None
    for lg in range(4):
        n = 1 << lg
        s = greedy[:n]
        total = gtot[n - 1]
        for _ in range(refine_passes):
            changed = False
            for k in range(n):
                shard.assign(s[:k] + s[k + 1:])
                tot = shard.totals()
                allreduce(tot)
                t, v = shard.argmin(tot, luma_pairs, chroma_pairs, s[k])
                if t != s[k]:
                    s[k] = t
                    changed = True
                total = v
            if not changed:
                break
        j = total + lam * nb * lg
        if best is None or j < best[0]:
            best = (j, n, list(s))
    j, n, s = best
    shard.assign(s)
    return dict(presets=s + greedy[n:], npresets=n, cost=j, block_ids=shard.block_ids())


def search_strengths_sharded(ctx: cdef.Context, rec: cdef.Frame, src: cdef.Frame, damping: int,
                             lam: int, rank: int, world: int, allreduce, coded=None,
                             refine_passes: int = 0, stream=None):
    """Section 5's search of one frame with its filter-block rows split over
    `world` ranks: this rank's band tables, then the collective selection.
    The context's metric and subset apply.  Returns the frame's presets
    (indices t = luma_q * width + chroma_q), N, J, and this rank's band:
    its first row, row count, tables and block ids."""
    fb_rows, fb_cols = -(-rec.height // 64), -(-rec.width // 64)
    r0, rn = band_rows(fb_rows, rank, world)
    nb = rn * fb_cols
    width = 64 if coded is None else 128
    dev = rec.y.device
    dl = torch.zeros(max(nb, 1) * width, dtype=torch.int64, device=dev)
    dc = torch.zeros(max(nb, 1) * width, dtype=torch.int64, device=dev)
    skipped = None if coded is None else torch.zeros(max(nb, 1), dtype=torch.uint8, device=dev)
    cdef.cdef_search_tables(ctx, [rec], [src], [damping], [r0], [rn], dl, dc,
                            None if coded is None else [coded], skipped, stream)
    shard = DeviceShard(ctx, dl, dc, nb, width, skipped, stream)
    out = select_presets(shard, allreduce, lam, refine_passes, *ctx.pairs)
    out.update(row_begin=r0, row_count=rn, dist_luma=dl[:nb * width], dist_chroma=dc[:nb * width],
               skipped=None if skipped is None else skipped[:nb])
    return out
