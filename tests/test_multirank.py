"""The benchmark's multi-process path on CPU ranks (gloo, world size 2):
every rank times its own replica, the job's time is the maximum over ranks,
and the whole-job rate counts every rank's frames."""
import os
import socket
import sys

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
