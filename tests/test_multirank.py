"""The multi-GPU benchmark's host logic on CPU: two gloo ranks (127.0.0.1)
combine their own timings and segment counts as the benchmark does under
torchrun -- the slowest rank's seconds and the sum of their bands' segments
(the split of one bundle over the ranks and the gather of its maps are tested
in test_shard.py)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    total_ms = [12.5, 20.0][rank]
    segs = [1000, 2345][rank]
    e2e = [0.3, 0.2][rank]
    out[rank] = bench.combine_over_ranks(dist, "cpu", total_ms, segs, e2e)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_like_the_benchmark():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        ms, segs, e2e = res[rank]
        assert ms == 20.0 and segs == 3345 and e2e == 0.3


def test_one_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_over_ranks(None, "cpu", 5.0, 7, 0.1) == (5.0, 7, 0.1)
