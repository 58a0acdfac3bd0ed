"""Host logic of the replicated multi-GPU bench, on CPU with gloo ranks.

Each rank times its own replica; the job's time is the slowest rank's and its
work is the sum over ranks (bench.aggregate).  Run as two gloo processes on
127.0.0.1; no GPU is involved."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

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
    times, work = bench.aggregate([10.0 + rank, 20.0 - rank], [100.0 * (rank + 1), 7.0], dist, "cpu")
    with open(os.path.join(out, "rank%d.txt" % rank), "w") as f:
        f.write(" ".join(repr(x) for x in times + work))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        vals = [float(x) for x in open(tmp_path / ("rank%d.txt" % r)).read().split()]
        # max over ranks of the times, sum over ranks of the work, identical on every rank
        assert vals == [11.0, 20.0, 300.0, 14.0]


def test_aggregate_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate([3.0, 4.0], [5.0, 6.0]) == ([3.0, 4.0], [5.0, 6.0])


def test_variant_pins_parse():
    import bench
    assert bench.parse_variants("") == {}
    assert bench.parse_variants("P1=20, P4=8") == {"P1 volumes": 20, "P4 forces": 8}
    with pytest.raises(KeyError):
        bench.parse_variants("P9=1")
