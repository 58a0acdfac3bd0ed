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


def test_oracle_cone_gives_the_full_evaluation():
    """The bench states its error on sampled particles whose oracle values come
    from their dependency cone alone; on a small workload those values equal a
    full FP64 evaluation (same per-particle sums), so the cone is complete."""
    import numpy as np
    import bench
    from oracle import crk as O
    from paper_2202_02840_gb300 import inputs
    st = inputs.zeldovich(24)
    s = np.sort(np.random.default_rng(3).choice(st["pos_h"].shape[0], 4, replace=False))
    p1, p2, gv, p4, ncone = bench.oracle_cone(st, s)
    ev = O.evaluate(st)
    assert 4 < ncone < st["pos_h"].shape[0]
    for a, b in ((p1["V"], ev["V"]), (p2["A"], ev["A"]), (p2["B"], ev["B"]), (p2["gA"], ev["gA"]),
                 (p2["gB"], ev["gB"]), (gv, ev["gv"]), (p4["acc"], ev["acc"]), (p4["dudt"], ev["dudt"]),
                 (p4["fscale"], ev["fscale"])):
        np.testing.assert_allclose(a[s], b[s], rtol=1e-13, atol=1e-13 * np.abs(b[s]).max())
    # a cone missing the gather neighbours of the union neighbours is wrong
    V_bad = O.volumes(st["pos_h"], targets=s)["V"]
    c_bad = O.corrections(st["pos_h"], V_bad, targets=s)
    assert not np.allclose(c_bad["A"][s], ev["A"][s], rtol=1e-9)
