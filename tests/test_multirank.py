"""The N > 1 host logic of bench.py on CPU with the gloo backend, world size 2:
each rank gets an independent shard of chains (distinct random streams), the
slowest rank's time is shared by the max-reduction, and the whole-job rate
is computed from it."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sh = bench.shard(world, rank, 200)
        my_ms = 1000.0 + 250.0 * rank
        ms_max = bench.max_over_ranks(my_ms, dist, "cpu")
        out[rank] = (sh["seed"], sh["first_chain"], ms_max, bench.aggregate(world, 200, 10, ms_max))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_and_max_timing():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    seeds = {res[r][0] for r in res}
    assert len(seeds) == 2                       # independent random streams
    assert {res[r][1] for r in res} == {0, 200}  # disjoint chain ranges
    for r in res:
        assert res[r][2] == 1250.0               # every rank sees the slowest time
        assert res[r][3] == pytest.approx(2 * 200 * 10 / 1.25)


def test_single_rank_needs_no_collective():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.aggregate(1, 200, 4, 2000.0) == pytest.approx(400.0)
