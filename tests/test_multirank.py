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


def test_bench_launcher_starts_two_ranks_with_the_rank_logic():
    """`bench.py --gpus 2` starts its own ranks (torch.distributed.run on
    127.0.0.1); the self-test runs only the rank logic on gloo: the world
    size against --gpus, distinct local ranks, the chain shards and seeds,
    and the max-over-ranks time behind the whole-job rate."""
    import json

    import bench
    r = bench.launch_ranks(2, ["--gpus", "2", "--rank-selftest", "--chains", "200"],
                           capture=True, timeout=240)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout  # rank 0 alone prints
    out = json.loads(lines[0])
    assert out["world"] == 2 and sorted(out["local_ranks"]) == [0, 1]
    assert [s["first_chain"] for s in out["shards"]] == [0, 200]
    assert len({s["seed"] for s in out["shards"]}) == 2
    assert out["ms_max"] == 110.0  # the slower rank's time
    assert out["value"] == pytest.approx(2 * 200 / 0.110)


def test_bench_refuses_a_world_size_other_than_gpus():
    import bench
    with pytest.raises(SystemExit, match="WORLD_SIZE is 1"):
        bench.check_world(4, 1)
