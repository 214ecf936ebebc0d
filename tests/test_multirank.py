"""The host logic of runs on several GPUs, on CPU with gloo and two ranks:
the slowest rank's time, the sharding of ensemble systems, the gather of
per-rank results. No GPU and no data-path collective is involved."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2312_02968_gb300 import replicas as R


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = R.rank_env()
        t = R.max_over_ranks(1.0 + 2.0 * rank, dist)  # rank 1 is the slow one
        costs = [R.system_cost(n, N) for n, N in [(64, 10000), (192, 1000000), (96, 50000), (128, 300000),
                                                  (64, 900000), (192, 20000), (96, 700000)]]
        shards = R.lpt_shard(costs, w)
        mine = shards[r]
        got = R.gather_to_root({"rank": r, "systems": mine, "time": t}, dist)
        if r == 0:
            q.put({"world": w, "t": t, "got": got, "shards": shards, "costs": costs})
        else:
            q.put({"rank": r, "t": t, "got": got})
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    root = next(x for x in res if "world" in x)
    other = next(x for x in res if "rank" in x)
    assert root["world"] == 2
    assert root["t"] == 3.0 and other["t"] == 3.0  # both see the slowest rank's time
    assert other["got"] is None
    got = root["got"]
    assert [g["rank"] for g in got] == [0, 1]
    # every system on exactly one rank
    allsys = sorted(i for g in got for i in g["systems"])
    assert allsys == list(range(7))
    # LPT keeps the loads within the largest item of each other
    loads = [sum(root["costs"][i] for i in s) for s in root["shards"]]
    assert abs(loads[0] - loads[1]) <= max(root["costs"])


def test_single_process_fallbacks():
    assert R.max_over_ranks(2.5) == 2.5
    assert R.gather_to_root({"a": 1}) == [{"a": 1}]
    assert R.lpt_shard([3.0, 1.0, 2.0], 1) == [[0, 1, 2]]
    sh = R.lpt_shard([5.0, 4.0, 3.0, 3.0, 2.0, 1.0], 3)
    assert sorted(sum(sh, [])) == list(range(6))
