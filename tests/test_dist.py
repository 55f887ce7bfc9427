"""Multi-rank host logic on CPU (gloo, world size 2): graph sharding and
the whole-job aggregation used by the benchmark."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1505_04086_gb300 import dist as D  # noqa: E402


def test_shard_graphs_cover_and_balance():
    sizes = [1000, 5, 300, 300, 7, 2048, 1, 64, 900, 33]
    for world in (1, 2, 3, 4):
        parts = [D.shard_graphs(sizes, r, world) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)
    with pytest.raises(ValueError):
        D.shard_graphs(sizes, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = [10, 20, 30, 40, 50]
        mine = D.shard_graphs(sizes, rank, world)
        units = sum(sizes[i] for i in mine)
        total, secs = D.aggregate(units, 1.0 + rank)
        q.put((rank, mine, total, secs))
    finally:
        dist.destroy_process_group()


def test_aggregate_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert sorted(res[0][1] + res[1][1]) == [0, 1, 2, 3, 4]
    for r in res:
        assert r[2] == 150.0      # all graphs' sizes, summed over ranks
        assert r[3] == 2.0        # slowest rank
    assert D.aggregate(5, 3.0) == (5.0, 3.0)  # no process group: local values
