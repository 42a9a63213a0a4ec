"""Multi-GPU form of the batched sweep, host side: the cost partition and the
host gather of results, run as two gloo ranks on the CPU (no GPU, no device
collective: the problems are independent)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1601_04640_gb300 import shard, synth


def test_partition_covers_sweep_once_and_balances():
    sweep = synth.batched_problems(4640, 512)
    for world in (1, 2, 3, 4, 8):
        parts = shard.partition(sweep, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sweep)))
        assert shard.imbalance(sweep, parts) < 1.02
    assert shard.partition(sweep, 1) == [list(range(512))]
    with pytest.raises(ValueError):
        shard.partition(sweep, 0)


def test_partition_is_deterministic_and_cost_ordered():
    probs = [dict(n=(n, n)) for n in (64, 512, 64, 512, 256)]
    a = shard.partition(probs, 2)
    assert a == shard.partition(probs, 2)
    # the two largest go to different ranks
    assert (1 in a[0]) != (3 in a[0])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sweep = synth.batched_problems(4640, 512)
        mine = shard.partition(sweep, world)[rank]
        # stand-in for the per-problem results a rank's Batch would return
        local = {i: float(sweep[i]["g"]) for i in mine}
        merged = shard.gather(local)
        slowest = shard.max_over_ranks(1.0 + rank)  # each rank's "time"
        q.put((rank, len(mine), len(merged), sorted(merged) == list(range(512)),
               all(merged[i] == float(sweep[i]["g"]) for i in merged), slowest))
    finally:
        dist.destroy_process_group()


def test_two_rank_gather_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert res[0][1] + res[1][1] == 512
    for r in res:
        assert r[2] == 512 and r[3] and r[4]
        assert r[5] == 2.0
