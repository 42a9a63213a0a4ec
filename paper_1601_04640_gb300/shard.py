"""Host-side sharding of a batched 2D sweep across GPUs (one process per GPU).

The problems of a sweep are independent, so the multi-GPU form partitions
them and needs no collective on the data path: each rank steps its own
subset with one `dgpe.Batch`, and the only exchange is a host-side gather of
per-problem results at the end (`torch.distributed.all_gather_object`, which
works over NCCL and gloo alike).

Cost model of one step of an N x N problem: N^2 log2 N (the transforms
dominate; the Crank-Nicolson and exponential substeps add terms linear in
N^2).  Partition: longest-processing-time-first greedy, ties broken by index,
so every rank computes the same assignment without communicating.
"""
import math


def cost(problem) -> float:
    nx, ny = problem["n"]
    return float(nx * ny) * math.log2(max(nx, ny))


def partition(problems, world: int):
    """Problem indices per rank: a list of `world` sorted index lists that
    together hold every index exactly once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(problems)), key=lambda i: (-cost(problems[i]), i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += cost(problems[i])
    return [sorted(p) for p in parts]


def imbalance(problems, parts) -> float:
    """max over ranks of the rank's cost / the mean cost (1 = perfect)."""
    loads = [sum(cost(problems[i]) for i in p) for p in parts]
    mean = sum(loads) / len(loads)
    return max(loads) / mean if mean > 0 else 1.0


def max_over_ranks(value: float) -> float:
    """The maximum of a host scalar over all ranks (the slowest rank's time);
    the value itself when no process group is running.  The reduction runs
    on a CUDA tensor under NCCL and a CPU tensor under gloo."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather(local: dict, group=None):
    """All ranks' {problem index: result} merged into one dict on every rank
    (host objects; no device buffers involved)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return dict(local)
    out = [None] * dist.get_world_size(group)
    dist.all_gather_object(out, local, group=group)
    merged = {}
    for d in out:
        merged.update(d)
    return merged
