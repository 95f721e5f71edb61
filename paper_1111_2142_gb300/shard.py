"""Multi-GPU layout of the method's independent work: one process per GPU.

The LW-ACM update has no data-path exchange between independent domains, so the
batched ensemble shards by domain (each rank advances its own subset, no
collective on the data path) and the single-domain benchmark runs one independent
domain per rank. Only the timing is combined across ranks: the whole job's
throughput is the units all ranks processed divided by the slowest rank's time.
"""
from __future__ import annotations


def partition(sizes, world_size: int):
    """Assign domains to ranks, balancing the node count: largest domain first,
    each to the currently least-loaded rank (ties to the lower rank). Returns one
    sorted list of domain indices per rank; deterministic, so every rank computes
    the same layout without communicating."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(sizes)), key=lambda b: (-int(sizes[b]), b))
    load = [0] * world_size
    parts = [[] for _ in range(world_size)]
    for b in order:
        r = min(range(world_size), key=lambda k: (load[k], k))
        parts[r].append(b)
        load[r] += int(sizes[b])
    return [sorted(p) for p in parts]


def aggregate_throughput(local_units: float, local_seconds: float, device=None):
    """Combine one rank's work and time over the default process group: returns
    (units summed over ranks, the slowest rank's seconds). Without an initialised
    group (one process) it returns the inputs. device: where the reduction tensors
    live (a CUDA device for NCCL, None / "cpu" for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(local_units), float(local_seconds)
    dev = device if device is not None else "cpu"
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=dev)
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())
