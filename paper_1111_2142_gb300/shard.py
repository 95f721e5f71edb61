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


def slabs(nz: int, world_size: int):
    """Split nz planes into world_size contiguous runs [z0, z1), sizes differing by
    at most one (the larger ones first). Every rank needs at least one plane."""
    if world_size < 1 or nz < world_size:
        raise ValueError("need 1 <= world_size <= nz")
    base, extra = divmod(nz, world_size)
    out, z = [], 0
    for r in range(world_size):
        n = base + (1 if r < extra else 0)
        out.append((z, z + n))
        z += n
    return out


class SlabHalo:
    """One periodic domain split along z across ranks (the one data-path exchange
    the method has when a single domain spans GPUs).

    Rank r owns planes [z0, z1) and keeps them at local planes 1 .. n of a slab of
    n + 2 planes; local planes 0 and n + 1 are ghost copies of the neighbouring
    ranks' edge planes. A step of the method on the slab, treated as periodic in z,
    updates the owned planes exactly (each depends only on planes z - 1 .. z + 1);
    the ghosts come out wrong and exchange() refreshes them before the next step.
    fields: per field a tensor (or numpy array) shaped (n + 2, ny, nx); torch
    tensors are exchanged with torch.distributed point-to-point calls (NCCL for CUDA
    tensors, gloo for CPU ones), numpy arrays through CPU tensors."""

    def __init__(self, nz: int, rank: int, world_size: int):
        self.rank, self.world_size = rank, world_size
        self.z0, self.z1 = slabs(nz, world_size)[rank]
        self.n = self.z1 - self.z0
        self.up = (rank + 1) % world_size    # owns the planes above
        self.down = (rank - 1) % world_size  # owns the planes below

    def exchange(self, fields):
        import numpy as np
        import torch
        if self.world_size == 1:
            for f in fields:
                f[0] = f[self.n]
                f[self.n + 1] = f[1]
            return
        import torch.distributed as dist
        tens = [torch.from_numpy(f) if isinstance(f, np.ndarray) else f for f in fields]
        ops, recv = [], []
        for k, t in enumerate(tens):
            top, bottom = t[self.n].contiguous(), t[1].contiguous()
            g_lo, g_hi = torch.empty_like(top), torch.empty_like(top)
            # my top plane is the upper neighbour's lower ghost, my bottom plane the
            # lower neighbour's upper ghost; tags keep the two directions apart
            ops += [dist.P2POp(dist.isend, top, self.up, tag=2 * k),
                    dist.P2POp(dist.isend, bottom, self.down, tag=2 * k + 1),
                    dist.P2POp(dist.irecv, g_lo, self.down, tag=2 * k),
                    dist.P2POp(dist.irecv, g_hi, self.up, tag=2 * k + 1)]
            recv.append((t, g_lo, g_hi))
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        for t, g_lo, g_hi in recv:
            t[0] = g_lo
            t[self.n + 1] = g_hi

    def interior(self, f):
        """The owned planes of a slab field."""
        return f[1:self.n + 1]
