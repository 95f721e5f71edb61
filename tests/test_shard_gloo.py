"""The multi-process path on CPU ranks (gloo, world size 2): the ensemble's
domain partition and the whole-job throughput reduction that bench.py uses."""
import os
import socket

import numpy as np
import pytest

from paper_1111_2142_gb300 import inputs
from paper_1111_2142_gb300.shard import SlabHalo, aggregate_throughput, partition, slabs


def test_partition_covers_and_balances():
    doms = inputs.ensemble_2d(256, seed=1)
    sizes = [d["nx"] * d["ny"] for d in doms]
    for ws in (1, 2, 3, 4, 8):
        parts = partition(sizes, ws)
        flat = sorted(b for p in parts for b in p)
        assert flat == list(range(256))
        loads = [sum(sizes[b] for b in p) for p in parts]
        # greedy largest-first: no rank exceeds the mean by more than the largest domain
        assert max(loads) - sum(loads) / ws <= max(sizes)
        assert partition(sizes, ws) == parts  # deterministic
    assert partition([5, 5], 4) == [[0], [1], [], []]
    with pytest.raises(ValueError):
        partition(sizes, 0)


def test_single_process_aggregate_is_identity():
    assert aggregate_throughput(12.0, 0.5) == (12.0, 0.5)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import oracle
        doms = inputs.ensemble_2d(12, seed=3, smin=8, smax=40)
        sizes = [d["nx"] * d["ny"] for d in doms]
        mine = partition(sizes, ws)[rank]
        out = {}
        for b in mine:
            d = doms[b]
            out[b] = oracle.step(9, d["d"], d["ux"], d["uy"], nu=d["nu"], nsteps=4, nthreads=1)
        gathered = [None] * ws
        dist.all_gather_object(gathered, out)
        units, secs = aggregate_throughput(sum(sizes[b] for b in mine) * 4, 0.1 * (rank + 1))
        if rank == 0:
            merged = {}
            for g in gathered:
                merged.update(g)
            q.put((sorted(merged), {b: [a.tolist() for a in v] for b, v in merged.items()}, units, secs,
                   sum(sizes) * 4))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_ensemble():
    """Each rank advances only its share of the domains; gathered, the results
    equal a one-process run bit for bit, and the reduction gives the total work
    over the slowest rank's time."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        keys, res, units, secs, total = q.get(timeout=120)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    assert keys == list(range(12))
    assert units == total and secs == pytest.approx(0.2)
    doms = inputs.ensemble_2d(12, seed=3, smin=8, smax=40)
    for b, d in enumerate(doms):
        ref = oracle.step(9, d["d"], d["ux"], d["uy"], nu=d["nu"], nsteps=4, nthreads=1)
        for a, r in zip(res[b], ref):
            assert np.array_equal(np.asarray(a), r)


def test_slabs_cover_every_plane():
    for nz, ws in ((7, 3), (16, 4), (5, 5), (9, 1)):
        s = slabs(nz, ws)
        assert s[0][0] == 0 and s[-1][1] == nz
        assert all(a[1] == b[0] for a, b in zip(s, s[1:]))
        assert max(b - a for a, b in s) - min(b - a for a, b in s) <= 1
    with pytest.raises(ValueError):
        slabs(3, 4)


def _slab_main(rank, ws, port, q, shape, T):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import oracle
        nz = shape[0]
        f = inputs.smooth_random(shape, seed=11, u_amp=0.05, d_amp=0.01)
        h = SlabHalo(nz, rank, ws)
        # owned planes plus ghosts, filled by one exchange
        sl = [np.zeros((h.n + 2,) + shape[1:]) for _ in f]
        for s_, g in zip(sl, f):
            s_[1:h.n + 1] = g[h.z0:h.z1]
        h.exchange(sl)
        for _ in range(T):
            sl = list(oracle.step(19, *sl, nu=0.02, nsteps=1, nthreads=1))
            h.exchange(sl)
        gathered = [None] * ws
        dist.all_gather_object(gathered, (h.z0, h.z1, [h.interior(s_).tolist() for s_ in sl]))
        if rank == 0:
            q.put(gathered)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws,shape", [(2, (6, 5, 7)), (3, (7, 4, 6))])
def test_slab_halo_exchange_reproduces_the_single_domain(ws, shape):
    """A periodic D3Q19 domain split along z over gloo ranks, each stepping its
    slab with one ghost plane per side and exchanging ghosts after every step,
    equals the undivided run bit for bit."""
    import multiprocessing as mp
    import oracle
    from paper_1111_2142_gb300.shard import SlabHalo  # noqa: F401  (spawned ranks import it)
    oracle.build()
    T = 5
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_main, args=(r, ws, port, q, shape, T)) for r in range(ws)]
    for p in procs:
        p.start()
    try:
        gathered = q.get(timeout=120)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    f = inputs.smooth_random(shape, seed=11, u_amp=0.05, d_amp=0.01)
    ref = oracle.step(19, *f, nu=0.02, nsteps=T, nthreads=1)
    for z0, z1, parts in gathered:
        for part, r in zip(parts, ref):
            assert np.array_equal(np.asarray(part), r[z0:z1])
