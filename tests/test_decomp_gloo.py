"""Multi-rank host logic of the slab decomposition, on CPU with gloo:
partition, halo exchange between processes (periodic and no-flux outer
faces, 2 and 3 ranks), max-over-ranks timing, and failure detection when a
rank leaves before the exchange (the survivor gets an error, not a hang)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, periodic, q):
    sys.path.insert(0, ROOT)
    import datetime

    import torch
    import torch.distributed as dist

    from paper_2404_01035_gb300.decomp import exchange_halos, slab_partition
    try:
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                                world_size=world, timeout=datetime.timedelta(seconds=30))
        F, nz, ny, nx = 3, 11, 4, 5
        g = torch.arange(F * nz * ny * nx, dtype=torch.float64).reshape(F, nz, ny, nx)
        z0, n = slab_partition(nz, world)[rank]
        slab = torch.full((F, n + 2, ny, nx), float("nan"), dtype=torch.float64)
        slab[:, 1:-1] = g[:, z0:z0 + n]
        exchange_halos(slab, rank, world, periodic)
        below = (z0 - 1) % nz if periodic else max(z0 - 1, 0)
        above = (z0 + n) % nz if periodic else min(z0 + n, nz - 1)
        ok = torch.equal(slab[:, 0], g[:, below]) and torch.equal(slab[:, -1], g[:, above])
        t = torch.tensor([float(rank + 1)])
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ok = ok and t.item() == world
        dist.destroy_process_group()
        q.put((rank, bool(ok), ""))
    except Exception as e:  # pragma: no cover - reported to the parent
        q.put((rank, False, repr(e)))


@pytest.mark.parametrize("world,periodic", [(2, True), (2, False), (3, True), (3, False)])
def test_halo_exchange_between_ranks(world, periodic):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, periodic, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    assert all(ok for _, ok, _ in res), res


def _failing_worker(rank, port, q):
    sys.path.insert(0, ROOT)
    import datetime

    import torch
    import torch.distributed as dist

    from paper_2404_01035_gb300.decomp import exchange_halos
    store = dist.TCPStore("127.0.0.1", port, 2, rank == 0, timeout=datetime.timedelta(seconds=30))
    dist.init_process_group("gloo", store=store, rank=rank, world_size=2,
                            timeout=datetime.timedelta(seconds=5))
    slab = torch.zeros(2, 6, 3, 3, dtype=torch.float64)
    exchange_halos(slab, rank, 2, True, store=store, step=0, timeout_s=3.0)   # step 0: both alive
    if rank == 1:
        q.put((rank, "left"))
        q.close()
        q.join_thread()      # flush the message before leaving abruptly
        os._exit(0)          # leaves between steps, before the next exchange
    try:
        exchange_halos(slab, rank, 2, True, store=store, step=1, timeout_s=3.0)
        q.put((rank, "no error"))
    except Exception as e:
        q.put((rank, "error: " + type(e).__name__))


def test_rank_leaving_before_exchange_is_detected():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_failing_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=30)
        if p.is_alive():
            p.terminate()
    assert res[1] == "left"
    assert res[0].startswith("error"), res


def test_slab_partition_covers_the_domain():
    from paper_2404_01035_gb300.decomp import slab_partition
    for nz, k in [(10, 3), (256, 7), (5, 5), (64, 1)]:
        parts = slab_partition(nz, k)
        assert sum(n for _, n in parts) == nz
        assert all(parts[i][0] + parts[i][1] == parts[i + 1][0] for i in range(k - 1))
        assert max(n for _, n in parts) - min(n for _, n in parts) <= 1
    with pytest.raises(ValueError):
        slab_partition(4, 5)


def _packed_worker(rank, world, port, periodic, q):
    sys.path.insert(0, ROOT)
    import datetime

    import torch
    import torch.distributed as dist

    from paper_2404_01035_gb300.decomp import exchange_packed, slab_partition
    try:
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                                world_size=world, timeout=datetime.timedelta(seconds=30))
        F, nz, ny, nx = 2, 9, 3, 4
        g = torch.arange(F * nz * ny * nx, dtype=torch.float64).reshape(F, nz, ny, nx)
        z0, n = slab_partition(nz, world)[rank]
        slab = torch.full((F, n + 2, ny, nx), float("nan"), dtype=torch.float64)
        slab[:, 1:-1] = g[:, z0:z0 + n]
        # a flat packed plane as the library lays it out: every field's plane
        pack = lambda face: slab[:, 1 if face == 0 else n].reshape(-1).clone()

        def unpack(face, t):
            slab[:, 0 if face == 0 else n + 1] = t.reshape(F, ny, nx)

        def mirror(face):
            slab[:, 0 if face == 0 else n + 1] = slab[:, 1 if face == 0 else n]

        for step in range(3):   # repeated exchanges reuse the tags safely
            exchange_packed(pack, unpack, mirror, rank, world, periodic, step=step)
        below = (z0 - 1) % nz if periodic else max(z0 - 1, 0)
        above = (z0 + n) % nz if periodic else min(z0 + n, nz - 1)
        ok = torch.equal(slab[:, 0], g[:, below]) and torch.equal(slab[:, -1], g[:, above])
        dist.destroy_process_group()
        q.put((rank, bool(ok), ""))
    except Exception as e:  # pragma: no cover - reported to the parent
        q.put((rank, False, repr(e)))


@pytest.mark.parametrize("world,periodic", [(1, True), (1, False), (2, True), (2, False), (3, True), (3, False)])
def test_packed_plane_exchange_between_ranks(world, periodic):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_packed_worker, args=(r, world, port, periodic, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    assert all(ok for _, ok, _ in res), res
