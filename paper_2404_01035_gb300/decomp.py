"""Slab decomposition of a 3-D domain along z.

Two uses of one partition:
  * `SlabDomain`: K contexts on one GPU ("virtual ranks"), advanced in lock
    step with ms_halo_exchange / ms_halo_mirror after every step; it must
    reproduce the undivided domain bit for bit.
  * `exchange_halos`: the same exchange between processes with
    torch.distributed point-to-point messages (one padded plane per side and
    field), for slabs held by different ranks.
"""
from __future__ import annotations

import numpy as np

from ._binding import MS_BC_HALO, _check, lib
from .simulation import Simulation

BC_PERIODIC, BC_NOFLUX = 3, 1


def slab_partition(nz: int, nslabs: int):
    """(first plane, number of planes) of each slab; sizes differ by at most one."""
    if nslabs < 1 or nslabs > nz:
        raise ValueError("need 1 <= nslabs <= nz")
    base, extra = divmod(nz, nslabs)
    out, z = [], 0
    for k in range(nslabs):
        n = base + (1 if k < extra else 0)
        out.append((z, n))
        z += n
    return out


class SlabDomain:
    """A 3-D problem split into z-slab contexts on one device."""

    def __init__(self, prob, nslabs: int, dtype: str = "f32", stream=None):
        if prob.dim != 3:
            raise ValueError("slab decomposition is along z of a 3-D domain")
        self.prob = prob
        self.outer = int(prob.bc[2])
        self.parts = slab_partition(prob.nz, nslabs)
        self.sims = []
        for z0, n in self.parts:
            sub = prob.copy(nz=n, bc=[prob.bc[0], prob.bc[1], MS_BC_HALO], phi0=None, mu0=None,
                            meta={**prob.meta, "z_origin": z0})
            self.sims.append(Simulation(sub, dtype=dtype, stream=stream))

    def close(self):
        for s in self.sims:
            s.close()

    def exchange(self):
        L = lib()
        K = len(self.sims)
        for k in range(K - 1):
            _check(L.ms_halo_exchange(self.sims[k].h, self.sims[k + 1].h), self.sims[k].h)
        if self.outer == BC_PERIODIC:
            _check(L.ms_halo_exchange(self.sims[-1].h, self.sims[0].h), self.sims[-1].h)
        else:
            _check(L.ms_halo_mirror(self.sims[0].h, 0), self.sims[0].h)
            _check(L.ms_halo_mirror(self.sims[-1].h, 1), self.sims[-1].h)

    def set_fields(self, phi, mu):
        for (z0, n), s in zip(self.parts, self.sims):
            s.set_fields(np.ascontiguousarray(phi[:, z0:z0 + n]), np.ascontiguousarray(mu[:, z0:z0 + n]))
        self.exchange()

    def step(self, n: int = 1):
        for _ in range(n):
            for s in self.sims:
                s.step(1)
            self.exchange()

    def get_fields(self):
        parts = [s.get_fields() for s in self.sims]
        return np.concatenate([p[0] for p in parts], axis=1), np.concatenate([p[1] for p in parts], axis=1)


def exchange_halos(slab, rank: int, world: int, periodic: bool, group=None, store=None,
                   step: int = 0, timeout_s: float = 10.0):
    """Fill the two ghost planes of `slab` ([F][nz_k + 2][...], ghost planes at
    index 0 and -1) from the neighbouring ranks' boundary planes.

    Outer faces: periodic -> ring neighbour; no-flux -> mirror of the own
    adjacent plane.  Works for CPU tensors (gloo) and CUDA tensors (NCCL).
    With a `store`, every rank first posts a heartbeat for `step` and waits
    (at most timeout_s) for its neighbours' heartbeats, so a rank that has
    left is reported as an error here instead of blocking the exchange.
    """
    import datetime

    import torch.distributed as dist
    up = rank + 1 if rank + 1 < world else (0 if periodic else None)
    down = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    if store is not None and world > 1:
        store.set(f"halo/{step}/{rank}", "1")
        peers = sorted({p for p in (up, down) if p is not None and p != rank})
        store.wait([f"halo/{step}/{p}" for p in peers], datetime.timedelta(seconds=timeout_s))
    ops = []
    send_top = slab[:, -2].contiguous()
    send_bot = slab[:, 1].contiguous()
    recv_top = slab[:, -1].clone()
    recv_bot = slab[:, 0].clone()
    if world > 1:
        # tag 1: a plane travelling up (sender's top -> receiver's bottom ghost),
        # tag 2: travelling down; with two ranks in a ring both go to one peer
        if up is not None:
            ops.append(dist.P2POp(dist.isend, send_top, up, group, tag=1))
            ops.append(dist.P2POp(dist.irecv, recv_top, up, group, tag=2))
        if down is not None:
            ops.append(dist.P2POp(dist.isend, send_bot, down, group, tag=2))
            ops.append(dist.P2POp(dist.irecv, recv_bot, down, group, tag=1))
        if ops:
            for r in dist.batch_isend_irecv(ops):
                r.wait()
    elif periodic:
        recv_top.copy_(send_bot)
        recv_bot.copy_(send_top)
    if up is None:
        recv_top.copy_(slab[:, -2])
    if down is None:
        recv_bot.copy_(slab[:, 1])
    slab[:, -1] = recv_top
    slab[:, 0] = recv_bot
    return slab
