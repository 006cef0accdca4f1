"""Slab decomposition of a 3-D domain along z.

Three uses of one partition:
  * `SlabDomain`: K contexts on one GPU ("virtual ranks"), advanced in lock
    step with ms_halo_exchange / ms_halo_mirror after every step; it must
    reproduce the undivided domain bit for bit.
  * `ShardedSimulation`: one slab context per process, the planes packed by
    the library (ms_halo_pack / ms_halo_unpack) and exchanged with
    torch.distributed point-to-point messages (`exchange_packed`), the
    diagnostics reduced over the ranks in FP64.
  * `exchange_halos`: the same exchange for slabs held as plain tensors
    ([F][nz_k + 2][...]).
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


def exchange_packed(pack, unpack, mirror, rank: int, world: int, periodic: bool, group=None, store=None,
                    step: int = 0, timeout_s: float = 10.0):
    """One halo exchange of a slab held by this rank, through packed planes.

    pack(face) -> tensor: the boundary plane on `face` (0 bottom, 1 top), in
    memory the process group can send (host for gloo, device for NCCL);
    unpack(face, tensor): write a neighbour's plane into the ghost plane on
    `face`; mirror(face): no-flux ghost plane (outer faces of a non-periodic
    domain).  The top plane travels up (tag 1) into the upper rank's bottom
    ghost, the bottom plane down (tag 2) into the lower rank's top ghost;
    periodic domains close the ring.  With a `store`, every rank first posts
    a heartbeat for `step` and waits at most timeout_s for its neighbours',
    so a rank that has left is reported here instead of blocking the
    exchange.
    """
    import datetime

    import torch.distributed as dist
    up = rank + 1 if rank + 1 < world else (0 if periodic else None)
    down = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    if world == 1:
        if periodic:
            top, bot = pack(1), pack(0)
            unpack(0, top)
            unpack(1, bot)
        else:
            mirror(0)
            mirror(1)
        return
    if store is not None:
        store.set(f"halo/{step}/{rank}", "1")
        peers = sorted({p for p in (up, down) if p is not None and p != rank})
        store.wait([f"halo/{step}/{p}" for p in peers], datetime.timedelta(seconds=timeout_s))
    ops, recv = [], {}
    if up is not None:
        top = pack(1)
        recv[1] = torch_empty_like(top)
        ops.append(dist.P2POp(dist.isend, top, up, group, tag=1))
        ops.append(dist.P2POp(dist.irecv, recv[1], up, group, tag=2))
    if down is not None:
        bot = pack(0)
        recv[0] = torch_empty_like(bot)
        ops.append(dist.P2POp(dist.isend, bot, down, group, tag=2))
        ops.append(dist.P2POp(dist.irecv, recv[0], down, group, tag=1))
    for r in dist.batch_isend_irecv(ops):
        r.wait()
    for face in (0, 1):
        if face in recv:
            unpack(face, recv[face])
        else:
            mirror(face)


def torch_empty_like(t):
    import torch
    return torch.empty_like(t)


class ShardedSimulation:
    """This rank's z-slab of a 3-D domain decomposed over processes.

    Each rank owns one library context whose z faces are MS_BC_HALO (its first
    global plane as the grid's z_origin, so the temperature field stays
    global); after every step (and after the state is loaded) the slabs swap
    one packed plane per side (ms_halo_pack / ms_halo_unpack) through
    torch.distributed: device tensors for NCCL, host copies for gloo.  The
    diagnostics are reduced over the ranks in FP64.
    """

    def __init__(self, prob, rank: int, world: int, dtype: str = "f32", stream=None, group=None,
                 store=None, timeout_s: float = 10.0):
        import torch
        import torch.distributed as dist
        if prob.dim != 3:
            raise ValueError("slab decomposition is along z of a 3-D domain")
        self._torch = torch
        self.prob, self.rank, self.world = prob, int(rank), int(world)
        self.group, self.store, self.timeout_s = group, store, timeout_s
        self.periodic = int(prob.bc[2]) == BC_PERIODIC
        self.parts = slab_partition(prob.nz, self.world)
        z0, n = self.parts[self.rank]
        self.z0, self.nz = z0, n
        sub = prob.copy(nz=n, bc=[prob.bc[0], prob.bc[1], MS_BC_HALO], phi0=None, mu0=None,
                        meta={**prob.meta, "z_origin": z0})
        self.sim = Simulation(sub, dtype=dtype, stream=stream)
        L = lib()
        self.nbytes = int(L.ms_halo_plane_bytes(self.sim.h))
        self._planes = torch.empty((4, self.nbytes), dtype=torch.uint8, device="cuda")
        host = self.world > 1 and dist.get_backend(group) == "gloo"
        self._host = torch.empty((4, self.nbytes), dtype=torch.uint8, pin_memory=True) if host else None
        self.exchanges = 0

    def close(self):
        self.sim.close()

    # -------------------------------------------------------------- exchange
    def _pack(self, face):
        """Boundary plane `face` packed on the device (host copy for gloo)."""
        buf = self._planes[face]
        _check(lib().ms_halo_pack(self.sim.h, face, buf.data_ptr()), self.sim.h)
        self.sim.stream.synchronize()
        if self._host is None:
            return buf
        h = self._host[face]
        h.copy_(buf)
        return h

    def _unpack(self, face, t):
        if not t.is_cuda:
            dst = self._planes[2 + face]
            dst.copy_(t)
            self._torch.cuda.current_stream().synchronize()
            t = dst
        _check(lib().ms_halo_unpack(self.sim.h, face, t.data_ptr()), self.sim.h)
        self.sim.stream.synchronize()

    def _mirror(self, face):
        _check(lib().ms_halo_mirror(self.sim.h, face), self.sim.h)

    def exchange(self):
        """Fill both ghost planes from the neighbouring ranks (or mirror / wrap
        the outer faces)."""
        exchange_packed(self._pack, self._unpack, self._mirror, self.rank, self.world, self.periodic,
                        self.group, self.store, self.exchanges, self.timeout_s)
        self.exchanges += 1

    # ------------------------------------------------------------ state, steps
    def set_fields(self, phi, mu):
        """This slab's fields ([F][nz_k][ny][nx]); then the first exchange."""
        self.sim.set_fields(phi, mu)
        self.exchange()

    def set_global_fields(self, phi, mu):
        """Cut this rank's planes out of the whole domain's fields."""
        z0, n = self.z0, self.nz
        self.set_fields(np.ascontiguousarray(phi[:, z0:z0 + n]), np.ascontiguousarray(mu[:, z0:z0 + n]))

    def step(self, n: int = 1):
        for _ in range(int(n)):
            self.sim.step(1)
            self.exchange()

    def get_fields(self):
        return self.sim.get_fields()

    def diag(self):
        """ms_diag of the whole domain: solute masses and the non-finite count
        summed, max |sum phi - 1|, max phi and the mu-diffusion number maxed,
        min phi minned over the ranks, in FP64."""
        import ctypes

        import torch
        import torch.distributed as dist
        NM = self.sim.NM
        out = np.zeros(NM + 7)
        st = lib().ms_diag(self.sim.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        if st not in (0, 5):   # MS_ERR_NONFINITE still fills the values
            _check(st, self.sim.h)
        v = torch.tensor(out[:NM + 5], dtype=torch.float64)
        if self.world > 1:
            dev = "cpu" if self._host is not None else "cuda"
            s = torch.cat([v[:NM], v[NM + 3:NM + 4]]).to(dev)
            mx = torch.stack([v[NM], v[NM + 2], v[NM + 4]]).to(dev)
            mn = v[NM + 1:NM + 2].clone().to(dev)
            dist.all_reduce(s, op=dist.ReduceOp.SUM, group=self.group)
            dist.all_reduce(mx, op=dist.ReduceOp.MAX, group=self.group)
            dist.all_reduce(mn, op=dist.ReduceOp.MIN, group=self.group)
            s, mx, mn = s.cpu(), mx.cpu(), mn.cpu()
            v[:NM] = s[:NM]
            v[NM + 3] = s[NM]
            v[NM], v[NM + 2], v[NM + 4] = mx[0], mx[1], mx[2]
            v[NM + 1] = mn[0]
        v = v.numpy()
        return {"mass": v[:NM].copy(), "sum_err": v[NM], "phi_min": v[NM + 1], "phi_max": v[NM + 2],
                "nonfinite": v[NM + 3], "mu_diffusion_number": v[NM + 4], "step": int(out[NM + 5]),
                "t": out[NM + 6]}
