"""Rank process of the sharded-solver GPU test (imported by spawned children)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def rank_main(rank, world, port, case, steps, q):
    sys.path.insert(0, ROOT)
    import datetime

    import torch
    import torch.distributed as dist

    import workloads as W
    from paper_2404_01035_gb300.decomp import ShardedSimulation
    try:
        torch.cuda.set_device(0)
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                                world_size=world, timeout=datetime.timedelta(seconds=60))
        prob, dtype = make_case(W, case)
        sh = ShardedSimulation(prob, rank, world, dtype=dtype)
        if case.endswith("split"):
            tiles = sh.sim.tiles()
            sh.sim.set_launch([i for i, t in enumerate(tiles) if t[2] == 1][0], 8)
        sh.set_global_fields(prob.phi0, prob.mu0)
        sh.step(steps)
        phi, mu = sh.get_fields()
        d = sh.diag()
        sh.close()
        dist.destroy_process_group()
        q.put((rank, phi, mu, d, ""))
    except Exception as e:  # pragma: no cover - reported to the parent
        q.put((rank, None, None, None, repr(e)))


def make_case(W, case):
    if case.startswith("periodic"):
        return W.small_multiphase(n=20, dim=3, N=3, NM=2, nx=24, ny=18, nz=22, bc=[3, 3, 3], rotate=True), "f64"
    if case.startswith("eutectic"):
        return W.eutectic_3d(n=48, steps=40), "f32"
    return W.small_multiphase(n=20, dim=3, N=3, NM=2, nx=24, ny=18, nz=21, bc=[3, 1, 1]), "f64"
