"""The sharded solver: one slab context per process (two processes, gloo,
both on cuda:0), the boundary planes packed by the library and exchanged
with torch.distributed after every step; the slabs together must equal one
context over the whole 3-D domain bit for bit, and the FP64 diagnostics
reduced over the ranks must equal the whole domain's."""
import os
import socket
import sys

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.parametrize("case", ["periodic", "noflux", "eutectic_split"])
def test_two_process_slabs_equal_the_whole_domain(case):
    import torch.multiprocessing as mp
    sys.path.insert(0, HERE)
    import sharded_worker
    from paper_2404_01035_gb300 import Simulation
    steps, world = 40, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=sharded_worker.rank_main, args=(r, world, port, case, steps, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=600) for _ in range(world)], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
    assert all(not r[4] for r in res), [r[4] for r in res]
    phi = np.concatenate([r[1] for r in res], axis=1)
    mu = np.concatenate([r[2] for r in res], axis=1)
    prob, dtype = sharded_worker.make_case(W, case)
    whole = Simulation(prob, dtype=dtype)
    if case.endswith("split"):
        tiles = whole.tiles()
        whole.set_launch([i for i, t in enumerate(tiles) if t[2] == 1][0], 8)
    whole.set_fields(prob.phi0, prob.mu0)
    whole.step(steps)
    wphi, wmu = whole.get_fields()
    d = whole.diag()
    whole.close()
    assert np.array_equal(phi, wphi) and np.array_equal(mu, wmu)
    for r in res:   # every rank holds the reduced diagnostics
        np.testing.assert_allclose(r[3]["mass"], d["mass"], rtol=1e-13)
        assert r[3]["phi_min"] == d["phi_min"] and r[3]["phi_max"] == d["phi_max"]
        assert r[3]["sum_err"] == d["sum_err"] and r[3]["nonfinite"] == 0
        np.testing.assert_allclose(r[3]["mu_diffusion_number"], d["mu_diffusion_number"], rtol=1e-15)
