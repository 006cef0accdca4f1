"""The windowed one-step oracle used for full-size sampled parity equals a
full-grid oracle step (checked on CPU, including no-flux faces and the
temperature gradient)."""
import numpy as np
import pytest

import oracle
import workloads as W

from gpu_util import pick_cells, windowed_one_step


@pytest.mark.parametrize("dim", [2, 3])
def test_windowed_step_equals_full_step(dim):
    p = W.small_multiphase(n=14, dim=dim, N=3, NM=2, nx=15, ny=13, nz=11, rotate=True,
                           bc=[W.BC_PERIODIC, W.BC_NOFLUX, W.BC_NOFLUX])
    t0 = 0.37
    full_phi, full_mu = oracle.run(p, p.phi0, p.mu0, 1, t0=t0)
    cells = pick_cells(p.phi0, np.random.default_rng(0), n_random=20, n_interface=30)
    wphi, wmu = windowed_one_step(p, p.phi0, p.mu0, cells, t0=t0)
    for n, (z, y, x) in enumerate(cells):
        np.testing.assert_allclose(wphi[n], full_phi[:, z, y, x], atol=1e-14)
        np.testing.assert_allclose(wmu[n], full_mu[:, z, y, x], atol=1e-14)
