"""Virtual ranks on one GPU: a 3-D domain split into z-slab contexts with a
halo exchange after every step reproduces the undivided domain bit for bit."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("outer,nslabs", [(W.BC_NOFLUX, 3), (W.BC_PERIODIC, 4)])
def test_slabs_equal_whole_domain_bitwise(outer, nslabs):
    from paper_2404_01035_gb300 import Simulation
    from paper_2404_01035_gb300.decomp import SlabDomain
    p = W.eutectic_3d(n=48, steps=40)
    p.bc = [W.BC_PERIODIC, W.BC_PERIODIC, outer]
    whole = Simulation(p, dtype="f32")
    whole.set_fields(p.phi0, p.mu0)
    whole.step(40)
    ref = whole.get_fields()
    whole.close()
    dom = SlabDomain(p, nslabs, dtype="f32")
    dom.set_fields(p.phi0, p.mu0)
    dom.step(40)
    got = dom.get_fields()
    dom.close()
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
