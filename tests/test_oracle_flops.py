"""The op-counting scalar of the oracle (count_flops), which gives the
algorithmic flops per cell of the step's ALU roof: it counts every binary
operation on state values, so the counts follow the branches the method
takes and nothing else."""
import numpy as np

import oracle
import workloads as W


def test_counts_follow_the_state_not_its_values():
    # a uniform periodic interface state: every cell takes the same branches
    p = W.binary_problem("cnt", 12, ny=10, Delta=0.2, R=0.0, delta=0.0)
    phi = np.stack([np.full((1, 10, 12), 0.3), np.full((1, 10, 12), 0.7)])
    mu = np.full((1, 1, 10, 12), 1.6)
    a, b = oracle.count_flops(p, phi, mu)
    assert a.min() == a.max() > 0 and b.min() == b.max() > 0
    # other values, same branches: the same counts
    a2, b2 = oracle.count_flops(p, phi * 0.5 + 0.25, mu * 1.3)
    assert np.array_equal(a, a2) and np.array_equal(b, b2)


def test_counts_match_the_oracle_step_and_its_branches():
    p = W.small_multiphase(n=10, dim=3, N=3, NM=2)
    a, b = oracle.count_flops(p, p.phi0, p.mu0)
    # an anisotropic pair with q = 0 skips its flux: a pure stencil costs less
    pure = np.zeros_like(p.phi0)
    pure[2] = 1.0
    ap, bp = oracle.count_flops(p, pure, p.mu0)
    assert ap.max() < a.min()
    # the mu sweep does not branch on phi: equal counts
    assert np.array_equal(b, bp)
    # grain growth holds mu: no mu-sweep arithmetic at all
    _, bg = oracle.count_flops(p, p.phi0, p.mu0, grain_growth=1)
    assert bg.max() == 0.0
    # the anti-trapping current adds arithmetic to the mu sweep only
    aa, ba = oracle.count_flops(p, p.phi0, p.mu0, anti_trapping=1)
    assert np.array_equal(aa, a) and (ba > b).all()
