"""The command-line driver on a GPU: a paper-format deck (tests/decks) run in
FP64 through `python -m paper_2404_01035_gb300.run`, its snapshots against
the oracle.  Collected after every other GPU test, so that a run stopping at
its first failure has run the rest."""
import os

import numpy as np
import pytest

import oracle
from paper_2404_01035_gb300 import infile as I

pytestmark = pytest.mark.gpu

DECKS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "decks")
FP64_TOL = 1e-10


def test_deck_through_the_driver_matches_the_oracle_fp64(tmp_path):
    from paper_2404_01035_gb300 import run
    deck, fill = os.path.join(DECKS, "ternary_2d.in"), os.path.join(DECKS, "ternary_2d.fill")
    out = tmp_path / "out"
    rc = run.main([deck, fill, "--dtype", "f64", "--out", str(out)])
    assert rc == 0
    files = sorted(os.listdir(out))
    assert files == ["step_0000000000.npz", "step_0000000020.npz", "step_0000000040.npz"]
    s = I.read_infile(deck)
    phi0 = I.read_filling(fill, s)
    mu0 = np.broadcast_to(I.liquid_mu(s, [0.38, 0.33])[:, None, None, None], (2,) + phi0.shape[1:]).copy()
    first = np.load(out / files[0])
    np.testing.assert_array_equal(first["phi"], phi0)
    np.testing.assert_array_equal(first["mu"], mu0)
    for name, n in ((files[1], 20), (files[2], 40)):
        snap = np.load(out / name)
        o_phi, o_mu = oracle.run(s, phi0, mu0, n)
        err = max(np.abs(snap["phi"] - o_phi).max(), np.abs(snap["mu"] - o_mu).max())
        assert err <= FP64_TOL, (name, err)
        assert int(snap["step"]) == n
        assert float(snap["t"]) == pytest.approx(n * s.dt, rel=1e-12)
