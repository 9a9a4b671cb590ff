"""Seeded input generators (no GPU): the load-scenario recipe.

Scenario 0 is the feeder's own draw; scenario k scales each load's a and b
(every phase) by one factor drawn from U[lo, hi], so Q/P stays and only the
draw differs; the bus, phases, connection and load model are untouched.
The same seed gives the same draws."""
import numpy as np

from paper_2501_08293_b300 import feeders as F


def test_load_scenarios_recipe():
    f = F.feeder_123(1)
    L = F.load_scenarios(f, 9, seed=4, lo=0.5, hi=1.0)
    assert L.shape == (9, len(f.loads))
    assert np.array_equal(L[0], f.loads)
    a0 = f.loads["a"]
    b0 = f.loads["b"]
    for k in range(1, 9):
        for name in L.dtype.names:
            if name not in ("a", "b"):
                assert np.array_equal(L[k][name], f.loads[name]), name
        for i in range(len(f.loads)):
            nz = np.flatnonzero(a0[i])
            if len(nz) == 0:
                continue
            fac = L[k]["a"][i, nz] / a0[i, nz]
            assert np.allclose(fac, fac[0], rtol=0, atol=1e-15)        # one factor per load
            assert 0.5 - 1e-15 <= fac[0] <= 1.0 + 1e-15
            assert np.allclose(L[k]["b"][i], b0[i] * fac[0], rtol=1e-15, atol=0)
    assert np.array_equal(L, F.load_scenarios(f, 9, seed=4, lo=0.5, hi=1.0))
    assert not np.array_equal(L[1:], F.load_scenarios(f, 9, seed=5, lo=0.5, hi=1.0)[1:])
