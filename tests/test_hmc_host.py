"""Host logic of the HMC update (paper_1111_5059_gb300/hmc.py): the
Metropolis rule and the update's random numbers."""
import math

import numpy as np

from oracle import dwf_oracle as O
from paper_1111_5059_gb300 import hmc


def test_accept_rule_matches_metropolis():
    for dH in (-1.0, 0.0, 1e-3, 0.5, 3.0):
        for u in (0.0, 0.1, 0.5, 0.9, 0.999):
            assert hmc.accept(dH, u) == O.metropolis_accept(dH, u)
    assert hmc.accept(0.5, math.exp(-0.5) - 1e-12) and not hmc.accept(0.5, math.exp(-0.5) + 1e-12)


def test_draw_is_seeded_and_streams_are_distinct():
    dims, Ls = (4, 2, 2, 4), 4
    p, etas, u = hmc.draw(7, dims, Ls, 2)
    p2, etas2, u2 = hmc.draw(7, dims, Ls, 2)
    assert np.array_equal(p, p2) and all(np.array_equal(a, b) for a, b in zip(etas, etas2)) and u == u2
    assert p.shape == (4, 4, 2, 2, 4, 8) and etas[0].shape == (Ls, 4, 2, 2, 4, 4, 3)
    assert not np.array_equal(etas[0], etas[1])
    assert 0.0 <= u < 1.0
    _, _, u3 = hmc.draw(8, dims, Ls, 2)
    assert u3 != u
    # unit-variance normals
    assert abs(np.var(np.concatenate([e.real.ravel() for e in etas])) - 1.0) < 0.1
