"""Host logic of the Hasenbusch ladders (Sec. 3): the telescoping mass ladder
and the continuous tuning of its intermediate masses, on force models whose
equal-force ladder is known in closed form."""
import math

import pytest

from paper_1111_5059_gb300 import hasenbusch as H


def test_geometric_ladder_and_terms():
    ms = H.geometric_ladder(0.01, 1)
    assert ms == pytest.approx([0.01, 0.1, 1.0], rel=1e-14)  # the 0.01/0.1, 0.1/1 split
    assert H.terms(ms) == [(ms[0], ms[1]), (ms[1], ms[2])]
    ms3 = H.geometric_ladder(0.002, 3)
    assert ms3[0] == 0.002 and ms3[-1] == 1.0
    r = [b / a for a, b in zip(ms3, ms3[1:])]
    assert max(r) / min(r) == pytest.approx(1.0, abs=1e-12)
    # the terms telescope: the product of the ratios is the whole ratio
    assert math.prod(r) == pytest.approx(1.0 / 0.002, rel=1e-12)
    with pytest.raises(ValueError):
        H.terms([0.1, 0.05, 1.0])
    with pytest.raises(ValueError):
        H.geometric_ladder(1.5, 2)


@pytest.mark.parametrize("p", [0.7, 1.0, 1.6])
def test_tuning_equalises_power_law_forces(p):
    # F_i = c_i w_i^p with w_i = log(m_i / m_{i-1}): equal forces need
    # w_i proportional to c_i^(-1/p), with the widths summing to log(1/m)
    c = [4.0, 2.0, 1.0, 0.5]
    m = 0.005

    def norms(ts):
        return [ci * math.log(b / a) ** p for ci, (a, b) in zip(c, ts)]

    start = H.geometric_ladder(m, 3)
    ms, hist = H.tune_ladder(start, norms, iters=40, rtol=1e-6, gamma=1.0 / p)
    assert ms[0] == m and ms[-1] == 1.0
    assert all(b > a for a, b in zip(ms, ms[1:]))
    f = hist[-1][1]
    assert max(f) / min(f) - 1.0 < 1e-6
    q = [ci ** (-1.0 / p) for ci in c]
    want_w = [qi / sum(q) * math.log(1.0 / m) for qi in q]
    got_w = [math.log(b / a) for a, b in zip(ms, ms[1:])]
    assert got_w == pytest.approx(want_w, rel=1e-5)


def test_tuning_with_mass_dependent_forces():
    # lighter terms carry more force at equal width: the tuned ladder packs
    # the light end more densely than the geometric one
    def norms(ts):
        return [math.log(b / a) / math.sqrt(a) for a, b in ts]

    start = H.geometric_ladder(0.01, 2)
    ms, hist = H.tune_ladder(start, norms, iters=30, rtol=1e-3)
    f = hist[-1][1]
    assert max(f) / min(f) - 1.0 < 1e-3
    assert math.log(ms[1] / ms[0]) < math.log(start[1] / start[0])
    assert hist[0][0] == start


def test_no_intermediate_mass_is_left_alone():
    calls = []

    def norms(ts):
        calls.append(ts)
        return [1.0] * len(ts)

    ms, hist = H.tune_ladder([0.01, 1.0], norms)
    assert ms == [0.01, 1.0] and len(calls) == 1
