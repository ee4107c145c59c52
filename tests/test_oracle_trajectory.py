"""Pins of the oracle's molecular-dynamics trajectories (CPU only): the
force-gradient integrator against the Omelyan 2MN integrator that Sec. 2
compares it with, whole trajectories with merged end momentum updates, and
the Metropolis test.

  * The 2MN parameter equals its published closed form.
  * A trajectory with merged end updates equals the same number of single
    steps (the merge only saves force evaluations: 3n+1 and 2n+1 of them).
  * Orders: |dH| over a trajectory of fixed length falls as tau^2 for
    Omelyan and as tau^4 for the force-gradient integrator; at the same step
    the force-gradient error is far smaller (what lets Sec. 2 raise the step).
  * An Omelyan trajectory is reversible (p -> -p retraces it).
"""
import numpy as np
import pytest

from oracle import dwf_oracle as O
from paper_1111_5059_gb300 import inputs as I

M5 = 1.8
TERMS = [(0.2, 1.0)]  # one Hasenbusch quotient with a Pauli-Villars denominator
LENGTH = 0.5          # trajectory length


@pytest.fixture(scope="module")
def md():
    dims, Ls = (4, 2, 2, 4), 4
    U = I.gauge_field(43, dims, 0.5)
    p = I.gaussian_momenta(43, dims)
    eo = O.EO(U, 0.1, M5, Ls)
    phis = [O.heatbath_phi(U, I.gaussian_spinor(44, dims, Ls) * eo.even, m1, m2, M5, tol=1e-14) for m1, m2 in TERMS]
    H0 = O.hamiltonian(U, p, phis, TERMS, M5)
    cache = {}

    def traj(integrator, n):
        if (integrator, n) not in cache:
            Uc, pc, nf = O.md_trajectory(U, p, LENGTH / n, n, phis, TERMS, M5, integrator=integrator)
            cache[integrator, n] = (Uc, pc, nf, O.hamiltonian(Uc, pc, phis, TERMS, M5) - H0)
        return cache[integrator, n]

    return U, p, phis, traj


def test_omelyan_lambda_closed_form():
    # minimiser of the norm of the leading error terms of the 2MN scheme
    r = (2.0 * np.sqrt(326.0) + 36.0) ** (1.0 / 3.0)
    assert abs(O.OMELYAN_LAMBDA - (0.5 - r / 12.0 + 1.0 / (6.0 * r))) < 1e-15


@pytest.mark.parametrize("integrator,forces", [("fgi", 7), ("omelyan", 5)])
def test_trajectory_merges_end_momentum_updates(md, integrator, forces):
    U, p, phis, traj = md
    Ut, pt, nf, _ = traj(integrator, 2)
    assert nf == forces
    step = O.fgi_step if integrator == "fgi" else O.omelyan_step
    Us, ps = U, p
    for _ in range(2):
        Us, ps = step(Us, ps, LENGTH / 2, phis, TERMS, M5)
    assert np.abs(Ut - Us).max() < 1e-11
    assert np.abs(pt - ps).max() < 1e-11


def test_omelyan_dH_scales_as_tau2(md):
    *_, traj = md
    ratio = traj("omelyan", 4)[3] / traj("omelyan", 8)[3]
    assert 3.0 < ratio < 5.5, ratio


def test_fgi_error_far_below_omelyan_at_equal_step(md):
    *_, traj = md
    dh_fgi, dh_om = abs(traj("fgi", 4)[3]), abs(traj("omelyan", 4)[3])
    assert dh_fgi < dh_om / 10, (dh_fgi, dh_om)


def test_omelyan_trajectory_is_reversible(md):
    U, p, phis, traj = md
    U1, p1, _, _ = traj("omelyan", 2)
    U2, p2, _ = O.md_trajectory(U1, -p1, LENGTH / 2, 2, phis, TERMS, M5, integrator="omelyan")
    assert np.abs(U2 - U).max() < 1e-10
    assert np.abs(-p2 - p).max() < 1e-10


def test_metropolis_accept():
    assert O.metropolis_accept(-3.0, 0.999)          # dH <= 0: always
    assert O.metropolis_accept(0.0, 0.999)
    assert O.metropolis_accept(np.log(2.0), 0.49)    # exp(-dH) = 1/2
    assert not O.metropolis_accept(np.log(2.0), 0.51)
    assert not O.metropolis_accept(800.0, 0.0)       # exp(-800) underflows to 0: reject
    with pytest.raises(ValueError):
        O.md_trajectory(None, None, 0.1, 1, [], [], M5, integrator="leapfrog")
