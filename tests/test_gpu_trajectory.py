"""Whole molecular-dynamics trajectories (Sec. 2) through dwf_md_trajectory,
against the FP64 oracle's md_trajectory.

  * Force-gradient (FGI) and Omelyan 2MN trajectories of a few steps on a small
    lattice with two Hasenbusch quotient terms: the final links and momenta
    equal the oracle's (the same merged end momentum updates), the number of
    force evaluations is 3 n + 1 (FGI) or 2 n + 1 (Omelyan), and H before and
    after equals the oracle's Hamiltonian.
  * Reversibility of an FGI trajectory with forecasting (p -> -p brings U and p
    back), at the small size and at 16^3 x 8 x Ls=16 (the force workload's size,
    quotient terms (0.01, 0.1) and (0.1, 1.0)).
  * At that size the FGI error is below Omelyan's at the same step, and the FGI
    |dH| falls by about 2^4 when the step is halved at fixed trajectory length
    (Sec. 2: a fourth-order integrator).
"""
import numpy as np
import pytest
import torch

from oracle import dwf_oracle as O
from paper_1111_5059_gb300 import inputs as I

pytestmark = pytest.mark.gpu

M5 = 1.8
TERMS = [(0.1, 0.4), (0.4, 1.0)]


def _to(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module")
def small(dwf):
    dims, Ls = (4, 2, 2, 4), 4
    U = I.gauge_field(60, dims, 0.5)
    eo = O.EO(U, 0.1, M5, Ls)
    phis = [O.heatbath_phi(U, I.gaussian_spinor(61 + k, dims, Ls) * eo.even, m1, m2, M5, tol=1e-14)
            for k, (m1, m2) in enumerate(TERMS)]
    p = I.gaussian_momenta(60, dims)
    lat = dwf.Lattice(dims, Ls, M5)
    lat.set_gauge(_to(U))
    yield lat, U, phis, p
    lat.close()


@pytest.mark.parametrize("integrator,nsteps", [("fgi", 2), ("omelyan", 3)])
def test_trajectory_matches_oracle(small, dwf, integrator, nsteps):
    lat, U, phis, p = small
    tau = 0.1
    Ut, pt = _to(U), _to(p)
    H0, H1, st, nf = dwf.md_trajectory(lat, TERMS, [_to(x) for x in phis], Ut, pt, tau, nsteps,
                                       integrator=integrator, tol=1e-13)
    Uo, po, no = O.md_trajectory(U, p, tau, nsteps, phis, TERMS, M5, tol=1e-14, integrator=integrator)
    assert nf == no == (3 * nsteps + 1 if integrator == "fgi" else 2 * nsteps + 1)
    assert np.abs(Ut.cpu().numpy() - Uo).max() < 1e-10
    assert np.abs(pt.cpu().numpy() - po).max() < 1e-9
    H0o = O.hamiltonian(U, p, phis, TERMS, M5, tol=1e-14)
    H1o = O.hamiltonian(Uo, po, phis, TERMS, M5, tol=1e-14)
    assert abs(H0 - H0o) <= 1e-11 * abs(H0o)
    assert abs(H1 - H1o) <= 1e-10 * abs(H1o)
    assert st["iters"] > 0
    lat.set_gauge(_to(U))


def test_fgi_trajectory_is_reversible(small, dwf):
    lat, U, phis, p = small
    phit = [_to(x) for x in phis]
    Ut, pt = _to(U), _to(p)
    dwf.md_trajectory(lat, TERMS, phit, Ut, pt, 0.1, 3, tol=1e-13)
    pt.neg_()
    dwf.md_trajectory(lat, TERMS, phit, Ut, pt, 0.1, 3, tol=1e-13)
    assert np.abs(Ut.cpu().numpy() - U).max() < 1e-10
    assert np.abs(-pt.cpu().numpy() - p).max() < 1e-9
    lat.set_gauge(_to(U))


def test_force_workload_trajectories(dwf):
    dims, Ls = (16, 16, 16, 8), 16
    terms = [(0.01, 0.1), (0.1, 1.0)]
    U = I.gauge_field(4, dims, 0.5)
    p = I.gaussian_momenta(4, dims)
    lat = dwf.Lattice(dims, Ls, M5)
    Ut = _to(U)
    lat.set_gauge(Ut)
    eta = [I.gaussian_spinor(50 + k, dims, Ls) for k in range(2)]
    phit = [_to(e) for e in eta]
    dH = {}
    for integ, tau, n in (("fgi", 0.2, 2), ("fgi", 0.1, 4), ("omelyan", 0.2, 2)):
        U1, p1 = Ut.clone(), _to(p)
        H0, H1, _, _ = dwf.md_trajectory(lat, terms, phit, U1, p1, tau, n, integrator=integ, tol=1e-12)
        dH[(integ, tau)] = H1 - H0
        if (integ, tau) == ("fgi", 0.2):
            # reversibility at this size
            p1.neg_()
            dwf.md_trajectory(lat, terms, phit, U1, p1, tau, n, integrator=integ, tol=1e-12)
            assert (U1 - Ut).abs().max().item() < 1e-9
            assert (p1 + _to(p)).abs().max().item() < 1e-8
    lat.close()
    # fourth order: halving the step at fixed length cuts |dH| by ~16 (8 to 32 allowed)
    ratio = abs(dH[("fgi", 0.2)]) / abs(dH[("fgi", 0.1)])
    assert 8.0 < ratio < 32.0, (dH, ratio)
    assert abs(dH[("fgi", 0.2)]) < abs(dH[("omelyan", 0.2)]), dH


def test_hmc_chain_matches_oracle(small, dwf):
    """Three HMC updates (heat bath, trajectory, Metropolis; Sec. 2) through
    hmc.hmc_update on the GPU against the same chain with the oracle's heat
    bath, trajectory, Hamiltonian and Metropolis rule, from the same random
    numbers: the same decisions, dH and links.  A long step makes rejections
    likely, so both branches are exercised."""
    from paper_1111_5059_gb300 import hmc

    lat, U, _, _ = small
    dims, Ls = lat.dims, lat.Ls
    Ut = _to(U)
    Uo = U.copy()
    decisions = []
    for seed in (11, 12, 13, 14):
        tau, n = 0.8, 1  # dH of 1.5-3: the chain accepts once and rejects three times
        r = hmc.hmc_update(lat, Ut, TERMS, tau, n, seed, tol=1e-13, inner="f64", delta=0.1)
        p, etas, u = hmc.draw(seed, dims, Ls, len(TERMS))
        phis = [O.heatbath_phi(Uo, e, m1, m2, M5, tol=1e-14) for e, (m1, m2) in zip(etas, TERMS)]
        H0 = O.hamiltonian(Uo, p, phis, TERMS, M5, tol=1e-14)
        U1, p1, _ = O.md_trajectory(Uo, p, tau, n, phis, TERMS, M5, tol=1e-14)
        dH = O.hamiltonian(U1, p1, phis, TERMS, M5, tol=1e-14) - H0
        ok = O.metropolis_accept(dH, u)
        assert r["accept"] == ok
        assert abs(r["dH"] - dH) <= 1e-9 * abs(H0), (r["dH"], dH)
        if ok:
            Uo = U1
        assert np.abs(Ut.cpu().numpy() - Uo).max() < 1e-10
        decisions.append(ok)
    lat.set_gauge(_to(U))
    assert len(set(decisions)) == 2, decisions  # both an acceptance and a rejection
