"""Hybrid Monte Carlo updates built on the library's trajectories (Sec. 2).

One update at gauge field U: draw Gaussian momenta p and, for each quotient
term (m1, m2), a Gaussian eta; set the pseudofermion phi = M2^-+ M1^+ eta by
the heat bath (dwf_heatbath), so that the term's action starts at |eta_e|^2;
integrate one molecular-dynamics trajectory (dwf_md_trajectory: the
force-gradient or the Omelyan 2MN integrator, merged end updates); accept
the new links with probability min(1, exp(-dH)), else keep U.

This module is host control flow: every field operation runs in the
library's kernels, and the random numbers come from the seeded
counter-based streams of inputs.py (update k of a chain uses seed k; term i's
eta is stream STREAM_ETA0 + i, the accept/reject uniform stream
STREAM_NOISE).
"""
from __future__ import annotations

import math

import torch

from . import dwf, inputs

STREAM_ETA0 = 100


def draw(seed: int, dims, Ls: int, nterms: int):
    """The update's random numbers: momenta [4][T][Z][Y][X][8], one eta per
    term (boundary-layout spinors) and the accept/reject uniform in [0, 1)."""
    p = inputs.gaussian_momenta(seed, dims)
    etas = [inputs.gaussian_spinor(seed, dims, Ls, stream=STREAM_ETA0 + i) for i in range(nterms)]
    u = float(inputs.uniform(inputs.stream_key(seed, inputs.STREAM_NOISE), 0, 1)[0])
    return p, etas, u


def accept(dH: float, u: float) -> bool:
    """Metropolis: accept with probability min(1, exp(-dH))."""
    return dH <= 0.0 or u < math.exp(-dH)


def hmc_update(lat: dwf.Lattice, U: torch.Tensor, terms, tau: float, nsteps: int, seed: int, integrator="fgi",
               tol=1e-10, inner="f32", delta=1e-4):
    """One HMC update of the device links U (boundary layout, updated in place
    on acceptance; the lattice's gauge field is left at the resulting U).
    Returns a dict with the decision, dH, H0, the uniform, CG iterations and
    force evaluations."""
    dev = U.device
    p, etas, u = draw(seed, lat.dims, lat.Ls, len(terms))
    lat.set_gauge(U)
    phis = [dwf.heatbath(lat, t, torch.from_numpy(e).to(dev), tol=tol, inner=inner, delta=delta)[0]
            for t, e in zip(terms, etas)]
    U1 = U.clone()
    pt = torch.from_numpy(p).to(dev)
    H0, H1, st, nf = dwf.md_trajectory(lat, terms, phis, U1, pt, tau, nsteps, integrator=integrator, tol=tol,
                                       inner=inner, delta=delta)
    dH = H1 - H0
    ok = accept(dH, u)
    if ok:
        U.copy_(U1)
    lat.set_gauge(U)
    return {"accept": ok, "dH": dH, "H0": H0, "u": u, "cg_iters": st["iters"], "force_evaluations": nf}
