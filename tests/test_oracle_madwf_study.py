"""The oracle's MADWF against the paper's qualitative findings (CPU only):
Shamir 4^2 x 2^2 x Ls=8, m = 0.02, through Moebius Ls'=4, one defect-correction
pass.

  * Fig. 1: the Moebius operator approximates the DWF one only up to a
    floor.  Solving the Moebius equation more accurately lowers the residual
    of the MADWF guess (and the iterations of the final DWF solve started
    from it) until that floor; beyond the turning point more Moebius
    iterations buy nothing.
  * The Moebius scale: with b - c = 1, the floor is lowest at
    b + c = Ls / Ls' (the reading of the paper's parameters for the Ls=32 ->
    Ls'=12 workload, corroborated by Fig. 1's L=32, L'=16, b=1.5, c=0.5).
"""
import numpy as np
import pytest

from oracle import dwf_oracle as O
from paper_1111_5059_gb300 import inputs as I

M5 = 1.8
DIMS, LS, LSP, MASS = (4, 4, 2, 2), 8, 4, 0.02


@pytest.fixture(scope="module")
def case():
    return I.gauge_field(8, DIMS, 0.5), I.gaussian_spinor(8, DIMS, LS)


def _one_pass(U, src, b, c, tol_mob, final):
    _, info = O.madwf(U, src, MASS, M5, LSP, b, c, n_dc=1, tol_pv=1e-12, tol_mob=tol_mob, tol_final=1e-10,
                      final=final)
    return info


def test_fig1_turning_point(case):
    U, src = case
    runs = {t: _one_pass(U, src, 1.5, 0.5, t, final=t in (1e-1, 1e-4, 1e-8)) for t in (1e-1, 1e-2, 1e-4, 1e-8)}
    res = {t: r["passes"][0] for t, r in runs.items()}
    mob = {t: r["mob_iters"] for t, r in runs.items()}
    # more Moebius iterations for tighter tolerances
    assert mob[1e-1] < mob[1e-2] < mob[1e-4] < mob[1e-8]
    # before the turning point the guess improves with the Moebius accuracy ...
    assert res[1e-2] < res[1e-1] / 4 and res[1e-4] < res[1e-2] / 2
    # ... after it the guess stays at the approximation's floor
    assert abs(res[1e-8] - res[1e-4]) < 0.01 * res[1e-8]
    assert res[1e-8] > 1e-4  # the floor is the operators' difference, far above the solve tolerance
    # the final DWF solve follows: fewer iterations from a better guess, none saved past the floor
    fin = {t: runs[t]["final_iters"] for t in (1e-1, 1e-4, 1e-8)}
    assert fin[1e-4] < 0.85 * fin[1e-1]
    assert abs(fin[1e-8] - fin[1e-4]) <= 0.05 * fin[1e-4]


def test_floor_lowest_at_b_plus_c_equal_Ls_over_Lsprime(case):
    U, src = case
    floor = {}
    for al in (1.5, LS / LSP, 3.0):
        floor[al] = _one_pass(U, src, (al + 1) / 2, (al - 1) / 2, 1e-12, final=False)["passes"][0]
    best = floor[LS / LSP]
    assert best < floor[1.5] / 5 and best < floor[3.0] / 5, floor
