"""Pins of the oracle's solvers, MADWF, force and force-gradient integrator
(CPU only).

  * CG on the normal equations reaches the dense LU solution of D(m) x = b.
  * MADWF (Sec. 4, four steps; Sec. 5 defect correction):
      - Eq. (recon) returns the exact solution when fed the exact y_1;
      - Eq. (mob_eq_5d): (P^-1 D'(m)^-1 D'(1) P c')_1 = D'_OV(m)^-1 c_1 (dense);
      - with the Moebius operator equal to the DWF one (b=1, c=0, Ls'=Ls) one
        MADWF pass is an exact solver;
      - the cost is two Pauli-Villars and one Moebius solve per pass (Sec. 4);
      - defect correction shrinks the residual pass by pass (Sec. 5).
  * Force (Sec. 2): central finite differences of the action along
    e^{h T_j} U_mu(n), with Richardson extrapolation; F traceless-antihermitian.
  * Heatbath: S(phi) = |eta|^2 exactly (Sec. 3 quotient action).
  * su(3) exponential against scipy's expm.
  * Force-gradient step (Sec. 2, Eqs. 1-6): reversibility with forecasting on,
    the O(tau^4) error of the exponential rewrite of Eq. (fg_approx), and
    dH over a fixed trajectory scaling as tau^4.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import dwf_oracle as O
from paper_1111_5059_gb300 import inputs as I

M5 = 1.8


def _src(seed, dims, Ls):
    return I.gaussian_spinor(seed, dims, Ls)


@pytest.mark.parametrize("bc", [(1.0, 0.0), (1.5, 0.5)])
def test_cg_matches_dense_lu(bc):
    b5, c5 = bc
    dims, Ls, m = (2, 2, 2, 4), 4, 0.04
    U = I.gauge_field(1, dims, 0.3)
    src = _src(1, dims, Ls)
    x, it, res = O.solve(U, src, m, M5, b5, c5, tol=1e-13)
    D = O.dense_matrix(lambda v: O.dwf_op(U, v, m, M5, b5, c5), src.shape)
    xd = np.linalg.solve(D, src.ravel()).reshape(src.shape)
    assert res <= 1e-13
    assert np.abs(x - xd).max() / np.abs(xd).max() < 1e-11
    assert it > 0


def test_config1_solve_residual():
    """4^4 x Ls=8, m_f = 0.04, eps = 0.3: the plain solve reaches 1e-12."""
    dims, Ls, m = (4, 4, 4, 4), 8, 0.04
    U = I.gauge_field(1, dims, 0.3)
    src = _src(1, dims, Ls)
    x, it, res = O.solve(U, src, m, M5, tol=1e-12)
    assert res <= 1e-12
    r = src - O.dwf_op(U, x, m, M5)
    assert np.sqrt(O.norm2(r) / O.norm2(src)) <= 1e-12


def _dense_setup(dims, Ls, m, b=1.0, c=0.0, seed=31):
    U = I.gauge_field(seed, dims, 0.6)
    shape = (Ls,) + (dims[3], dims[2], dims[1], dims[0]) + (4, 3)
    D = O.dense_matrix(lambda v: O.dwf_op(U, v, m, M5, b, c), shape)
    D1 = O.dense_matrix(lambda v: O.dwf_op(U, v, 1.0, M5, b, c), shape)
    P = O.dense_matrix(O.P_op, shape)
    Pi = O.dense_matrix(O.Pinv_op, shape)
    return U, shape, D, D1, P, Pi


def test_recon_exact_with_exact_y1():
    dims, Ls, m = (2, 2, 2, 2), 4, 0.05
    U, shape, D, D1, P, Pi = _dense_setup(dims, Ls, m)
    rng = np.random.default_rng(0)
    b = rng.standard_normal(D.shape[0]) + 1j * rng.standard_normal(D.shape[0])
    x = np.linalg.solve(D, b)
    c = (Pi @ np.linalg.solve(D1, b)).reshape(shape)
    y = (Pi @ x).reshape(shape)
    w = c.copy()
    w[0] = -y[0]
    u = (Pi @ np.linalg.solve(D1, D @ (P @ w.ravel()))).reshape(shape)
    yr = u.copy()
    yr[0] = y[0]
    xr = P @ yr.ravel()
    assert np.abs(xr - x).max() / np.abs(x).max() < 1e-12
    # and the first slice of u is -D_OV y_1 (left side of Eq. recon)
    K = Pi @ np.linalg.solve(D1, D @ P)
    n4 = 16 * 12
    assert np.abs(u[0].ravel() + K[:n4, :n4] @ y[0].ravel()).max() < 1e-11


@pytest.mark.parametrize("bcL", [(11 / 6, 5 / 6, 3), (1.5, 0.5, 2)])
def test_mobius_5d_form_gives_4d_solution(bcL):
    b, c, Lp = bcL
    dims, m = (2, 2, 2, 2), 0.05
    U, shape, Dm, D1m, P, Pi = _dense_setup(dims, Lp, m, b, c)
    rng = np.random.default_rng(2)
    c1 = rng.standard_normal((2, 2, 2, 2, 4, 3)) + 1j * rng.standard_normal((2, 2, 2, 2, 4, 3))
    cp = np.zeros(shape, dtype=np.complex128)
    cp[0] = c1
    z = np.linalg.solve(Dm, D1m @ (P @ cp.ravel()))
    y1 = (Pi @ z).reshape(shape)[0]
    DW = O.dense_matrix(lambda v: O.wilson_op(U, v[None], M5)[0], (2, 2, 2, 2, 4, 3))
    g5 = np.kron(np.eye(16), np.kron(O.GAMMA5, np.eye(3)))
    Dov = O.d_ov_closed_form(DW, g5, m, Lp, b, c)
    assert np.abs(Dov @ y1.ravel() - c1.ravel()).max() < 1e-11


def test_madwf_exact_when_mobius_equals_dwf():
    dims, Ls, m = (4, 2, 2, 4), 4, 0.05
    U = I.gauge_field(4, dims, 0.5)
    src = _src(4, dims, Ls)
    x, info = O.madwf(U, src, m, M5, Ls, 1.0, 0.0, n_dc=1, tol_pv=1e-13, tol_mob=1e-13,
                      final=False)
    assert info["passes"][0] < 1e-11
    assert info["pv_solves"] == 2 and info["mob_solves"] == 1


def test_madwf_defect_correction_and_final_solve():
    """Shamir Ls=8 through Moebius Ls'=4 with b-c=1, b+c=Ls/Ls'=2 (b=1.5, c=0.5)."""
    dims, Ls, m = (4, 4, 2, 2), 8, 0.02
    U = I.gauge_field(8, dims, 0.5)
    src = _src(8, dims, Ls)
    x, info = O.madwf(U, src, m, M5, 4, 1.5, 0.5, n_dc=3, tol_pv=1e-12, tol_mob=1e-12,
                      tol_final=1e-12)
    p = info["passes"]
    assert p[0] < 0.5 and p[1] < p[0] and p[2] < p[1]
    assert info["pv_solves"] == 6 and info["mob_solves"] == 3
    assert info["final_res"] <= 1e-12
    r = src - O.dwf_op(U, x, m, M5)
    assert np.sqrt(O.norm2(r) / O.norm2(src)) <= 1e-12


# ---------------------------------------------------------------- force


def _action(U, phi, m1, m2, tol=1e-14):
    return O.quotient_solution(U, phi, m1, m2, M5, tol=tol)[2]


def _perturb(U, mu, site, j, h):
    Up = U.copy()
    Up[(mu,) + site] = scipy.linalg.expm(h * O.T_GEN[j]) @ U[(mu,) + site]
    return Up


def test_heatbath_action_equals_eta_norm():
    dims, Ls = (4, 2, 2, 4), 4
    U = I.gauge_field(14, dims, 0.5)
    eo = O.EO(U, 0.1, M5, Ls)
    eta = _src(15, dims, Ls) * eo.even
    phi = O.heatbath_phi(U, eta, 0.1, 1.0, M5, tol=1e-14)
    S = _action(U, phi, 0.1, 1.0)
    assert abs(S - O.norm2(eta)) / O.norm2(eta) < 1e-11


@pytest.mark.parametrize("masses", [(0.1, 1.0), (0.05, 0.3)])
def test_force_matches_finite_differences(masses):
    m1, m2 = masses
    dims, Ls = (4, 2, 2, 4), 4
    U = I.gauge_field(16, dims, 0.5)
    eo = O.EO(U, m1, M5, Ls)
    phi = _src(17, dims, Ls) * eo.even
    X, Y, S, _ = O.quotient_solution(U, phi, m1, m2, M5, tol=1e-14)
    F = O.quotient_force(U, X, Y, phi, m1, m2, M5)
    rng = np.random.default_rng(9)
    for _ in range(6):
        mu = int(rng.integers(4))
        site = (int(rng.integers(4)), int(rng.integers(2)), int(rng.integers(2)), int(rng.integers(4)))
        j = int(rng.integers(8))
        h = 1e-3
        d1 = (_action(_perturb(U, mu, site, j, h), phi, m1, m2)
              - _action(_perturb(U, mu, site, j, -h), phi, m1, m2)) / (2 * h)
        d2 = (_action(_perturb(U, mu, site, j, h / 2), phi, m1, m2)
              - _action(_perturb(U, mu, site, j, -h / 2), phi, m1, m2)) / h
        fd = (4 * d2 - d1) / 3
        assert abs(fd - F[(mu,) + site + (j,)]) < 1e-7 * (1 + np.abs(F).max())
    Fm = O.algebra_matrix(F)
    assert np.abs(Fm + O.dagger(Fm)).max() < 1e-13
    assert np.abs(np.trace(Fm, axis1=-2, axis2=-1)).max() < 1e-13


def test_quotient_force_vanishes_for_equal_masses_and_grows_linearly():
    """Sec. 3: the quotient det(M(m1)^+ M(m1)) / det(M(m2)^+ M(m2)) is 1 for
    m1 = m2, so S = |phi|^2 whatever the links and the force is zero; for a
    split m2 = m1 + mu the force is proportional to mu at small mu."""
    dims, Ls, m = (4, 2, 2, 4), 4, 0.1
    U = I.gauge_field(18, dims, 0.5)
    eo = O.EO(U, m, M5, Ls)
    phi = _src(19, dims, Ls) * eo.even
    X, Y, S, _ = O.quotient_solution(U, phi, m, m, M5, tol=1e-14)
    assert abs(S - O.norm2(phi)) < 1e-11 * O.norm2(phi)
    assert np.abs(O.quotient_force(U, X, Y, phi, m, m, M5)).max() < 1e-10
    norms = []
    for mu in (1e-3, 2e-3):
        X, Y, _, _ = O.quotient_solution(U, phi, m, m + mu, M5, tol=1e-14)
        norms.append(np.abs(O.quotient_force(U, X, Y, phi, m, m + mu, M5)).max())
    assert 1.9 < norms[1] / norms[0] < 2.1, norms


def test_su3_exp_matches_expm():
    rng = np.random.default_rng(3)
    comp = rng.standard_normal((5, 8)) * 2
    Xm = O.algebra_matrix(comp)
    E = O.su3_exp(Xm)
    for k in range(5):
        assert np.abs(E[k] - scipy.linalg.expm(Xm[k])).max() < 1e-13
    assert np.abs(np.linalg.det(E) - 1).max() < 1e-13
    assert np.allclose(O.algebra_components(Xm), comp)


# ---------------------------------------------------------------- integrator

_TERMS = [(0.1, 0.4), (0.4, 1.0)]


def _hmc_setup(seed=40):
    dims, Ls = (4, 2, 2, 4), 4
    U = I.gauge_field(seed, dims, 0.5)
    p = I.gaussian_momenta(seed, dims)
    eo = O.EO(U, 0.1, M5, Ls)
    phis = [O.heatbath_phi(U, _src(seed + k + 1, dims, Ls) * eo.even, m1, m2, M5, tol=1e-14)
            for k, (m1, m2) in enumerate(_TERMS)]
    return U, p, phis


def test_fgi_reversibility_with_forecasting():
    U, p, phis = _hmc_setup()
    tau = 0.1
    U1, p1 = O.fgi_step(U, p, tau, phis, _TERMS, M5, tol=1e-13, forecast=True)
    U2, p2 = O.fgi_step(U1, -p1, tau, phis, _TERMS, M5, tol=1e-13, forecast=True)
    assert np.abs(U2 - U).max() < 1e-10
    assert np.abs(-p2 - p).max() < 1e-10


def test_fg_exponential_rewrite_error_is_tau4():
    """F(exp(-tau^2/24 F^j T_j) U) - [F - tau^2/24 F^j e_j F] = O(tau^4) (Eq. fg_approx)."""
    U, p, phis = _hmc_setup(41)
    _, F, _ = O.action_and_force(U, phis, _TERMS, M5, tol=1e-14)
    h = 1e-4
    Fp = O.action_and_force(O.link_update(U, F, h), phis, _TERMS, M5, tol=1e-14)[1]
    Fm = O.action_and_force(O.link_update(U, F, -h), phis, _TERMS, M5, tol=1e-14)[1]
    DF = (Fp - Fm) / (2 * h)
    errs = []
    for tau in (0.4, 0.2):
        Fg = O.action_and_force(O.link_update(U, F, -tau * tau / 24), phis, _TERMS, M5, tol=1e-14)[1]
        errs.append(np.abs(Fg - (F - tau * tau / 24 * DF)).max())
    ratio = errs[0] / errs[1]
    assert 12 < ratio < 20, (errs, ratio)


def test_dH_scales_as_tau4():
    """|dH| over a trajectory of length 1/2 drops by ~2^4 when the step halves."""
    U, p, phis = _hmc_setup(42)
    H0 = O.hamiltonian(U, p, phis, _TERMS, M5, tol=1e-13)
    dH = []
    for n in (2, 4):
        tau = 0.5 / n
        Uc, pc = U, p
        for _ in range(n):
            Uc, pc = O.fgi_step(Uc, pc, tau, phis, _TERMS, M5, tol=1e-13)
        dH.append(abs(O.hamiltonian(Uc, pc, phis, _TERMS, M5, tol=1e-13) - H0))
    ratio = dH[0] / dH[1]
    assert 12 < ratio < 20, (dH, ratio)


def _even_subspace(eo, shape):
    idx = np.flatnonzero(np.broadcast_to(eo.even, shape))

    def embed(v):
        full = np.zeros(int(np.prod(shape)), dtype=np.complex128)
        full[idx] = v
        return full.reshape(shape)

    return idx, embed


def test_quotient_action_is_the_determinant_ratio():
    """Sec. 3: a quotient term (m1, m2) stands for det(M2^+ M2) / det(M1^+ M1).
    The oracle's action S(phi) = |Y|^2 with Y = M1 X, X = (M1^+ M1)^-1 M2^+ phi
    (quotient_solution) is the Gaussian form phi^+ W^+ W phi of the linear map
    W : phi -> Y; integrating exp(-S) over phi gives det(W^+ W)^-1, so
    |det W|^2 must equal |det M2|^2 / |det M1|^2, M = M_pc on the even
    subspace (dense, from the oracle's operator).  A Hasenbusch ladder's terms
    multiply to the ratio of its end masses (the telescoping of Sec. 3)."""
    dims, Ls = (2, 2, 2, 2), 4
    U = I.gauge_field(31, dims, 0.6)
    shape = (Ls,) + tuple(reversed(dims)) + (4, 3)
    eo_any = O.EO(U, 0.1, M5, Ls)
    idx, embed = _even_subspace(eo_any, shape)
    n = idx.size

    def dense_M(m):
        eo = O.EO(U, m, M5, Ls)
        return np.stack([eo.Mpc(embed(np.eye(1, n, j, dtype=np.complex128)[0])).ravel()[idx] for j in range(n)], 1)

    def logdet2_W(m1, m2):
        M1 = dense_M(m1)
        N1 = M1.conj().T @ M1

        def solve_normal(eo, v):  # dense (M1^+ M1)^-1 on the even subspace
            return embed(np.linalg.solve(N1, v.ravel()[idx]))

        cols = []
        for j in range(n):
            phi = embed(np.eye(1, n, j, dtype=np.complex128)[0])
            _, Y, _, _ = O.quotient_solution(U, phi, m1, m2, M5, dense=solve_normal)
            cols.append(Y.ravel()[idx])
        return 2 * np.linalg.slogdet(np.stack(cols, 1))[1]

    def logdet2_M(m):
        return 2 * np.linalg.slogdet(dense_M(m))[1]

    ladder = [0.02, 0.2, 1.0]
    terms = [logdet2_W(a, b) for a, b in zip(ladder, ladder[1:])]
    for (a, b), t in zip(zip(ladder, ladder[1:]), terms):
        assert t == pytest.approx(logdet2_M(b) - logdet2_M(a), abs=1e-8)
    assert sum(terms) == pytest.approx(logdet2_M(1.0) - logdet2_M(0.02), abs=1e-8)
    # a swapped term (M1 and M2 exchanged) would give the inverse ratio
    assert abs(terms[0] - (logdet2_M(0.02) - logdet2_M(0.2))) > 1.0
