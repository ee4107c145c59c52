"""GPU pseudofermion action, fermion force and force-gradient integrator
(Sec. 2 and 3) through the C ABI, against the FP64 oracle.

  * S and F^j = e_j S of two Hasenbusch quotient terms equal the oracle's to
    1e-9 relative (the oracle solves for X with its own CG).
  * The complex-matrix gradient G = 2 dS/d conj(U) matches central finite
    differences of the GPU action along a random complex direction, and its
    projection on the Lie algebra reproduces F (Re tr(G^+ T_j U) = F^j).
  * torch.autograd through QuotientAction returns G.
  * fgi_link_update equals the oracle's exp (eigh) update.
  * One FGI PQPQP step equals the oracle's step; it is reversible (p -> -p)
    to solver precision, and force-gradient forecasting (Sec. 2) reduces the
    iterations of the second solve.
  * At 16^3 x 8 x Ls=16 (the force workload's size): the GPU's solutions X
    by the oracle's operator, S and F against the oracle's formulas on those
    X to 1e-9; finite differences of the GPU action along a random direction
    against the force, and reversibility of one step.
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
    U = I.gauge_field(40, dims, 0.5)
    eo = O.EO(U, 0.1, M5, Ls)
    phis = [O.heatbath_phi(U, I.gaussian_spinor(41 + k, dims, Ls) * eo.even, m1, m2, M5, tol=1e-14)
            for k, (m1, m2) in enumerate(TERMS)]
    p = I.gaussian_momenta(40, dims)
    lat = dwf.Lattice(dims, Ls, M5)
    lat.set_gauge(_to(U))
    yield lat, U, phis, p
    lat.close()


def test_action_and_force_match_oracle(small, dwf):
    lat, U, phis, p = small
    S, F, _, st = dwf.force(lat, TERMS, [_to(x) for x in phis], tol=1e-13)
    So, Fo, _ = O.action_and_force(U, phis, TERMS, M5, tol=1e-14)
    assert abs(S - So) / So < 1e-11
    # the action-only entry point runs the same solves
    assert abs(dwf.action_value(lat, TERMS, [_to(x) for x in phis], tol=1e-13) - S) <= 1e-14 * abs(S)
    Fg = F.cpu().numpy()
    assert np.abs(Fg - Fo).max() / np.abs(Fo).max() < 1e-9
    assert st["iters"] > 0


def test_matrix_gradient_fd_and_lie_projection(small, dwf):
    lat, U, phis, p = small
    phit = [_to(x) for x in phis]
    Ut = _to(U)
    lat.set_gauge(Ut)
    S0, F, G, _ = dwf.force(lat, TERMS, phit, want_grad=True, tol=1e-14)
    rng = np.random.default_rng(5)
    d = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    h = 1e-5
    vals = []
    for sgn in (+1, -1):
        lat.set_gauge(_to(U + sgn * h * d))
        vals.append(dwf.force(lat, TERMS, phit, want_force=False, tol=1e-14)[0])
    fd = (vals[0] - vals[1]) / (2 * h)
    lin = float(np.sum((np.conj(G.cpu().numpy()) * d).real))
    assert abs(fd - lin) < 1e-6 * (1 + abs(lin))
    # Lie derivative along T_j U from G:  Re tr(G^+ T_j U) = F^j
    Gm = G.cpu().numpy()
    proj = np.einsum("...ba,jbc,...ca->...j", np.conj(Gm), O.T_GEN, U).real
    assert np.abs(proj - F.cpu().numpy()).max() < 1e-10 * (1 + np.abs(proj).max())
    lat.set_gauge(Ut)


def test_autograd_returns_matrix_gradient(small, dwf):
    lat, U, phis, p = small
    Ut = _to(U).requires_grad_(True)
    S = dwf.action(lat, Ut, TERMS, [_to(x) for x in phis], tol=1e-13)
    (g,) = torch.autograd.grad(S, Ut)
    _, _, G, _ = dwf.force(lat, TERMS, [_to(x) for x in phis], want_force=False, want_grad=True, tol=1e-13)
    assert torch.allclose(g, G, rtol=1e-9, atol=1e-12)
    So = O.action_and_force(U, phis, TERMS, M5, tol=1e-14)[0]
    assert abs(S.item() - So) / So < 1e-11


def test_link_update_matches_oracle(small, dwf):
    lat, U, phis, p = small
    for coeff in (0.05, -0.1 ** 2 / 24, 1.3):
        got = dwf.fgi_link_update(lat, _to(p), coeff, _to(U)).cpu().numpy()
        want = O.link_update(U, p, coeff)
        assert np.abs(got - want).max() < 1e-13
        assert np.abs(np.linalg.det(got) - 1).max() < 1e-13


def test_fgi_step_matches_oracle_and_is_reversible(small, dwf):
    lat, U, phis, p = small
    tau = 0.1
    phit = [_to(x) for x in phis]
    Ut, pt = _to(U), _to(p)
    st, fg = dwf.fgi_step(lat, TERMS, phit, Ut, pt, tau, forecast=True, tol=1e-13)
    Uo, po = O.fgi_step(U, p, tau, phis, TERMS, M5, tol=1e-14)
    assert np.abs(Ut.cpu().numpy() - Uo).max() < 1e-10
    assert np.abs(pt.cpu().numpy() - po).max() < 1e-9
    assert fg[1] < fg[0]  # forecasting: the U' solve starts from the U solution
    pt.neg_()
    dwf.fgi_step(lat, TERMS, phit, Ut, pt, tau, forecast=True, tol=1e-13)
    assert np.abs(Ut.cpu().numpy() - U).max() < 1e-10
    assert np.abs(-pt.cpu().numpy() - p).max() < 1e-9
    lat.set_gauge(_to(U))


def test_force_workload_size_matches_oracle(dwf):
    """16^3 x 8 x Ls=16 with quotient terms (0.01, 0.1) and (0.1, 1.0): the
    GPU's solutions X are checked by the oracle's operator (|M2^+ phi -
    M1^+ M1 X| <= 1e-12 |M2^+ phi|, the solve's target), and the GPU's S and F against the
    oracle's action and force evaluated on those same X (Sec. 2: F^j = e_j S),
    F to 1e-9 relative to its largest component.  The residual bar allows
    1.5x the solve's target for the rounding of M1^+ M1 X in FP64, which the
    library's and the oracle's evaluations do in different orders."""
    dims, Ls = (16, 16, 16, 8), 16
    terms = [(0.01, 0.1), (0.1, 1.0)]
    U = I.gauge_field(4, dims, 0.5)
    lat = dwf.Lattice(dims, Ls, M5)
    lat.set_gauge(_to(U))
    eta = [I.gaussian_spinor(50 + k, dims, Ls) for k in range(2)]
    phit = [_to(e) for e in eta]
    Xs = [torch.zeros_like(p) for p in phit]
    S, F, _, _ = dwf.force(lat, terms, phit, X_io=Xs, tol=1e-12)
    lat.close()
    Fo = np.zeros(F.shape)
    So = 0.0
    for (m1, m2), phi, Xt in zip(terms, eta, Xs):
        X = Xt.cpu().numpy()
        eo1, eo2 = O.EO(U, m1, M5, Ls), O.EO(U, m2, M5, Ls)
        v = eo2.Mpc(phi * eo2.even, True)
        Y = eo1.Mpc(X)
        res = np.sqrt(O.norm2(v - eo1.Mpc(Y, True)) / O.norm2(v))
        assert res <= 1.5e-12, (m1, m2, res)
        So += O.norm2(Y)
        Fo += O.quotient_force(U, X, Y, phi * eo2.even, m1, m2, M5)
    assert abs(S - So) <= 1e-11 * So
    Fg = F.cpu().numpy()
    assert np.abs(Fg - Fo).max() <= 1e-9 * np.abs(Fo).max()


def test_force_workload_size_properties(dwf):
    """16^3 x 8 x Ls=16 with quotient terms (0.01, 0.1) and (0.1, 1.0)."""
    dims, Ls = (16, 16, 16, 8), 16
    terms = [(0.01, 0.1), (0.1, 1.0)]
    U = I.gauge_field(4, dims, 0.5)
    p = I.gaussian_momenta(4, dims)
    lat = dwf.Lattice(dims, Ls, M5)
    Ut = _to(U)
    lat.set_gauge(Ut)
    eta = [I.gaussian_spinor(50 + k, dims, Ls) for k in range(2)]
    phit = [_to(e) for e in eta]  # a Gaussian phi (only even sites enter)
    S0, F, G, _ = dwf.force(lat, terms, phit, want_grad=True, tol=1e-12)
    # finite differences of S along exp(h omega^j T_j) U for a random omega
    rng = np.random.default_rng(1)
    om = _to(rng.standard_normal(tuple(F.shape)))
    h = 1e-4
    vals = []
    for sgn in (+1, -1):
        lat.set_gauge(dwf.fgi_link_update(lat, om, sgn * h, Ut))
        vals.append(dwf.force(lat, terms, phit, want_force=False, tol=1e-13)[0])
    fd = (vals[0] - vals[1]) / (2 * h)
    lin = float(torch.sum(F * om).item())
    assert abs(fd - lin) < 1e-5 * abs(lin)
    # reversibility of one step (tau = 0.1) at this size, in mixed precision
    lat.set_gauge(Ut)
    U1, p1 = Ut.clone(), _to(p)
    H0 = dwf.hamiltonian(lat, terms, phit, U1, p1)
    dwf.fgi_step(lat, terms, phit, U1, p1, 0.1, tol=1e-11, inner="f32")
    H1 = dwf.hamiltonian(lat, terms, phit, U1, p1)
    assert abs(H1 - H0) < 1e-2 * abs(H0)
    p1.neg_()
    dwf.fgi_step(lat, terms, phit, U1, p1, 0.1, tol=1e-11, inner="f32")
    assert (U1 - Ut).abs().max().item() < 1e-8
    assert (p1 + _to(p)).abs().max().item() < 1e-7
    lat.close()


def test_heatbath_matches_oracle(small, dwf):
    """phi = M2^-+ M1^+ eta (dwf_heatbath) element by element against the
    oracle's heat bath, and the term's action at that field is |eta_e|^2."""
    lat, U, phis, _ = small
    dims, Ls = lat.dims, lat.Ls
    eta = I.gaussian_spinor(71, dims, Ls)
    for m1, m2 in TERMS:
        phi, st = dwf.heatbath(lat, (m1, m2), _to(eta), tol=1e-13)
        want = O.heatbath_phi(U, eta, m1, m2, M5, tol=1e-14)
        got = phi.cpu().numpy()
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
        assert st["iters"] > 0
        ee = eta * O.EO(U, m1, M5, Ls).even
        S = dwf.action_value(lat, [(m1, m2)], [phi], tol=1e-13)
        assert abs(S - O.norm2(ee)) <= 1e-10 * O.norm2(ee)


def test_heatbath_at_force_workload_size(dwf):
    """16^3 x 8 x Ls=16, terms (0.01, 0.1) and (0.1, 1): S(phi) = |eta_e|^2."""
    dims, Ls = (16, 16, 16, 8), 16
    U = I.gauge_field(4, dims, 0.5)
    lat = dwf.Lattice(dims, Ls, M5)
    lat.set_gauge(_to(U))
    eta = _to(I.gaussian_spinor(72, dims, Ls))
    for term in ((0.01, 0.1), (0.1, 1.0)):
        phi, _ = dwf.heatbath(lat, term, eta, tol=1e-12)
        S = dwf.action_value(lat, [term], [phi], tol=1e-12)
        e2 = float((eta.abs() ** 2 * _even_mask(dims, Ls)).sum())
        assert abs(S - e2) <= 1e-9 * e2, (S, e2)
    lat.close()


def _even_mask(dims, Ls):
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    m = ((x + y + z + t) % 2 == 0).astype(np.float64)
    return torch.from_numpy(np.broadcast_to(m[None, :, :, :, :, None, None], (Ls, T, Z, Y, X, 4, 3)).copy()).cuda()


def test_hasenbusch_ladder_tuning_balances_gpu_forces(dwf):
    """The tuning loop of the Hasenbusch ladder (Sec. 3) driven by GPU force
    norms of heat-bath pseudofermions: the tuned terms' RMS forces agree to
    10 %, the end masses stay put and the ladder stays ordered."""
    from paper_1111_5059_gb300 import hasenbusch as Hb

    dims, Ls, m = (4, 4, 4, 8), 8, 0.02
    lat = dwf.Lattice(dims, Ls, M5)
    lat.set_gauge(_to(I.gauge_field(9, dims, 0.5)))
    etas = [_to(I.gaussian_spinor(90 + i, dims, Ls)) for i in range(3)]

    def norms(ts):
        out = []
        for i, t in enumerate(ts):
            phi, _ = dwf.heatbath(lat, t, etas[i], tol=1e-11)
            _, F, _, _ = dwf.force(lat, [t], [phi], tol=1e-10)
            out.append(float((F * F).sum(dim=-1).mean().sqrt()))
        return out

    start = Hb.geometric_ladder(m, 2)
    ms, hist = Hb.tune_ladder(start, norms, iters=10, rtol=0.1)
    f = hist[-1][1]
    assert max(f) / min(f) < 1.1, hist
    assert ms[0] == m and ms[-1] == 1.0 and ms[0] < ms[1] < ms[2] < ms[3]
    lat.close()
