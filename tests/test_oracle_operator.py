"""Pins of the oracle's domain-wall operator against what the paper and the
mathematics fix (CPU only).

Each test is chosen so that a plausible slip in the oracle (a wrong hop
direction, a transposed link, a wrong projector, a misplaced wall or a wrong
P) fails it:
  * Dirac algebra identities of the chiral basis;
  * the free-field (unit-link) momentum-space closed form of D_W;
  * an explicit matrix-element assembly of D_W on a tiny lattice;
  * adjointness, gamma5 R5 hermiticity, gauge covariance;
  * Moebius(b=1, c=0) against the textbook Shamir form;
  * the even-odd Schur complement against the dense matrix;
  * the block structure of Eq. (ov_eq) (Sec. 4) and the closed form of its
    (1,1) block, the overlap-type operator with eps_L(H) (domain-wall/overlap
    literature cited by the paper as MD_trans, borici_2004).
"""
import itertools

import numpy as np
import pytest

from oracle import dwf_oracle as O
from paper_1111_5059_gb300 import inputs as I

M5 = 1.8


def _rand_spinor(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ---------------------------------------------------------------- algebra


def test_gamma_algebra():
    g, g5 = O.GAMMA, O.GAMMA5
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2 * (mu == nu) * np.eye(4))
            assert np.isclose(np.trace(g[mu] @ g[nu]), 4 * (mu == nu))
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))
    assert np.allclose(g5 @ g5, np.eye(4))
    for mu in range(4):
        assert np.allclose(g5 @ g[mu], -g[mu] @ g5)
    # tr(g5 g_a g_b g_c g_d) = 4 eps_abcd with eps_0123 = +1
    for perm in itertools.permutations(range(4)):
        sgn = np.linalg.det(np.eye(4)[list(perm)])
        val = np.trace(g5 @ g[perm[0]] @ g[perm[1]] @ g[perm[2]] @ g[perm[3]])
        assert np.isclose(val, 4 * sgn)
    assert np.allclose(O.P_PLUS @ O.P_MINUS, 0)
    assert np.allclose(O.P_PLUS + O.P_MINUS, np.eye(4))


def test_generators_normalisation():
    T = O.T_GEN
    for i in range(8):
        assert np.allclose(T[i], -T[i].conj().T)
        assert abs(np.trace(T[i])) < 1e-15
        for j in range(8):
            assert np.isclose(np.trace(T[i] @ T[j]), -0.5 * (i == j))
    # su(3) structure constant f_123 = 1: [T_1, T_2] = - f_123 T_3 with T = i lambda / 2
    assert np.allclose(T[0] @ T[1] - T[1] @ T[0], -T[2])


# ---------------------------------------------------------------- free field


def _shift_mats(Ls, m):
    """Fifth-dimension hops written out: up: s <- s+1 (wall -m), dn: s <- s-1 (wall -m)."""
    up = np.diag(np.ones(Ls - 1), 1)
    dn = np.diag(np.ones(Ls - 1), -1)
    up[Ls - 1, 0] = -m
    dn[0, Ls - 1] = -m
    return up, dn


@pytest.mark.parametrize("bc_t", [1, -1])
@pytest.mark.parametrize("bc", [(1.0, 0.0), (1.5, 0.5)])
def test_free_field_closed_form(bc_t, bc):
    """U = 1: a plane wave e^{ip.n} chi(s,spin) v maps to e^{ip.n} [D(p) chi] v with
    D_W(p) = i sum g_mu sin p_mu + sum (1 - cos p_mu) - M5."""
    b, c = bc
    dims = (4, 4, 4, 4)
    Ls, m = 4, 0.07
    X, Y, Z, T = dims
    U = np.zeros((4, T, Z, Y, X, 3, 3), dtype=np.complex128)
    U[...] = np.eye(3)
    rng = np.random.default_rng(7)
    t, z, y, x = O.coords(dims)
    up, dn = _shift_mats(Ls, m)
    I4, Is = np.eye(4), np.eye(Ls)
    Pp, Pm = np.diag([1, 1, 0, 0]), np.diag([0, 0, 1, 1])
    Q = np.kron(up, Pm) + np.kron(dn, Pp)          # (s,spin) x (s',spin')
    g = O.GAMMA
    kt_shift = 0.5 if bc_t == -1 else 0.0
    for k in itertools.product(range(4), repeat=4):
        p = 2 * np.pi * np.array([k[0], k[1], k[2], k[3] + kt_shift]) / np.array([X, Y, Z, T])
        DWp = sum(1j * g[mu] * np.sin(p[mu]) for mu in range(4)) + (np.sum(1 - np.cos(p)) - M5) * I4
        Dp = np.kron(Is, DWp) @ (b * np.eye(4 * Ls) + c * Q) + np.eye(4 * Ls) - Q
        chi = _rand_spinor(rng, (Ls, 4))
        v = _rand_spinor(rng, (3,))
        wave = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        psi = np.einsum("tzyx,si,a->stzyxia", wave, chi, v)
        out = O.dwf_op(U, psi, m, M5, b, c, bc_t)
        want = np.einsum("tzyx,si,a->stzyxia", wave, (Dp @ chi.reshape(-1)).reshape(Ls, 4), v)
        assert np.abs(out - want).max() < 1e-12


# ---------------------------------------------------------------- dense assembly


def _dense_wilson_elements(U, dims, bc_t):
    """D_W assembled element by element from its definition (explicit loops)."""
    X, Y, Z, T = dims
    N = X * Y * Z * T

    def idx(x, y, z, t):
        return ((t * Z + z) * Y + y) * X + x

    D = np.zeros((N, 4, 3, N, 4, 3), dtype=np.complex128)
    ext = (X, Y, Z, T)
    for (t, z, y, x) in itertools.product(range(T), range(Z), range(Y), range(X)):
        n = idx(x, y, z, t)
        D[n, :, :, n, :, :] += (4 - M5) * np.einsum("ij,ab->iajb", np.eye(4), np.eye(3))
        c = [x, y, z, t]
        for mu in range(4):
            f, bk = list(c), list(c)
            f[mu] += 1
            bk[mu] -= 1
            ph_f = -1.0 if (mu == 3 and bc_t == -1 and f[3] == T) else 1.0
            ph_b = -1.0 if (mu == 3 and bc_t == -1 and bk[3] == -1) else 1.0
            f = [f[i] % ext[i] for i in range(4)]
            bk = [bk[i] % ext[i] for i in range(4)]
            nf, nb = idx(*f), idx(*bk)
            Uf = U[mu, t, z, y, x]
            Ub = U[mu, bk[3], bk[2], bk[1], bk[0]].conj().T
            D[n, :, :, nf, :, :] += -0.5 * ph_f * np.einsum("ij,ab->iajb", np.eye(4) - O.GAMMA[mu], Uf)
            D[n, :, :, nb, :, :] += -0.5 * ph_b * np.einsum("ij,ab->iajb", np.eye(4) + O.GAMMA[mu], Ub)
    return D.reshape(N * 12, N * 12)


@pytest.mark.parametrize("bc_t", [1, -1])
def test_wilson_matches_element_assembly(bc_t):
    dims = (4, 2, 2, 4)
    U = I.gauge_field(3, dims, 0.6)
    X, Y, Z, T = dims
    Dd = O.dense_matrix(lambda v: O.wilson_op(U, v[None], M5, bc_t)[0], (T, Z, Y, X, 4, 3))
    De = _dense_wilson_elements(U, dims, bc_t)
    assert np.abs(Dd - De).max() < 1e-14


@pytest.mark.parametrize("bc", [(1.0, 0.0), (1.5, 0.5)])
@pytest.mark.parametrize("bc_t", [1, -1])
def test_adjoint_and_gamma5_hermiticity(bc, bc_t):
    b, c = bc
    dims, Ls, m = (2, 2, 2, 2), 4, 0.1
    U = I.gauge_field(11, dims, 0.6)
    shape = (Ls, 2, 2, 2, 2, 4, 3)
    D = O.dense_matrix(lambda v: O.dwf_op(U, v, m, M5, b, c, bc_t), shape)
    Dd = O.dense_matrix(lambda v: O.dwf_op(U, v, m, M5, b, c, bc_t, dag=True), shape)
    assert np.abs(Dd - D.conj().T).max() < 1e-14
    # Gamma5 = gamma5 R5 (R5: s -> Ls-1-s).  Gamma5 D B^-1 is hermitian; B = 1 for Shamir.
    G5 = O.dense_matrix(lambda v: O.spin_mul(O.GAMMA5, v[::-1]), shape)
    Bm = O.dense_matrix(lambda v: b * v + c * O.q_op(v, m), shape)
    H = G5 @ D @ np.linalg.inv(Bm)
    assert np.abs(H - H.conj().T).max() < 1e-13
    if c == 0.0:
        assert np.abs(G5 @ D - (G5 @ D).conj().T).max() < 1e-14


@pytest.mark.parametrize("bc", [(1.0, 0.0), (1.5, 0.5)])
def test_gauge_covariance(bc):
    b, c = bc
    dims, Ls, m = (4, 2, 2, 4), 4, 0.05
    U = I.gauge_field(5, dims, 0.6)
    G = I.gauge_transform(6, dims)
    UG = np.empty_like(U)
    for mu in range(4):
        UG[mu] = G @ U[mu] @ O.dagger(O.shift(G, mu, +1, 0))
    rng = np.random.default_rng(1)
    psi = _rand_spinor(rng, (Ls,) + (dims[3], dims[2], dims[1], dims[0]) + (4, 3))
    Gpsi = np.einsum("...ab,s...ib->s...ia", G, psi)
    lhs = O.dwf_op(UG, Gpsi, m, M5, b, c, bc_t=-1)
    rhs = np.einsum("...ab,s...ib->s...ia", G, O.dwf_op(U, psi, m, M5, b, c, bc_t=-1))
    assert np.abs(lhs - rhs).max() < 1e-12


def test_mobius_b1_c0_is_textbook_shamir():
    dims, Ls, m = (4, 4, 2, 2), 6, 0.03
    U = I.gauge_field(2, dims, 0.6)
    rng = np.random.default_rng(3)
    psi = _rand_spinor(rng, (Ls, 2, 2, 4, 4, 4, 3))
    Pp = np.diag([1.0, 1, 0, 0])
    Pm = np.diag([0.0, 0, 1, 1])
    DW = O.wilson_op(U, psi, M5)
    want = DW + psi
    for s in range(Ls):
        if s + 1 < Ls:
            want[s] -= O.spin_mul(Pm, psi[s + 1])
        else:
            want[s] += m * O.spin_mul(Pm, psi[0])
        if s >= 1:
            want[s] -= O.spin_mul(Pp, psi[s - 1])
        else:
            want[s] += m * O.spin_mul(Pp, psi[Ls - 1])
    got = O.dwf_op(U, psi, m, M5, 1.0, 0.0)
    assert np.array_equal(got, O.dwf_op(U, psi, m, M5))
    assert np.abs(got - want).max() < 1e-13


@pytest.mark.parametrize("bc", [(1.0, 0.0), (1.5, 0.5)])
def test_pointwise_matches_whole_lattice(bc):
    b, c = bc
    dims, Ls, m = (4, 2, 4, 2), 5, 0.2
    U = I.gauge_field(9, dims, 0.5)
    rng = np.random.default_rng(4)
    psi = _rand_spinor(rng, (Ls, 2, 4, 2, 4, 4, 3))
    full = O.dwf_op(U, psi, m, M5, b, c, bc_t=-1)
    sites = [tuple(int(v) for v in (rng.integers(Ls), rng.integers(2), rng.integers(4),
                                    rng.integers(2), rng.integers(4))) for _ in range(20)]
    sites += [(0, 0, 0, 0, 0), (Ls - 1, 1, 3, 1, 3)]
    got = O.dwf_op_at(U, psi, m, M5, b, c, -1, sites)
    want = np.array([full[s] for s in sites])
    assert np.abs(got - want).max() < 1e-13


# ---------------------------------------------------------------- even-odd


@pytest.mark.parametrize("bc", [(1.0, 0.0), (1.5, 0.5)])
def test_even_odd_schur_complement(bc):
    b, c = bc
    dims, Ls, m = (2, 2, 2, 4), 4, 0.1
    U = I.gauge_field(12, dims, 0.6)
    shape = (Ls, 4, 2, 2, 2, 4, 3)
    D = O.dense_matrix(lambda v: O.dwf_op(U, v, m, M5, b, c), shape)
    eo = O.EO(U, m, M5, Ls, b, c)
    ev = np.broadcast_to(eo.even, shape).ravel()
    od = ~ev
    Dee, Deo, Doe, Doo = D[np.ix_(ev, ev)], D[np.ix_(ev, od)], D[np.ix_(od, ev)], D[np.ix_(od, od)]
    schur = Dee - Deo @ np.linalg.solve(Doo, Doe)
    Mpc = O.dense_matrix(lambda v: eo.Mpc(v * eo.even), shape)[np.ix_(ev, ev)]
    MpcD = O.dense_matrix(lambda v: eo.Mpc(v * eo.even, True), shape)[np.ix_(ev, ev)]
    assert np.abs(Mpc - schur).max() < 1e-13
    assert np.abs(MpcD - schur.conj().T).max() < 1e-13
    # the diagonal blocks carry no links: D_ee = A
    A = O.dense_matrix(lambda v: eo.A(v * eo.even), shape)[np.ix_(ev, ev)]
    assert np.abs(Dee - A).max() < 1e-14


# ---------------------------------------------------------------- DW -> overlap


def test_P_shifts_half_the_spin_components():
    """P moves the P+ half of the spinor by one slice in s and leaves P- in place."""
    rng = np.random.default_rng(5)
    y = _rand_spinor(rng, (5, 2, 2, 2, 2, 4, 3))
    Py = O.P_op(y)
    assert np.array_equal(Py[:, ..., 2:, :], y[:, ..., 2:, :])
    assert np.array_equal(Py[:, ..., :2, :], np.roll(y, -1, axis=0)[:, ..., :2, :])
    assert np.abs(O.Pinv_op(Py) - y).max() == 0
    assert np.abs(O.P_op(O.Pinv_op(y)) - y).max() == 0


@pytest.mark.parametrize("bcL", [(1.0, 0.0, 4), (1.5, 0.5, 4), (11 / 6, 5 / 6, 3)])
@pytest.mark.parametrize("bc_t", [1, -1])
def test_ov_eq_block_structure_and_closed_form(bcL, bc_t):
    """P^-1 D(1)^-1 D(m) P is identity outside its first block column (Eq. ov_eq);
    its (1,1) block D_OV(m) = (1+m)/2 + (1-m)/2 g5 eps_L(H), H = g5 (b+c) D_W / (2 + (b-c) D_W)."""
    b, c, Ls = bcL
    dims, m = (2, 2, 2, 2), 0.1
    U = I.gauge_field(21, dims, 0.6)
    shape = (Ls, 2, 2, 2, 2, 4, 3)
    D = O.dense_matrix(lambda v: O.dwf_op(U, v, m, M5, b, c, bc_t), shape)
    D1 = O.dense_matrix(lambda v: O.dwf_op(U, v, 1.0, M5, b, c, bc_t), shape)
    P = O.dense_matrix(O.P_op, shape)
    Pi = O.dense_matrix(O.Pinv_op, shape)
    K = Pi @ np.linalg.solve(D1, D @ P)
    n4 = 16 * 12
    rest = K[:, n4:]
    want = np.eye(K.shape[0])[:, n4:]
    assert np.abs(rest - want).max() < 1e-13
    DW = O.dense_matrix(lambda v: O.wilson_op(U, v[None], M5, bc_t)[0], (2, 2, 2, 2, 4, 3))
    g5 = np.kron(np.eye(16), np.kron(O.GAMMA5, np.eye(3)))
    Dov = O.d_ov_closed_form(DW, g5, m, Ls, b, c)
    assert np.abs(K[:n4, :n4] - Dov).max() < 1e-12
    assert np.abs(g5 @ Dov @ g5 - Dov.conj().T).max() < 1e-12
    # D_OV(1) = 1
    K1 = Pi @ np.linalg.solve(D1, D1 @ P)
    assert np.abs(K1[:n4, :n4] - np.eye(n4)).max() < 1e-13
