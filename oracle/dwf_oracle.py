"""Plain FP64 CPU oracle for the domain-wall hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and its ``--impl reference`` arm) may
import this module.  The CUDA library never calls it and shares no code with
it; both sides only consume the seeded fields of
``paper_1111_5059_gb300/inputs.py``.

Everything is complex128 / float64 numpy, written for a reader to check against
the paper by eye: whole-lattice ``np.roll`` shifts, ``matmul`` colour and spin
products, dense Ls x Ls fifth-dimension matrices, library LU / eigh where a
step is a plain linear-algebra definition.

Paper: Yin & Mawhinney, "Improving DWF Simulations: the Force Gradient
Integrator and the Moebius Accelerated DWF Solver" (Lattice 2011).
  Sec. 2 (Eqs. 1-6)   force-gradient PQPQP integrator, U' = exp(-tau^2/24 F^j T_j) U;
                      the Omelyan 2MN integrator it is compared with, whole
                      trajectories and the Metropolis test
  Sec. 3 (Eqs. 7-8)   Hasenbusch quotient actions
  Sec. 4 (Eqs. 9-16)  D_DW(m) x = b, the domain-wall -> overlap transformation,
                      Eq. (ov_eq), (trans_5d_4d_source), (dwf_eq_4d), (mob_eq_4d),
                      (recon), (mob_eq_5d) and the four-step MADWF algorithm
  Sec. 5              defect correction, Table 1

Readings (the paper defines none of these; each is pinned by a test that a
plausible mistake fails):
  * Euclidean chiral basis, hermitian gamma_mu, gamma5 = g1 g2 g3 g4 =
    diag(1,1,-1,-1), P+- = (1 +- gamma5)/2.
  * Wilson: D_W = (4 - M5) - 1/2 D_hop,
      D_hop psi(n) = sum_mu (1-g_mu) U_mu(n) psi(n+mu) + (1+g_mu) U_mu(n-mu)^+ psi(n-mu),
    periodic in x,y,z; t periodic (bc_t=+1) or antiperiodic (bc_t=-1).
  * Moebius / Shamir: D(m) = D_W (b + c Q(m)) + 1 - Q(m),
      Q(m) psi_s = P- psi_{s+1} + P+ psi_{s-1},  psi_{Ls} := -m psi_0,
      psi_{-1} := -m psi_{Ls-1};  Shamir is b=1, c=0.
  * Even-odd: A = (4-M5)(b+cQ) + 1 - Q on each parity, M_eo = -1/2 D_hop^{eo} B,
    M_pc = A - M_eo A^-1 M_oe on even sites.
  * P (the paper defers it to its ref. MD_trans):
      (P^-1 x)_s = P- x_s + P+ x_{s-1 mod Ls},  (P y)_s = P- y_s + P+ y_{s+1 mod Ls};
    the paper's first slice "s = 1" is index 0 here.
  * Generators T_j = i lambda_j / 2, tr(T_i T_j) = -delta_ij / 2; p = p^j T_j;
    H = 1/2 sum (p^j)^2 + S_f;  dU/dt = p U, dp^j/dt = -F^j, F^j = e_j(S).
  * Quotient action S = |M1^-dag M2^dag phi|^2 with M = M_pc (Sec. 3).
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------
# Dirac algebra
# ---------------------------------------------------------------------------


def gamma_matrices():
    """Hermitian Euclidean gamma matrices in the chiral basis, and gamma5."""
    s1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    s2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    s3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    Z = np.zeros((2, 2), dtype=np.complex128)
    I = np.eye(2, dtype=np.complex128)
    g = [np.block([[Z, -1j * s], [1j * s, Z]]) for s in (s1, s2, s3)]
    g.append(np.block([[Z, I], [I, Z]]))
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return np.array(g), g5


GAMMA, GAMMA5 = gamma_matrices()
ID4 = np.eye(4, dtype=np.complex128)
P_PLUS = (ID4 + GAMMA5) / 2
P_MINUS = (ID4 - GAMMA5) / 2


def generators():
    """su(3) generators T_j = i lambda_j / 2 (Gell-Mann lambda_j), shape (8,3,3)."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1], l[1][1, 0] = -1j, 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2], l[4][2, 0] = -1j, 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2], l[6][2, 1] = -1j, 1j
    l[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return 0.5j * l


T_GEN = generators()

# ---------------------------------------------------------------------------
# Lattice geometry.  4D fields: axes (t, z, y, x, ...); 5D spinors: axes
# (s, t, z, y, x, spin, colour).  Direction mu = 0,1,2,3 is x, y, z, t.
# ---------------------------------------------------------------------------


def _axis(mu: int, lead: int) -> int:
    return lead + 3 - mu


def shift(f: np.ndarray, mu: int, sign: int, lead: int, bc_t: int = 1) -> np.ndarray:
    """g(n) = f(n + sign*mu_hat) with periodic wrap; -1 across the t boundary if bc_t = -1."""
    ax = _axis(mu, lead)
    g = np.roll(f, -sign, axis=ax)
    if mu == 3 and bc_t == -1:
        idx = [slice(None)] * g.ndim
        idx[ax] = -1 if sign > 0 else 0
        g[tuple(idx)] *= -1
    return g


def colour_mul(U: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(U psi)(s,n,spin,a) = sum_b U(n)_{ab} psi(s,n,spin,b)."""
    return np.matmul(psi, np.swapaxes(U, -1, -2)[None])


def spin_mul(G: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(G psi)(...,i,a) = sum_j G_{ij} psi(...,j,a)."""
    return np.matmul(G, psi)


def dagger(M: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(M, -1, -2))


def coords(dims):
    """Arrays t, z, y, x of shape (T,Z,Y,X)."""
    X, Y, Z, T = dims
    return np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")


def parity(dims) -> np.ndarray:
    """(x+y+z+t) mod 2 on the (T,Z,Y,X) grid."""
    t, z, y, x = coords(dims)
    return (x + y + z + t) % 2


# ---------------------------------------------------------------------------
# 4D Wilson operator (the D_W inside D_DW, Eq. dirac_eq)
# ---------------------------------------------------------------------------


def wilson_hop(U: np.ndarray, psi: np.ndarray, bc_t: int = 1, dag: bool = False) -> np.ndarray:
    """D_hop psi at every s; with dag=True its adjoint (projectors 1 -+ g_mu swapped)."""
    sg = -1.0 if dag else 1.0
    out = np.zeros_like(psi)
    for mu in range(4):
        fwd = colour_mul(U[mu], shift(psi, mu, +1, 1, bc_t))
        out += spin_mul(ID4 - sg * GAMMA[mu], fwd)
        Ub = dagger(shift(U[mu], mu, -1, 0))
        bwd = colour_mul(Ub, shift(psi, mu, -1, 1, bc_t))
        out += spin_mul(ID4 + sg * GAMMA[mu], bwd)
    return out


def wilson_op(U, psi, M5, bc_t=1, dag=False):
    """D_W = (4 - M5) - 1/2 D_hop (and its adjoint)."""
    return (4.0 - M5) * psi - 0.5 * wilson_hop(U, psi, bc_t, dag)


# ---------------------------------------------------------------------------
# Fifth dimension (the P+- hop with the m wall)
# ---------------------------------------------------------------------------


def s_hops(Ls: int, m: float):
    """Real Ls x Ls matrices S_up: psi_s <- psi_{s+1} (psi_Ls := -m psi_0) and
    S_dn: psi_s <- psi_{s-1} (psi_{-1} := -m psi_{Ls-1})."""
    S_up = np.zeros((Ls, Ls))
    S_dn = np.zeros((Ls, Ls))
    for s in range(Ls):
        if s + 1 < Ls:
            S_up[s, s + 1] += 1.0
        else:
            S_up[s, 0] += -m
        if s - 1 >= 0:
            S_dn[s, s - 1] += 1.0
        else:
            S_dn[s, Ls - 1] += -m
    return S_up, S_dn


def fifth(Mp: np.ndarray, Mm: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Apply the real matrix Mp over s to the P+ part and Mm to the P- part."""
    return (np.tensordot(Mp, spin_mul(P_PLUS, psi), axes=(1, 0))
            + np.tensordot(Mm, spin_mul(P_MINUS, psi), axes=(1, 0)))


def q_mats(Ls: int, m: float):
    """Q(m) per chirality: on P+ it is S_dn, on P- it is S_up."""
    S_up, S_dn = s_hops(Ls, m)
    return S_dn, S_up


def q_op(psi: np.ndarray, m: float, dag: bool = False) -> np.ndarray:
    Qp, Qm = q_mats(psi.shape[0], m)
    if dag:
        return fifth(Qp.T, Qm.T, psi)
    return fifth(Qp, Qm, psi)


# ---------------------------------------------------------------------------
# 5D domain-wall operator D_DW(m) (Shamir) and its Moebius generalisation
# ---------------------------------------------------------------------------


def dwf_op(U, psi, m, M5, b=1.0, c=0.0, bc_t=1, dag=False):
    """D(m) psi = D_W (b + c Q(m)) psi + psi - Q(m) psi, or its adjoint."""
    if not dag:
        Bpsi = b * psi + c * q_op(psi, m)
        return wilson_op(U, Bpsi, M5, bc_t) + psi - q_op(psi, m)
    W = wilson_op(U, psi, M5, bc_t, dag=True)
    return b * W + c * q_op(W, m, dag=True) + psi - q_op(psi, m, dag=True)


def dwf_op_at(U, psi, m, M5, b, c, bc_t, sites):
    """(D(m) psi) at the 5D sites (s,t,z,y,x), evaluated one by one from the
    definition (for checks at sizes where a whole-lattice pass is too slow)."""
    Ls, T, Z, Y, X = psi.shape[:5]
    ext = (X, Y, Z, T)

    def q_at(s, n):
        t, z, y, x = n
        up = psi[s + 1, t, z, y, x] if s + 1 < Ls else -m * psi[0, t, z, y, x]
        dn = psi[s - 1, t, z, y, x] if s >= 1 else -m * psi[Ls - 1, t, z, y, x]
        return P_MINUS @ up + P_PLUS @ dn

    def b_at(s, n):
        t, z, y, x = n
        return b * psi[s, t, z, y, x] + c * q_at(s, n)

    out = []
    for (s, t, z, y, x) in sites:
        n = (t, z, y, x)
        acc = (4.0 - M5) * b_at(s, n) + psi[s, t, z, y, x] - q_at(s, n)
        xyzt = [x, y, z, t]
        for mu in range(4):
            fw = list(xyzt)
            bw = list(xyzt)
            fw[mu] += 1
            bw[mu] -= 1
            phase_f = phase_b = 1.0
            if mu == 3 and bc_t == -1:
                if fw[3] == T:
                    phase_f = -1.0
                if bw[3] == -1:
                    phase_b = -1.0
            fw = [fw[i] % ext[i] for i in range(4)]
            bw = [bw[i] % ext[i] for i in range(4)]
            nf = (fw[3], fw[2], fw[1], fw[0])
            nb = (bw[3], bw[2], bw[1], bw[0])
            Uf = U[mu][n]
            Ub = dagger(U[mu][nb])
            acc = acc - 0.5 * (ID4 - GAMMA[mu]) @ (phase_f * b_at(s, nf) @ Uf.T)
            acc = acc - 0.5 * (ID4 + GAMMA[mu]) @ (phase_b * b_at(s, nb) @ Ub.T)
        out.append(acc)
    return np.array(out)


# ---------------------------------------------------------------------------
# Even-odd preconditioning.  One-parity fields are whole-lattice arrays that
# vanish on the other parity.
# ---------------------------------------------------------------------------


class EO:
    """Even-odd blocks of D(m) for fixed (U, m, M5, b, c, Ls, bc_t)."""

    def __init__(self, U, m, M5, Ls, b=1.0, c=0.0, bc_t=1):
        self.U, self.m, self.M5, self.Ls, self.b, self.c, self.bc_t = U, m, M5, Ls, b, c, bc_t
        dims = (U.shape[4], U.shape[3], U.shape[2], U.shape[1])
        par = parity(dims)
        self.even = (par == 0)[None, :, :, :, :, None, None]
        self.odd = (par == 1)[None, :, :, :, :, None, None]
        Qp, Qm = q_mats(Ls, m)
        I = np.eye(Ls)
        self.Bp, self.Bm = b * I + c * Qp, b * I + c * Qm
        self.Ap = (4.0 - M5) * self.Bp + I - Qp
        self.Am = (4.0 - M5) * self.Bm + I - Qm
        self.Aip, self.Aim = np.linalg.inv(self.Ap), np.linalg.inv(self.Am)

    # s-local blocks (no links)
    def A(self, x, dag=False):
        return fifth(self.Ap.T, self.Am.T, x) if dag else fifth(self.Ap, self.Am, x)

    def Ainv(self, x, dag=False):
        return fifth(self.Aip.T, self.Aim.T, x) if dag else fifth(self.Aip, self.Aim, x)

    def B(self, x, dag=False):
        return fifth(self.Bp.T, self.Bm.T, x) if dag else fifth(self.Bp, self.Bm, x)

    # off-diagonal blocks: M_eo (odd -> even) and M_oe (even -> odd)
    def Moff(self, x, dag=False):
        """-1/2 D_hop B x (or its adjoint -1/2 B^+ D_hop^+ x); parity flips."""
        if not dag:
            return -0.5 * wilson_hop(self.U, self.B(x), self.bc_t)
        return -0.5 * self.B(wilson_hop(self.U, x, self.bc_t, dag=True), dag=True)

    def Mpc(self, x, dag=False):
        """M_pc = A - M_eo A^-1 M_oe on even sites (or its adjoint)."""
        if not dag:
            return self.A(x) - self.Moff(self.Ainv(self.Moff(x)))
        return self.A(x, True) - self.Moff(self.Ainv(self.Moff(x, True), True), True)

    def prepare(self, b):
        """b'_e = b_e - M_eo A^-1 b_o."""
        be, bo = b * self.even, b * self.odd
        return be - self.Moff(self.Ainv(bo)) * self.even

    def reconstruct(self, xe, b):
        """x_o = A^-1 (b_o - M_oe x_e); returns x_e + x_o."""
        bo = b * self.odd
        xo = self.Ainv(bo - self.Moff(xe) * self.odd)
        return xe * self.even + xo * self.odd


# ---------------------------------------------------------------------------
# Solvers: CG on the normal equations (CGLS form) and the full solve
# ---------------------------------------------------------------------------


def vdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def norm2(a) -> float:
    return float(np.vdot(a.ravel(), a.ravel()).real)


def cgls(apply_M, apply_Mdag, rhs, x0, tol, maxiter, ref_norm=None):
    """CG on M^+ M x = M^+ rhs, monitoring the residual rhs - M x.

    Stops when |rhs - M x| <= tol * ref_norm (recomputed at exit).
    Returns (x, iterations, final relative residual)."""
    ref = np.sqrt(norm2(rhs)) if ref_norm is None else ref_norm
    x = x0.copy()
    r = rhs - apply_M(x)
    s = apply_Mdag(r)
    p = s.copy()
    gam = norm2(s)
    it = 0
    while it < maxiter:
        if np.sqrt(norm2(r)) <= tol * ref:
            r = rhs - apply_M(x)
            if np.sqrt(norm2(r)) <= tol * ref:
                break
            s = apply_Mdag(r)
            p = s.copy()
            gam = norm2(s)
        q = apply_M(p)
        alpha = gam / norm2(q)
        x = x + alpha * p
        r = r - alpha * q
        s = apply_Mdag(r)
        gnew = norm2(s)
        p = s + (gnew / gam) * p
        gam = gnew
        it += 1
    res = np.sqrt(norm2(rhs - apply_M(x))) / ref
    return x, it, res


def solve(U, b, m, M5, b5=1.0, c5=0.0, bc_t=1, tol=1e-12, maxiter=100000, x0=None):
    """x = D(m)^-1 b by even-odd CG on M_pc^+ M_pc, then odd reconstruction.

    The residual target is the full unpreconditioned |b - D x| / |b|.
    Returns (x, iterations, true relative residual)."""
    Ls = b.shape[0]
    eo = EO(U, m, M5, Ls, b5, c5, bc_t)
    bp = eo.prepare(b)
    xe0 = np.zeros_like(b) if x0 is None else x0 * eo.even
    bn = np.sqrt(norm2(b))
    xe, it, _ = cgls(eo.Mpc, lambda v: eo.Mpc(v, True), bp, xe0, tol, maxiter, ref_norm=bn)
    x = eo.reconstruct(xe, b)
    res = np.sqrt(norm2(b - dwf_op(U, x, m, M5, b5, c5, bc_t))) / bn
    return x, it, res


def dense_matrix(apply, shape) -> np.ndarray:
    """The matrix of a linear map on arrays of ``shape``, column by column."""
    N = int(np.prod(shape))
    Mat = np.empty((N, N), dtype=np.complex128)
    e = np.zeros(N, dtype=np.complex128)
    for j in range(N):
        e[j] = 1.0
        Mat[:, j] = apply(e.reshape(shape)).ravel()
        e[j] = 0.0
    return Mat


# ---------------------------------------------------------------------------
# Domain wall -> overlap transformation (Sec. 4, Eqs. ov_eq, trans_5d_4d_source)
# ---------------------------------------------------------------------------


def P_op(y: np.ndarray) -> np.ndarray:
    """(P y)_s = P- y_s + P+ y_{s+1 mod Ls}."""
    return spin_mul(P_MINUS, y) + spin_mul(P_PLUS, np.roll(y, -1, axis=0))


def Pinv_op(x: np.ndarray) -> np.ndarray:
    """(P^-1 x)_s = P- x_s + P+ x_{s-1 mod Ls}; slice 0 is the 4D quark field."""
    return spin_mul(P_MINUS, x) + spin_mul(P_PLUS, np.roll(x, 1, axis=0))


def eps_L(H: np.ndarray, L: int) -> np.ndarray:
    """[(1+H)^L - (1-H)^L] [(1+H)^L + (1-H)^L]^-1 for hermitian H, by eigh."""
    lam, V = np.linalg.eigh(H)
    a, bb = (1 + lam) ** L, (1 - lam) ** L
    return (V * ((a - bb) / (a + bb))) @ dagger(V)


def d_ov_closed_form(DW: np.ndarray, g5: np.ndarray, m, L, b, c) -> np.ndarray:
    """Effective 4D operator of a Moebius/Shamir 5D operator (dense):
    (1+m)/2 + (1-m)/2 g5 eps_L(H),  H = g5 (b+c) D_W (2 + (b-c) D_W)^-1."""
    N = DW.shape[0]
    I = np.eye(N)
    H = g5 @ ((b + c) * DW) @ np.linalg.inv(2 * I + (b - c) * DW)
    H = 0.5 * (H + dagger(H))
    return 0.5 * (1 + m) * I + 0.5 * (1 - m) * g5 @ eps_L(H, L)


# ---------------------------------------------------------------------------
# MADWF (Sec. 4 four-step algorithm + Sec. 5 defect correction)
# ---------------------------------------------------------------------------


def madwf(U, src, m, M5, Ls_in, b_in, c_in, bc_t=1, n_dc=3, tol_pv=1e-10,
          tol_mob=1e-10, tol_final=1e-10, solve_fn=None, final=True):
    """Moebius-accelerated solve of the Shamir D_DW(m) x = src.

    Each defect-correction pass (Sec. 5) runs the four steps of Sec. 4 on the
    current residual and adds the guess; the final solve (Eq. dirac_eq) starts
    from the accumulated guess.  Returns (x, info)."""
    solve_fn = solve_fn or solve
    Ls = src.shape[0]
    x = np.zeros_like(src)
    info = {"pv_solves": 0, "mob_solves": 0, "passes": [], "pv_iters": 0, "mob_iters": 0}
    bn = np.sqrt(norm2(src))
    for _ in range(n_dc):
        r = src - dwf_op(U, x, m, M5, 1.0, 0.0, bc_t)
        # step 1: c = P^-1 D_DW(1)^-1 r   (Eq. trans_5d_4d_source)
        ct, it, _ = solve_fn(U, r, 1.0, M5, 1.0, 0.0, bc_t, tol=tol_pv)
        info["pv_solves"] += 1
        info["pv_iters"] += it
        cvec = Pinv_op(ct)
        # steps 2-3: D'_DW(m) P y' = D'_DW(1) P c',  c' = (c_1, 0, ..., 0)  (Eq. mob_eq_5d)
        cp = np.zeros((Ls_in,) + src.shape[1:], dtype=src.dtype)
        cp[0] = cvec[0]
        rhs = dwf_op(U, P_op(cp), 1.0, M5, b_in, c_in, bc_t)
        z, it, _ = solve_fn(U, rhs, m, M5, b_in, c_in, bc_t, tol=tol_mob)
        info["mob_solves"] += 1
        info["mob_iters"] += it
        y1 = Pinv_op(z)[0]
        # step 4: (-D_OV y'_1, y'_2, ...) = P^-1 D(1)^-1 D(m) P (-y'_1, c_2, ...)  (Eq. recon)
        w = cvec.copy()
        w[0] = -y1
        u_t, it, _ = solve_fn(U, dwf_op(U, P_op(w), m, M5, 1.0, 0.0, bc_t), 1.0, M5,
                              1.0, 0.0, bc_t, tol=tol_pv)
        info["pv_solves"] += 1
        info["pv_iters"] += it
        y = Pinv_op(u_t)
        y[0] = y1
        x = x + P_op(y)
        info["passes"].append(np.sqrt(norm2(src - dwf_op(U, x, m, M5, 1.0, 0.0, bc_t))) / bn)
    if final:
        x, it, res = solve_fn(U, src, m, M5, 1.0, 0.0, bc_t, tol=tol_final, x0=x)
        info["final_iters"] = it
        info["final_res"] = res
    return x, info


# ---------------------------------------------------------------------------
# SU(3) algebra, pseudofermion action and fermion force (Sec. 2-3)
# ---------------------------------------------------------------------------


def algebra_matrix(comp: np.ndarray) -> np.ndarray:
    """X = sum_j X^j T_j from components (..., 8)."""
    return np.einsum("...j,jab->...ab", comp, T_GEN)


def algebra_components(Xm: np.ndarray) -> np.ndarray:
    """X^j = -2 tr(T_j X) for X in su(3) (tr(T_i T_j) = -delta_ij/2)."""
    return (-2.0 * np.einsum("jab,...ba->...j", T_GEN, Xm)).real


def su3_exp(Xm: np.ndarray) -> np.ndarray:
    """exp(X) for anti-hermitian X: X = iH, exp(X) = V e^{i lambda} V^+ (eigh of H)."""
    H = -1j * Xm
    H = 0.5 * (H + dagger(H))
    lam, V = np.linalg.eigh(H)
    return np.einsum("...ab,...b,...cb->...ac", V, np.exp(1j * lam), np.conj(V))


def heatbath_phi(U, eta, m1, m2, M5, b=1.0, c=0.0, bc_t=1, tol=1e-13):
    """phi = M2^-dag M1^dag eta on even sites (so that S(phi) = |eta|^2)."""
    Ls = eta.shape[0]
    eo1 = EO(U, m1, M5, Ls, b, c, bc_t)
    eo2 = EO(U, m2, M5, Ls, b, c, bc_t)
    v = eo1.Mpc(eta * eo1.even, True)
    # M2^+ phi = v  <=>  phi = M2 (M2^+ M2)^-1 ... solve with CGLS on M2^+.
    phi, _, _ = cgls(lambda x: eo2.Mpc(x, True), eo2.Mpc, v, np.zeros_like(v), tol, 100000)
    return phi


def quotient_solution(U, phi, m1, m2, M5, b=1.0, c=0.0, bc_t=1, tol=1e-13, x0=None, dense=None):
    """X = (M1^+ M1)^-1 M2^+ phi and Y = M1 X; returns (X, Y, S, iters)."""
    Ls = phi.shape[0]
    eo1 = EO(U, m1, M5, Ls, b, c, bc_t)
    eo2 = EO(U, m2, M5, Ls, b, c, bc_t)
    v = eo2.Mpc(phi, True)
    if dense is not None:
        X = dense(eo1, v)
        it = 0
    else:
        # M1^+ M1 X = v: CGLS on the system M1^+ Y = v, i.e. M1^+ (M1 X) = v.
        X0 = np.zeros_like(v) if x0 is None else x0
        X, it = _cg_normal(eo1, v, X0, tol)
    Y = eo1.Mpc(X)
    S = norm2(Y)
    return X, Y, S, it


def _cg_normal(eo, v, x0, tol, maxiter=100000):
    """Plain CG on (M^+ M) X = v."""
    x = x0.copy()
    r = v - eo.Mpc(eo.Mpc(x), True)
    p = r.copy()
    rr = norm2(r)
    vn = norm2(v)
    it = 0
    while rr > tol * tol * vn and it < maxiter:
        Ap = eo.Mpc(eo.Mpc(p), True)
        alpha = rr / vdot(p, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        rn = norm2(r)
        p = r + (rn / rr) * p
        rr = rn
        it += 1
    return x, it


def _link_outer(U, Lf, Rf, bc_t):
    """G_mu(n) = sum_s [ (1-g_mu) (U_mu(n) R(n+mu)) (x) L(n)^+
                         - (1+g_mu) R(n) (x) (U_mu(n) L(n+mu))^+ ]  (colour 3x3),
    the link derivative  d/dh Re[L^+ D_hop(e^{hT}U) R] = Re tr(T G)."""
    G = np.zeros(U.shape, dtype=np.complex128)
    for mu in range(4):
        V = colour_mul(U[mu], shift(Rf, mu, +1, 1, bc_t))
        W = colour_mul(U[mu], shift(Lf, mu, +1, 1, bc_t))
        PV = spin_mul(ID4 - GAMMA[mu], V)
        PR = spin_mul(ID4 + GAMMA[mu], Rf)
        G[mu] = (np.einsum("s...ib,s...ia->...ba", PV, np.conj(Lf))
                 - np.einsum("s...ib,s...ia->...ba", PR, np.conj(W)))
    return G


def quotient_force(U, X, Y, phi, m1, m2, M5, b=1.0, c=0.0, bc_t=1):
    """F^j(n,mu) = e_j S for S = phi^+ M2 X, X = (M1^+M1)^-1 M2^+ phi, Y = M1 X.

    dS = 2 Re[phi^+ dM2 X] - 2 Re[Y^+ dM1 X] with
    Re[L^+ dM R] = 1/2 Re[L_e^+ dD_hop (B A^-1 M_oe R)] + 1/2 Re[(A^-+ M_eo^+ L)^+ dD_hop (B R)].
    Returns components float64 [4][T][Z][Y][X][8]."""
    Ls = X.shape[0]
    G = np.zeros(U.shape, dtype=np.complex128)
    for (Lv, mass, sgn) in ((phi, m2, +1.0), (Y, m1, -1.0)):
        eo = EO(U, mass, M5, Ls, b, c, bc_t)
        R_o = eo.B(eo.Ainv(eo.Moff(X))) * eo.odd
        R_e = eo.B(X) * eo.even
        L_o = eo.Ainv(eo.Moff(Lv * eo.even, True), True) * eo.odd
        L_e = Lv * eo.even
        # 2 * 1/2 * Re[...]: one outer product over both parities
        G += sgn * _link_outer(U, L_e + L_o, R_o + R_e, bc_t)
    # F^j = Re tr(T_j G)
    return np.einsum("jab,...ba->...j", T_GEN, G).real


def action_and_force(U, phis, terms, M5, b=1.0, c=0.0, bc_t=1, tol=1e-13, guesses=None):
    """Sum over quotient terms (m1, m2) of S and F. Returns (S, F, solutions)."""
    S = 0.0
    F = np.zeros(U.shape[:5] + (8,))
    sols = []
    for k, ((m1, m2), phi) in enumerate(zip(terms, phis)):
        x0 = None if guesses is None else guesses[k]
        X, Y, Sk, _ = quotient_solution(U, phi, m1, m2, M5, b, c, bc_t, tol, x0=x0)
        S += Sk
        F += quotient_force(U, X, Y, phi, m1, m2, M5, b, c, bc_t)
        sols.append(X)
    return S, F, sols


def link_update(U, comp, coeff):
    """U <- exp(coeff * sum_j comp^j T_j) U."""
    return np.einsum("...ab,...bc->...ac", su3_exp(coeff * algebra_matrix(comp)), U)


def fgi_step(U, p, tau, phis, terms, M5, b=1.0, c=0.0, bc_t=1, tol=1e-13, forecast=True):
    """One force-gradient PQPQP step (Eq. 1) with the two-step FG update (Sec. 2):
    P(tau/6) Q(tau/2) [F(U); U' = exp(-tau^2/24 F^j T_j) U; p -= 2/3 tau F(U')] Q(tau/2) P(tau/6).
    With forecast=True the U' solve starts from the U solution."""
    _, F, _ = action_and_force(U, phis, terms, M5, b, c, bc_t, tol)
    p = p - tau / 6 * F
    U = link_update(U, p, tau / 2)
    _, F, sols = action_and_force(U, phis, terms, M5, b, c, bc_t, tol)
    Up = link_update(U, F, -tau * tau / 24)
    _, Fp, _ = action_and_force(Up, phis, terms, M5, b, c, bc_t, tol,
                                guesses=sols if forecast else None)
    p = p - 2.0 / 3.0 * tau * Fp
    U = link_update(U, p, tau / 2)
    _, F, _ = action_and_force(U, phis, terms, M5, b, c, bc_t, tol)
    p = p - tau / 6 * F
    return U, p


def hamiltonian(U, p, phis, terms, M5, b=1.0, c=0.0, bc_t=1, tol=1e-13):
    S = sum(quotient_solution(U, phi, m1, m2, M5, b, c, bc_t, tol)[2]
            for (m1, m2), phi in zip(terms, phis))
    return 0.5 * float(np.sum(p * p)) + S


# ---------------------------------------------------------------------------
# Trajectories: the force-gradient integrator against Omelyan's (Sec. 2)
# ---------------------------------------------------------------------------

# The second-order minimum-norm ("2MN") parameter of Omelyan, Mryglod and
# Folk, Comput. Phys. Commun. 151 (2003) 272 -- the integrator Sec. 2
# compares the force-gradient integrator with.
OMELYAN_LAMBDA = 0.1931833275037836


def omelyan_step(U, p, tau, phis, terms, M5, b=1.0, c=0.0, bc_t=1, tol=1e-13, lam=OMELYAN_LAMBDA):
    """One Omelyan 2MN step: P(lam tau) Q(tau/2) P((1 - 2 lam) tau) Q(tau/2) P(lam tau)."""
    _, F, _ = action_and_force(U, phis, terms, M5, b, c, bc_t, tol)
    p = p - lam * tau * F
    U = link_update(U, p, tau / 2)
    _, F, _ = action_and_force(U, phis, terms, M5, b, c, bc_t, tol)
    p = p - (1.0 - 2.0 * lam) * tau * F
    U = link_update(U, p, tau / 2)
    _, F, _ = action_and_force(U, phis, terms, M5, b, c, bc_t, tol)
    p = p - lam * tau * F
    return U, p


def md_trajectory(U, p, tau, nsteps, phis, terms, M5, b=1.0, c=0.0, bc_t=1, tol=1e-13, integrator="fgi"):
    """nsteps steps of length tau of the force-gradient integrator (as in
    fgi_step, with forecasting) or of Omelyan's 2MN (omelyan_step).

    The closing momentum update of a step and the opening one of the next use
    the force at the same U, so they are applied as one update of twice the
    weight: a trajectory evaluates the force 3 nsteps + 1 (FGI) or
    2 nsteps + 1 (Omelyan) times instead of 4 nsteps or 3 nsteps.
    Returns (U, p, force evaluations)."""
    if integrator not in ("fgi", "omelyan"):
        raise ValueError(integrator)
    a = 1.0 / 6.0 if integrator == "fgi" else OMELYAN_LAMBDA  # weight of the end momentum updates
    count = 0

    def force(Ux, guesses=None):
        nonlocal count
        count += 1
        return action_and_force(Ux, phis, terms, M5, b, c, bc_t, tol, guesses=guesses)

    _, F, _ = force(U)
    p = p - a * tau * F
    for k in range(nsteps):
        U = link_update(U, p, tau / 2)
        if integrator == "fgi":
            _, F, sols = force(U)
            _, Fp, _ = force(link_update(U, F, -tau * tau / 24), guesses=sols)
            p = p - 2.0 / 3.0 * tau * Fp
        else:
            _, F, _ = force(U)
            p = p - (1.0 - 2.0 * a) * tau * F
        U = link_update(U, p, tau / 2)
        _, F, _ = force(U)
        p = p - (a if k == nsteps - 1 else 2.0 * a) * tau * F
    return U, p, count


def metropolis_accept(dH: float, u: float) -> bool:
    """Accept a trajectory with probability min(1, exp(-dH)); u is a uniform
    number in [0, 1) that the caller draws."""
    return dH <= 0.0 or u < float(np.exp(-dH))
