"""Solves at the benchmark sizes, checked on sampled sites by the oracle.

The oracle evaluates (D(m) x)(s, n) one 5D site at a time from its
definition; at every sampled site the residual b - D x must not exceed the
global bound tol * |b| that the solve claims (a single entry is bounded by
the norm).  Sizes and parameters are those bench.py times:

  * Shamir 16^3 x 32 x Ls=16, m_f = 0.01, eps = 0.5, seed 2: FP64 CG to
    1e-12 and mixed FP32 / FP16-storage CG to 1e-10;
  * MADWF: Shamir 24^3 x 64 x Ls=32, m_f = 0.002, eps = 0.6, seed 3, through
    Moebius Ls'=12 (b = 11/6, c = 5/6), three defect-correction passes,
    Pauli-Villars tolerance 1e-6, Moebius 1e-5, final 1e-10.
"""
import numpy as np
import pytest
import torch

from oracle import dwf_oracle as O
from paper_1111_5059_gb300 import inputs as I

pytestmark = pytest.mark.gpu

M5 = 1.8


def _sites(dims, Ls, n, seed):
    rng = np.random.default_rng(seed)
    X, Y, Z, T = dims
    pick = [(0, 0, 0, 0, 0), (Ls - 1, T - 1, Z - 1, Y - 1, X - 1)]  # both walls, both corners
    pick += [tuple(int(v) for v in (rng.integers(Ls), rng.integers(T), rng.integers(Z), rng.integers(Y),
                                    rng.integers(X))) for _ in range(n)]
    return pick


def _check_sampled(U, x, b, m, tol, sites, b5=1.0, c5=0.0):
    got = O.dwf_op_at(U, x, m, M5, b5, c5, 1, sites)
    want = np.array([b[s] for s in sites])
    bound = tol * np.sqrt(O.norm2(b))
    worst = float(np.abs(got - want).max())
    assert worst <= bound, (worst, bound)


@pytest.fixture(scope="module")
def mixed_case(dwf):
    dims, Ls = (16, 16, 16, 32), 16
    U = I.gauge_field(2, dims, 0.5)
    b = I.gaussian_spinor(2, dims, Ls)
    lat = dwf.Lattice(dims, Ls, M5)
    lat.set_gauge(torch.from_numpy(U).cuda())
    yield lat, U, b, _sites(dims, Ls, 30, 11)
    lat.close()


@pytest.mark.parametrize("inner,tol", [("f64", 1e-12), ("f32", 1e-10), ("f16", 1e-10)])
def test_cg_16x32_Ls16_sampled(mixed_case, inner, tol):
    lat, U, b, sites = mixed_case
    r = lat.cg(0.01, torch.from_numpy(b).cuda(), tol=tol, inner=inner, delta=0.01)
    assert r.stats["true_resid"] <= tol
    _check_sampled(U, r.x.cpu().numpy(), b, 0.01, tol, sites)


def test_madwf_24x64_Ls32_sampled(dwf):
    dims, Ls, Lp = (24, 24, 24, 64), 32, 12
    U = I.gauge_field(3, dims, 0.6)
    b = I.gaussian_spinor(3, dims, Ls)
    Ut = torch.from_numpy(U).cuda()
    outer = dwf.Lattice(dims, Ls, M5)
    inner = dwf.Lattice(dims, Lp, M5, 11 / 6, 5 / 6)
    outer.set_gauge(Ut)
    inner.set_gauge(Ut)
    r = dwf.madwf_solve(outer, inner, 0.002, torch.from_numpy(b).cuda(), n_dc=3, tol_pv=1e-6, tol_mob=1e-5,
                        tol_final=1e-10, inner_prec="f32", delta=0.01)
    st = r.stats
    assert st["passes"] == 3 and st["total"]["true_resid"] <= 1e-10
    # the defect correction reduces the residual pass by pass (Sec. 5)
    pr = st["pass_resid"]
    assert all(pr[k + 1] < pr[k] for k in range(len(pr) - 1))
    _check_sampled(U, r.x.cpu().numpy(), b, 0.002, 1e-10, _sites(dims, Ls, 30, 12))
    outer.close()
    inner.close()
