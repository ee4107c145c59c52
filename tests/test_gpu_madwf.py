"""GPU MADWF (Sec. 4 four-step algorithm, Sec. 5 defect correction) through the
C ABI against the FP64 oracle.

  * With tight inner tolerances the defect-correction residual after every
    pass is fixed by the Moebius approximation alone, so the GPU's per-pass
    residuals must equal the oracle MADWF's (same passes, same operators).
  * Inner operator equal to the outer one (b=1, c=0, Ls'=Ls): one pass solves
    the system (Eq. recon is exact when y'_1 = y_1).
  * The final warm-started solve reaches |b - D x| / |b| <= 1e-10 measured by
    the oracle's operator, with two Pauli-Villars and one Moebius solve per pass.
"""
import numpy as np
import pytest
import torch

from oracle import dwf_oracle as O
from paper_1111_5059_gb300 import inputs as I

pytestmark = pytest.mark.gpu

M5 = 1.8


def _to(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _pair(dwf, dims, Ls, Lp, b, c, U):
    outer = dwf.Lattice(dims, Ls, M5)
    inner = dwf.Lattice(dims, Lp, M5, b, c)
    Ut = _to(U)
    outer.set_gauge(Ut)
    inner.set_gauge(Ut)
    return outer, inner


def test_madwf_pass_residuals_match_oracle(dwf):
    dims, Ls, Lp, m = (4, 4, 2, 2), 8, 4, 0.02
    U = I.gauge_field(8, dims, 0.5)
    src = I.gaussian_spinor(8, dims, Ls)
    outer, inner = _pair(dwf, dims, Ls, Lp, 1.5, 0.5, U)
    r = dwf.madwf_solve(outer, inner, m, _to(src), n_dc=3, tol_pv=1e-12, tol_mob=1e-12, tol_final=1e-12,
                        inner_prec="f64")
    xo, info = O.madwf(U, src, m, M5, Lp, 1.5, 0.5, n_dc=3, tol_pv=1e-12, tol_mob=1e-12, tol_final=1e-12)
    st = r.stats
    assert st["passes"] == 3
    assert st["pv"]["iters"] > 0 and st["mobius"]["iters"] > 0
    got, want = np.array(st["pass_resid"]), np.array(info["passes"])
    assert np.all(np.abs(got - want) <= 1e-6 * want + 1e-11), (got, want)
    x = r.x.cpu().numpy()
    res = np.sqrt(O.norm2(src - O.dwf_op(U, x, m, M5)) / O.norm2(src))
    assert res <= 1e-12
    assert np.sqrt(O.norm2(x - xo) / O.norm2(xo)) < 1e-9
    outer.close()
    inner.close()


def test_madwf_one_pass_exact_when_inner_equals_outer(dwf):
    dims, Ls, m = (4, 2, 2, 4), 6, 0.05
    U = I.gauge_field(4, dims, 0.5)
    src = I.gaussian_spinor(4, dims, Ls)
    outer, inner = _pair(dwf, dims, Ls, Ls, 1.0, 0.0, U)
    r = dwf.madwf_solve(outer, inner, m, _to(src), n_dc=1, tol_pv=1e-13, tol_mob=1e-13, tol_final=1e-10,
                        inner_prec="f64")
    assert r.stats["pass_resid"][0] < 1e-10
    assert r.stats["final_cg"]["iters"] == 0
    outer.close()
    inner.close()


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_madwf_mixed_reaches_1e10(dwf, prec):
    """8^4 x Ls=16 Shamir through Moebius Ls'=6 (b - c = 1, b + c = 16/6)."""
    dims, Ls, Lp, m = (8, 8, 8, 8), 16, 6, 0.01
    al = Ls / Lp
    b5, c5 = (al + 1) / 2, (al - 1) / 2
    U = I.gauge_field(3, dims, 0.5)
    src = I.gaussian_spinor(3, dims, Ls)
    outer, inner = _pair(dwf, dims, Ls, Lp, b5, c5, U)
    r = dwf.madwf_solve(outer, inner, m, _to(src), n_dc=3, tol_pv=1e-8, tol_mob=1e-5, tol_final=1e-10,
                        inner_prec=prec)
    st = r.stats
    assert st["passes"] == 3
    assert all(a > b for a, b in zip(st["pass_resid"], st["pass_resid"][1:]))
    x = r.x.cpu().numpy()
    res = np.sqrt(O.norm2(src - O.dwf_op(U, x, m, M5)) / O.norm2(src))
    assert res <= 1e-10
    # fewer final-solve iterations than a cold-start solve
    cold = outer.cg(m, _to(src), tol=1e-10, inner=prec)
    assert st["final_cg"]["iters"] < cold.stats["iters"]
    outer.close()
    inner.close()


@pytest.mark.parametrize("n_dc,tol_pv,tol_mob", [(1, 1e-3, 1e-2), (2, 1e-4, 1e-3)])
def test_madwf_fp32_passes(dwf, n_dc, tol_pv, tol_mob):
    """Loose intermediate tolerances (the benchmark's settings, and two
    passes): the passes' FP64-field hops compute in FP32.  Pass residuals as
    the oracle's MADWF with the same tolerances (its solves in FP64), and the
    final solve reaches 1e-10 by the oracle's operator."""
    dims, Ls, Lp, m = (4, 4, 4, 8), 16, 6, 0.01
    al = Ls / Lp
    b5, c5 = (al + 1) / 2, (al - 1) / 2
    U = I.gauge_field(3, dims, 0.5)
    src = I.gaussian_spinor(3, dims, Ls)
    outer, inner = _pair(dwf, dims, Ls, Lp, b5, c5, U)
    r = dwf.madwf_solve(outer, inner, m, _to(src), n_dc=n_dc, tol_pv=tol_pv, tol_mob=tol_mob, tol_final=1e-10,
                        inner_prec="f32", delta=1e-3, check_every=1)
    st = r.stats
    _, info = O.madwf(U, src, m, M5, Lp, b5, c5, n_dc=n_dc, tol_pv=tol_pv, tol_mob=tol_mob, tol_final=1e-10)
    assert st["passes"] == n_dc
    for got, want in zip(st["pass_resid"][:n_dc], info["passes"]):
        # both are |b - D x| / |b| after inexact inner solves: equal up to
        # those solves' tolerances, not to rounding
        assert 0.5 * want < got < 2.0 * want, (got, want)
    x = r.x.cpu().numpy()
    res = np.sqrt(O.norm2(src - O.dwf_op(U, x, m, M5)) / O.norm2(src))
    assert res <= 1e-10
    outer.close()
    inner.close()


def test_madwf_rejects_mismatched_lattices(dwf):
    U = I.gauge_field(1, (4, 4, 4, 4), 0.3)
    outer = dwf.Lattice((4, 4, 4, 4), 8, M5)
    inner = dwf.Lattice((4, 4, 4, 2), 4, M5, 1.5, 0.5)
    outer.set_gauge(_to(U))
    src = torch.zeros(outer.spinor_shape, dtype=torch.complex128, device="cuda")
    with pytest.raises(dwf.DWFError, match="4D extents"):
        dwf.madwf_solve(outer, inner, 0.04, src)
    mob_outer = dwf.Lattice((4, 4, 4, 4), 8, M5, 1.5, 0.5)
    mob_outer.set_gauge(_to(U))
    inner2 = dwf.Lattice((4, 4, 4, 4), 4, M5, 1.5, 0.5)
    inner2.set_gauge(_to(U))
    with pytest.raises(dwf.DWFError, match="Shamir"):
        dwf.madwf_solve(mob_outer, inner2, 0.04, src)
    for lat in (outer, inner, mob_outer, inner2):
        lat.close()
