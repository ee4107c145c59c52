"""GPU solves (through the C ABI) against the FP64 oracle.

Primary criterion: the true residual |b - D(m) x| / |b| of the GPU solution,
computed by the ORACLE's operator: <= 1e-12 for plain FP64 CG, <= 1e-10 for
mixed precision (FP32 / FP16 storage with FP64 reliable updates).
Secondary: |x_gpu - x_oracle| / |x_oracle| against the oracle's own solve,
bounded by the solves' tolerance times a condition-number allowance.
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


def _true_res(U, x, b, m, b5=1.0, c5=0.0, bc_t=1):
    r = b - O.dwf_op(U, x, m, M5, b5, c5, bc_t)
    return np.sqrt(O.norm2(r) / O.norm2(b))


@pytest.fixture(scope="module")
def small(dwf):
    """4^4 x Ls=8, m_f = 0.04, eps = 0.3 (the small plain-Shamir workload)."""
    dims, Ls = (4, 4, 4, 4), 8
    U = I.gauge_field(1, dims, 0.3)
    b = I.gaussian_spinor(1, dims, Ls)
    lat = dwf.Lattice(dims, Ls, M5)
    lat.set_gauge(_to(U))
    xo, it, res = O.solve(U, b, 0.04, M5, tol=1e-13)
    yield lat, U, b, xo
    lat.close()


def test_cg_fp64_small_matches_oracle(small):
    lat, U, b, xo = small
    r = lat.cg(0.04, _to(b), tol=1e-12, inner="f64")
    x = r.x.cpu().numpy()
    assert r.stats["true_resid"] <= 1e-12
    assert _true_res(U, x, b, 0.04) <= 1e-12
    assert np.sqrt(O.norm2(x - xo) / O.norm2(xo)) < 1e-9
    assert r.stats["iters"] > 0 and r.stats["op_count"] == r.stats["iters"] * 8


@pytest.mark.parametrize("inner", ["f32", "f16"])
def test_cg_mixed_small_matches_oracle(small, inner):
    lat, U, b, xo = small
    r = lat.cg(0.04, _to(b), tol=1e-10, inner=inner, delta=0.1)
    x = r.x.cpu().numpy()
    assert _true_res(U, x, b, 0.04) <= 1e-10
    assert r.stats["reliable_updates"] >= 1
    assert np.sqrt(O.norm2(x - xo) / O.norm2(xo)) < 1e-7


def test_cg_warm_start_from_solution_takes_no_iterations(small):
    lat, U, b, xo = small
    r = lat.cg(0.04, _to(b), x0=_to(xo), tol=1e-10)
    assert r.stats["iters"] == 0
    assert _true_res(U, r.x.cpu().numpy(), b, 0.04) <= 1e-10


@pytest.mark.parametrize("bc", [(1.5, 0.5, -1), (11 / 6, 5 / 6, 1)])
def test_cg_mobius_matches_oracle(dwf, bc):
    b5, c5, bc_t = bc
    dims, Ls, m = (4, 4, 2, 6), 6, 0.02
    U = I.gauge_field(7, dims, 0.5)
    src = I.gaussian_spinor(7, dims, Ls)
    lat = dwf.Lattice(dims, Ls, M5, b5, c5, bc_t)
    lat.set_gauge(_to(U))
    for inner, tol in (("f64", 1e-12), ("f32", 1e-10)):
        r = lat.cg(m, _to(src), tol=tol, inner=inner)
        assert _true_res(U, r.x.cpu().numpy(), src, m, b5, c5, bc_t) <= tol
    lat.close()


@pytest.mark.parametrize("Ls", [5, 12])
@pytest.mark.parametrize("inner", ["f32", "f16"])
def test_cg_mixed_ragged_shapes(dwf, Ls, inner):
    """Odd Ls (a padding slot in the slice-pair layout), Ls = 12 (Lh = 6 pairs,
    21 sites per CTA) and a ragged last CTA (Vh = 96)."""
    dims, m = (4, 4, 2, 6), 0.05
    U = I.gauge_field(9, dims, 0.5)
    src = I.gaussian_spinor(9, dims, Ls)
    lat = dwf.Lattice(dims, Ls, M5)
    lat.set_gauge(_to(U))
    r = lat.cg(m, _to(src), tol=1e-10, inner=inner)
    assert _true_res(U, r.x.cpu().numpy(), src, m) <= 1e-10
    lat.close()


def test_zero_source_gives_zero(small, dwf):
    lat, U, b, xo = small
    r = lat.cg(0.04, torch.zeros(lat.spinor_shape, dtype=torch.complex128, device="cuda"))
    assert torch.count_nonzero(r.x) == 0


def test_max_iter_reports_not_converged(small, dwf):
    lat, U, b, xo = small
    r = lat.cg(0.04, _to(b), tol=1e-12, max_iter=3, raise_on_fail=False)
    assert r.status == 4  # DWF_ERR_NOT_CONVERGED
    assert r.stats["iters"] == 3
    assert r.stats["true_resid"] > 1e-12


def test_nan_source_reports_nan(small, dwf):
    lat, U, b, xo = small
    bad = b.copy()
    bad[0, 0, 0, 0, 0, 0, 0] = np.nan
    r = lat.cg(0.04, _to(bad), raise_on_fail=False)
    assert r.status == 5  # DWF_ERR_NAN
