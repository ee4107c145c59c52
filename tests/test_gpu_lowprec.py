"""The FP32 and FP16-storage operator of the mixed-precision solvers, element by
element against the FP64 oracle, through dwf_apply_Mpc_prec (which runs the
solvers' own inner-iteration hop launches: M_pc = M~ B, Sec. 4).

Tolerances (max |gpu - oracle| over max |oracle|), derived from the storage:
  * FP32: the input is rounded to FP32 (relative 6e-8) and every output
    element of M_pc is a sum of a few hundred FP32 products (two Wilson hops of
    8 directions with 6 complex multiply-adds per colour row, plus the
    fifth-dimension recurrences).  The worst-case bound n * u * sum|terms|
    with n ~ 100 and sum|terms| / max|out| ~ 10 is about 6e-5; the rounding
    errors are not aligned, so the observed error is far below it.  Bar: 1e-5.
  * FP16 storage: every stored spinor slice is scaled by its largest
    component and rounded to FP16 (11 significant bits: relative error at
    most 2^-11 = 4.9e-4) on input and after the first hop, and the links are
    FP16 as well; the errors of independent roundings add in quadrature over
    the terms of an output element.  Bar: 2e-3.
  * FP64: the FP64 path through the same entry point, 1e-13 (as dwf_apply_Mpc).
  * FP64 fields in FP32 arithmetic (dwf_set_fp64_arithmetic(1), the
    arithmetic of the MADWF passes' loose solves): inputs truncated to FP32
    (relative error below 2^-23) and FP32 links; the FP32 bar, 1e-5.

Shapes: the bench's fifth-dimension extents (Ls = 12 Moebius, 16 and 32
Shamir) on lattices of several site groups with a ragged tail, the
Pauli-Villars mass, an odd Ls (per-slice FP16 kernel, shared-memory epilogue)
and Moebius parameters whose inverse needs the dense fallback.

The bounded device wait: with a consumer wait limit of 0 polls every wait of
the FP32 hop kernel gives up at once; the call must report DWF_ERR_TIMEOUT
and the handle must stay usable (the kernel drains the copies it issued
before it exits, so nothing is left in flight).
"""
import numpy as np
import pytest
import torch

from oracle import dwf_oracle as O
from paper_1111_5059_gb300 import inputs as I

pytestmark = pytest.mark.gpu

M5 = 1.8
TOL = {"f64": 1e-13, "f32": 1e-5, "f16": 2e-3, "f64-in-f32": 1e-5}

CASES = [
    # dims (X,Y,Z,T), Ls, b, c, bc_t, m
    ((8, 8, 8, 8), 32, 1.0, 0.0, 1, 0.002),        # headline Ls, light mass
    ((8, 8, 8, 8), 32, 1.0, 0.0, 1, 1.0),          # Pauli-Villars mass
    ((8, 4, 4, 8), 12, 11 / 6, 5 / 6, 1, 0.002),   # headline Moebius Ls' = 12
    ((6, 2, 2, 2), 12, 11 / 6, 5 / 6, -1, 0.01),   # Vh = 24: 5 sites per group, ragged last group
    ((4, 4, 8, 8), 16, 1.0, 0.0, -1, 0.01),        # Ls = 16 (the mixed CG workload's)
    ((4, 2, 4, 6), 16, 1.5, 0.5, 1, 0.05),         # Moebius ladder parameters, Ls = 16
    ((2, 4, 2, 4), 5, 11 / 6, 5 / 6, -1, 0.3),     # odd Ls
    ((4, 4, 4, 4), 8, 0.5, 0.55, 1, 0.1),          # |c/b| > 1: dense fifth-dimension fallback
]


def _to(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"{c[0]}x{c[1]}-b{c[2]:.2f}-c{c[3]:.2f}-m{c[5]}")
def case(request, dwf):
    dims, Ls, b, c, bc_t, m = request.param
    U = I.gauge_field(21, dims, 0.6)
    psi = I.gaussian_spinor(22, dims, Ls)
    lat = dwf.Lattice(dims, Ls, M5, b, c, bc_t)
    lat.set_gauge(_to(U))
    eo = O.EO(U, m, M5, Ls, b, c, bc_t)
    want = {dag: eo.Mpc(psi * eo.even, dag) for dag in (False, True)}
    yield lat, psi, m, want, eo
    lat.close()


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("dag", [False, True])
def test_Mpc_at_storage_precision_matches_oracle(case, prec, dag):
    lat, psi, m, want, eo = case
    got = lat.apply_Mpc_prec(m, _to(psi), prec=prec, dag=dag).cpu().numpy()
    err = _rel(got, want[dag])
    assert err < TOL[prec], (prec, dag, err)
    assert np.all(got[np.broadcast_to(eo.odd, got.shape)] == 0)
    if prec != "f64":
        # the rounding is really that of the storage: not FP64-exact
        assert err > 1e-12


def test_timed_out_wait_reports_and_handle_stays_usable(dwf):
    dims, Ls, m = (8, 8, 8, 8), 16, 0.01
    U = I.gauge_field(23, dims, 0.5)
    psi = _to(I.gaussian_spinor(24, dims, Ls))
    lat = dwf.Lattice(dims, Ls, M5)
    lat.set_gauge(_to(U))
    ref = lat.apply_Mpc_prec(m, psi, prec="f32")
    lat.set_wait_limit(0)
    with pytest.raises(dwf.DWFError) as ei:
        lat.apply_Mpc_prec(m, psi, prec="f32")
    assert ei.value.status == 6 and "bounded device wait" in str(ei.value)
    # a second timed-out launch on the same handle reports again
    with pytest.raises(dwf.DWFError, match="TIMEOUT"):
        lat.apply_Mpc_prec(m, psi, prec="f32", dag=True)
    lat.set_wait_limit(-1)
    again = lat.apply_Mpc_prec(m, psi, prec="f32")
    assert torch.equal(again, ref)
    torch.cuda.synchronize()
    lat.close()


@pytest.mark.parametrize("dag", [False, True])
def test_Mpc_on_fp64_fields_in_fp32_arithmetic(case, dag):
    lat, psi, m, want, eo = case
    lat.set_fp64_arithmetic(1)
    try:
        got = lat.apply_Mpc_prec(m, _to(psi), prec="f64", dag=dag).cpu().numpy()
    finally:
        lat.set_fp64_arithmetic(0)
    err = _rel(got, want[dag])
    assert err < TOL["f64-in-f32"], err
    assert err > 1e-12  # the FP32 path did run
    back = lat.apply_Mpc_prec(m, _to(psi), prec="f64", dag=dag).cpu().numpy()
    assert _rel(back, want[dag]) < TOL["f64"]  # and mode 0 restores FP64
