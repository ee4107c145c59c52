"""GPU parity of the operators (through the C ABI) against the FP64 oracle,
element by element, on lattices the oracle handles in seconds.

Shapes cover several CTA tiles with a ragged tail (Vh not a multiple of the
sites per CTA), odd and maximal Ls, both t boundary conditions, Shamir and
Moebius.  FP64 bar: max |gpu - oracle| <= 1e-13 * max |oracle|.
"""
import numpy as np
import pytest
import torch

from oracle import dwf_oracle as O
from paper_1111_5059_gb300 import inputs as I

pytestmark = pytest.mark.gpu

M5 = 1.8
TOL64 = 1e-13

CASES = [
    # dims (X,Y,Z,T), Ls, b, c, bc_t, m
    ((4, 4, 4, 4), 8, 1.0, 0.0, 1, 0.04),      # the 4^4 x 8 small case
    ((6, 2, 2, 2), 8, 1.0, 0.0, -1, 0.1),      # Vh = 24: ragged tail of a 16-site CTA
    ((4, 2, 4, 6), 12, 1.5, 0.5, 1, 0.002),    # Moebius, Ls = 12 (10 sites per CTA, ragged)
    ((2, 4, 2, 4), 5, 11 / 6, 5 / 6, -1, 0.3),  # odd Ls
    ((2, 2, 2, 2), 1, 1.0, 0.0, 1, 0.5),        # Ls = 1 (both walls on one slice)
    ((2, 2, 2, 4), 64, 1.2, 0.2, 1, 0.01),      # maximum Ls
]


def _to(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(params=CASES, ids=lambda c: f"{c[0]}x{c[1]}-b{c[2]:.2f}-c{c[3]:.2f}-bc{c[4]}")
def setup(request, dwf):
    dims, Ls, b, c, bc_t, m = request.param
    U = I.gauge_field(3, dims, 0.5)
    psi = I.gaussian_spinor(4, dims, Ls)
    lat = dwf.Lattice(dims, Ls, M5, b, c, bc_t)
    lat.set_gauge(_to(U))
    yield lat, U, psi, (dims, Ls, b, c, bc_t, m)
    lat.close()


def test_apply_M_matches_oracle(setup):
    lat, U, psi, (dims, Ls, b, c, bc_t, m) = setup
    got = lat.apply_M(m, _to(psi)).cpu().numpy()
    want = O.dwf_op(U, psi, m, M5, b, c, bc_t)
    assert _rel(got, want) < TOL64


def test_apply_Mdag_matches_oracle(setup):
    lat, U, psi, (dims, Ls, b, c, bc_t, m) = setup
    got = lat.apply_M(m, _to(psi), dag=True).cpu().numpy()
    want = O.dwf_op(U, psi, m, M5, b, c, bc_t, dag=True)
    assert _rel(got, want) < TOL64


def test_apply_MdagM_matches_oracle(setup):
    lat, U, psi, (dims, Ls, b, c, bc_t, m) = setup
    got = lat.apply_MdagM(m, _to(psi)).cpu().numpy()
    want = O.dwf_op(U, O.dwf_op(U, psi, m, M5, b, c, bc_t), m, M5, b, c, bc_t, dag=True)
    assert _rel(got, want) < TOL64


@pytest.mark.parametrize("dag", [False, True])
def test_apply_Mpc_matches_oracle(setup, dag):
    lat, U, psi, (dims, Ls, b, c, bc_t, m) = setup
    eo = O.EO(U, m, M5, Ls, b, c, bc_t)
    got = lat.apply_Mpc(m, _to(psi), dag=dag).cpu().numpy()
    want = eo.Mpc(psi * eo.even, dag)
    assert _rel(got, want) < TOL64
    assert np.all(got[np.broadcast_to(eo.odd, got.shape)] == 0)


def test_apply_is_deterministic(setup):
    lat, U, psi, (dims, Ls, b, c, bc_t, m) = setup
    x = _to(psi)
    a = lat.apply_MdagM(m, x)
    bb = lat.apply_MdagM(m, x)
    assert torch.equal(a, bb)


def test_invalid_arguments_are_reported(dwf):
    with pytest.raises(dwf.DWFError, match="INVALID_ARG"):
        dwf.Lattice((3, 4, 4, 4), 8)
    with pytest.raises(dwf.DWFError, match="INVALID_ARG"):
        dwf.Lattice((4, 4, 4, 4), 0)
    lat = dwf.Lattice((4, 4, 4, 4), 4)
    x = torch.zeros(lat.spinor_shape, dtype=torch.complex128, device="cuda")
    with pytest.raises(dwf.DWFError, match="gauge field not set"):
        lat.apply_M(0.1, x)
    with pytest.raises(ValueError):
        lat.apply_M(0.1, torch.zeros((5, 4, 4, 4, 4, 4, 3), dtype=torch.complex128, device="cuda"))
    with pytest.raises(TypeError):
        lat.apply_M(0.1, torch.zeros(lat.spinor_shape, dtype=torch.complex64, device="cuda"))
    lat.close()


def test_large_lattice_sampled_sites(dwf):
    """16^3 x 32 x Ls=16 (the 2nd workload's lattice): D(m) psi at sampled 5D
    sites against the oracle's one-site evaluation."""
    dims, Ls, m = (16, 16, 16, 32), 16, 0.01
    U = I.gauge_field(2, dims, 0.5)
    psi = I.gaussian_spinor(2, dims, Ls)
    lat = dwf.Lattice(dims, Ls, M5, 1.0, 0.0, 1)
    lat.set_gauge(_to(U))
    got = lat.apply_M(m, _to(psi)).cpu().numpy()
    rng = np.random.default_rng(0)
    sites = [(int(rng.integers(Ls)), int(rng.integers(32)), int(rng.integers(16)), int(rng.integers(16)),
              int(rng.integers(16))) for _ in range(48)]
    sites += [(0, 0, 0, 0, 0), (Ls - 1, 31, 15, 15, 15), (0, 31, 0, 15, 0)]
    want = O.dwf_op_at(U, psi, m, M5, 1.0, 0.0, 1, sites)
    g = np.array([got[s] for s in sites])
    assert _rel(g, want) < TOL64
    lat.close()
