"""The slab residual used at the benchmark sizes (tests/oracle_residual.py)
equals the whole-lattice oracle residual restricted to the slab's
timeslices, for Shamir and Moebius, slabs inside the lattice and across its
periodic t boundary (CPU)."""
import numpy as np
import pytest

import oracle_residual as R
from oracle import dwf_oracle as O
from paper_1111_5059_gb300 import inputs as I


@pytest.mark.parametrize("b5,c5", [(1.0, 0.0), (1.5, 0.5)])
@pytest.mark.parametrize("t0,n", [(0, 2), (6, 3), (3, 1)])
def test_slab_residual_equals_whole_lattice_rows(b5, c5, t0, n):
    dims, Ls, m = (4, 2, 4, 8), 6, 0.1
    U = I.gauge_field(1, dims, 0.5)
    x = I.gaussian_spinor(2, dims, Ls)
    b = I.gaussian_spinor(3, dims, Ls)
    full = b - O.dwf_op(U, x, m, 1.8, b5, c5)
    rows = R.slab_rows(dims[3], t0, n)
    r2, b2 = R.slab_residual(U, x[:, rows], b[:, rows[1:-1]], rows, m, 1.8, b5, c5)
    assert abs(r2 - O.norm2(full[:, rows[1:-1]])) <= 1e-12 * r2
    assert b2 == O.norm2(b[:, rows[1:-1]])


@pytest.mark.parametrize("b5,c5", [(1.0, 0.0), (11 / 6, 5 / 6)])
@pytest.mark.parametrize("dag", [False, True])
def test_patch_Mpc_equals_whole_lattice_Mpc(b5, c5, dag):
    """M_pc at single even sites from a 6^4 patch equals the whole-lattice
    oracle's M_pc there (the same arithmetic: exactly), including sites next
    to the lattice's periodic boundaries and a direction of extent 6."""
    dims, Ls, m = (8, 6, 6, 8), 5, 0.002
    U = I.gauge_field(3, dims, 0.6)
    x = I.gaussian_spinor(3, dims, Ls)
    eo = O.EO(U, m, 1.8, Ls, b5, c5, 1)
    full = eo.Mpc(x * eo.even, dag)
    for c in ((0, 0, 0, 0), (7, 5, 1, 1), (3, 2, 4, 7)):
        got = R.Mpc_at(U, x, m, 1.8, c, b5, c5, dag)
        assert np.array_equal(got, full[:, c[3], c[2], c[1], c[0]])
