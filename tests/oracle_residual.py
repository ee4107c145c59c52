"""Oracle residuals of GPU solutions at sizes where one whole-lattice pass of
the oracle is too slow or too large: the residual b - D(m) x restricted to a
slab of consecutive timeslices, computed by the oracle's own operator.

D(m) couples a timeslice only to its two neighbours in t (the Wilson hop) and
to nothing else outside it (the fifth-dimension operators act within one 4D
site), so (D x) on the timeslices t0 .. t0+n-1 is exactly the oracle's D(m)
applied on the sub-lattice of timeslices t0-1 .. t0+n (periodic in its own
t), read on its interior rows: the wrap of the sub-lattice only reaches its
first and last rows, which are discarded.  Test infrastructure only.
"""
import numpy as np

from oracle import dwf_oracle as O


def slab_rows(T, t0, n):
    """Timeslices t0-1 .. t0+n (mod T): the slab with one halo slice on each side."""
    return [(t0 - 1 + k) % T for k in range(n + 2)]


def slab_residual(U, x_slab, b_slab, rows, m, M5, b5=1.0, c5=0.0):
    """(|b - D(m) x|^2, |b|^2) over the interior timeslices rows[1:-1].

    U: whole gauge field (periodic in t); x_slab: the solution on `rows`
    (the slab and its two halo slices, as returned by slab_rows); b_slab: the
    source on rows[1:-1]."""
    Us = np.ascontiguousarray(U[:, rows])
    y = O.dwf_op(Us, x_slab, m, M5, b5, c5, 1)
    r = b_slab - y[:, 1:-1]
    return O.norm2(r), O.norm2(b_slab)


def patch_index(center, dims, half=3):
    """Indices (per direction x, y, z, t) of the 2*half sites around `center`
    (periodic in the whole lattice), with the centre at local index `half`."""
    return [[(c - half + k) % L for k in range(2 * half)] for c, L in zip(center, dims)]


def Mpc_at(U, x, m, M5, center, b5=1.0, c5=0.0, dag=False):
    """M_pc x (or M_pc^+ x) at one even site of the whole lattice, from the
    oracle's even-odd operator on the 6^4 patch around it.

    M_pc = A - M_eo A^-1 M_oe reaches two sites from its output site (an odd
    neighbour and that neighbour's even neighbours), so every site the centre
    depends on lies inside the patch with its real field values; the patch's
    own periodic wrap only changes sites at local index 0 and 5 in some
    direction, two or more steps from the centre along it, which feed the
    centre through no path of length two.  The patch origin has the centre's
    parity, so patch and lattice agree on which sites are even.  U: boundary
    layout [4][T][Z][Y][X][3][3] (t periodic); x: [Ls][T][Z][Y][X][4][3];
    center: (x, y, z, t) with x + y + z + t even.  Returns [Ls][4][3]."""
    X, Y, Z, T = U.shape[4], U.shape[3], U.shape[2], U.shape[1]
    assert sum(center) % 2 == 0
    ix, iy, iz, it = patch_index(center, (X, Y, Z, T))
    Up = U[:, it][:, :, iz][:, :, :, iy][:, :, :, :, ix]
    xp = x[:, it][:, :, iz][:, :, :, iy][:, :, :, :, ix]
    Ls = x.shape[0]
    eo = O.EO(np.ascontiguousarray(Up), m, M5, Ls, b5, c5, 1)
    y = eo.Mpc(np.ascontiguousarray(xp) * eo.even, dag)
    return y[:, 3, 3, 3, 3]
