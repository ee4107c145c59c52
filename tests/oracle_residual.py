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
