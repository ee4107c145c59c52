"""Page-locked, huge-page-backed host buffers (dwf_host_alloc / dwf_host_free)
as the host side of the copies around a solve.

  * host_empty returns zeroed memory that torch sees as pinned; data copied
    host -> device -> host through it comes back bit-exact, for a buffer
    smaller than one huge page and one spanning several;
  * a solve whose source and solution go through such buffers gives the same
    solution as one from ordinary device tensors;
  * freeing (the tensor going out of scope) and allocating again works, and
    the library reports a pointer it did not allocate.
"""
import ctypes
import gc

import numpy as np
import pytest
import torch

from paper_1111_5059_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(3, 5, 7), (160, 1024, 1024)])  # 1.7 KB and 2.7 GB of complex128
def test_host_buffer_round_trip(dwf, shape):
    h = dwf.host_empty(shape)
    assert h.is_pinned() and tuple(h.shape) == shape and h.dtype == torch.complex128
    assert not torch.any(h[:2] != 0) and not torch.any(h[-2:] != 0)
    g = torch.Generator().manual_seed(1)
    src = torch.randn(shape[-2:], dtype=torch.complex128, generator=g)
    h[0] = src
    h[-1] = 2 * src
    d = torch.empty(shape, dtype=torch.complex128, device="cuda")
    d.copy_(h, non_blocking=True)
    back = dwf.host_empty(shape)
    back.copy_(d, non_blocking=True)
    torch.cuda.synchronize()
    assert torch.equal(back[0], src) and torch.equal(back[-1], 2 * src)
    del h, back, d
    gc.collect()


def test_solve_through_host_buffers(dwf):
    dims, Ls = (8, 8, 8, 8), 8
    lat = dwf.Lattice(dims, Ls, 1.8)
    lat.set_gauge(torch.from_numpy(inputs.gauge_field(7, dims, 0.5)).cuda())
    arr = inputs.gaussian_spinor(7, dims, Ls)
    bh = dwf.host_empty(arr.shape)
    bh.copy_(torch.from_numpy(arr))
    xh = dwf.host_empty(arr.shape)
    bd = torch.empty(arr.shape, dtype=torch.complex128, device="cuda")
    xd = torch.empty_like(bd)
    bd.copy_(bh, non_blocking=True)
    lat.cg(0.05, bd, tol=1e-10, inner="f32", out=xd)
    xh.copy_(xd, non_blocking=True)
    torch.cuda.synchronize()
    ref = lat.cg(0.05, torch.from_numpy(arr).cuda(), tol=1e-10, inner="f32").x.cpu()
    assert torch.equal(xh, ref)
    lat.close()


def test_free_and_foreign_pointer(dwf):
    for _ in range(3):
        h = dwf.host_empty((1 << 20,))
        h.fill_(1.0)
        del h
        gc.collect()
    L = dwf.lib()
    buf = ctypes.create_string_buffer(64)
    assert L.dwf_host_free(ctypes.cast(buf, ctypes.c_void_p)) == 1
    assert np.all(dwf.host_empty((4,)).numpy() == 0)
