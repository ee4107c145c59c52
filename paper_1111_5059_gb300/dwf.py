"""Thin Python binding of ``libdwf.so`` (C ABI in ``include/dwf.h``).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  Fields are torch CUDA tensors (complex128, the
boundary layouts of ``dwf.h``); PyTorch provides device memory and streams.
There is no CPU fallback: a missing library or a CPU tensor raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdwf.so")

DWF_F64, DWF_F32, DWF_F16 = 0, 1, 2
_PREC = {"f64": DWF_F64, "f32": DWF_F32, "f16": DWF_F16}
STATUS = {0: "DWF_OK", 1: "DWF_ERR_INVALID_ARG", 2: "DWF_ERR_CUDA", 3: "DWF_ERR_OOM",
          4: "DWF_ERR_NOT_CONVERGED", 5: "DWF_ERR_NAN", 6: "DWF_ERR_TIMEOUT"}


class DWFError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("Ls", ctypes.c_int), ("M5", ctypes.c_double),
                ("b", ctypes.c_double), ("c", ctypes.c_double), ("bc_t", ctypes.c_int)]


class CGParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("inner", ctypes.c_int),
                ("delta", ctypes.c_double), ("check_every", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("hop_calls", ctypes.c_longlong), ("op_count", ctypes.c_longlong),
                ("true_resid", ctypes.c_double), ("seconds", ctypes.c_double),
                ("launches", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_VP = ctypes.c_void_p


def _declare(lib):
    H = _VP
    sigs = {
        "dwf_create_lattice": [ctypes.POINTER(Params), _VP, ctypes.POINTER(H)],
        "dwf_destroy_lattice": [H],
        "dwf_set_gauge": [H, _VP],
        "dwf_apply_M": [H, ctypes.c_double, _VP, _VP],
        "dwf_apply_Mdag": [H, ctypes.c_double, _VP, _VP],
        "dwf_apply_MdagM": [H, ctypes.c_double, _VP, _VP],
        "dwf_apply_Mpc": [H, ctypes.c_double, ctypes.c_int, _VP, _VP],
        "dwf_cg": [H, ctypes.c_double, _VP, _VP, ctypes.POINTER(CGParams), ctypes.POINTER(Stats)],
        "dwf_set_kernel_timing": [H, ctypes.c_int],
        "dwf_get_kernel_time": [H, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)],
        "dwf_get_launch_count": [H, ctypes.POINTER(ctypes.c_longlong)],
    }
    for name, args in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.dwf_last_error.argtypes = [H]
    lib.dwf_last_error.restype = ctypes.c_char_p


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1111_5059_gb300.build.build(); "
                               "this package has no CPU fallback")
        _lib = ctypes.CDLL(LIB_PATH)
        _declare(_lib)
    return _lib


def _check(status: int, handle=None):
    if status != 0:
        msg = lib().dwf_last_error(handle).decode(errors="replace")
        raise DWFError(status, msg)


def _ptr(t: torch.Tensor, shape=None, dtype=torch.complex128) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor (this library has no CPU path)")
    if t.dtype != dtype:
        raise TypeError(f"expected dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return t.data_ptr()


@dataclass
class SolveResult:
    x: torch.Tensor
    stats: dict
    status: int


class Lattice:
    """A lattice handle: geometry, Moebius/Shamir parameters, packed gauge field."""

    def __init__(self, dims, Ls, M5=1.8, b=1.0, c=0.0, bc_t=1, stream=None, device=None):
        self.dims = tuple(int(d) for d in dims)
        self.Ls, self.M5, self.b, self.c, self.bc_t = int(Ls), float(M5), float(b), float(c), int(bc_t)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        p = Params((ctypes.c_int * 4)(*self.dims), self.Ls, self.M5, self.b, self.c, self.bc_t)
        h = _VP()
        with torch.cuda.device(self.device):
            _check(lib().dwf_create_lattice(ctypes.byref(p), _VP(self.stream.cuda_stream), ctypes.byref(h)))
        self._h = h
        X, Y, Z, T = self.dims
        self.spinor_shape = (self.Ls, T, Z, Y, X, 4, 3)
        self.gauge_shape = (4, T, Z, Y, X, 3, 3)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().dwf_destroy_lattice(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, fn, *args):
        with torch.cuda.device(self.device):
            _check(fn(self._h, *args), self._h)

    def set_kernel_timing(self, enable: bool = True):
        """Bracket hop launches with CUDA events (enabling also resets the totals)."""
        self._call(lib().dwf_set_kernel_timing, int(bool(enable)))

    def kernel_time(self, prec: str = "f32") -> dict:
        """Summed device time (ms), launches and algorithmic bytes of the hop kernels of one precision."""
        ms, n, by = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double()
        self._call(lib().dwf_get_kernel_time, _PREC[prec], ctypes.byref(ms), ctypes.byref(n), ctypes.byref(by))
        return {"ms": ms.value, "launches": n.value, "bytes": by.value}

    def launch_count(self) -> int:
        n = ctypes.c_longlong()
        self._call(lib().dwf_get_launch_count, ctypes.byref(n))
        return n.value

    def set_gauge(self, U: torch.Tensor):
        self._call(lib().dwf_set_gauge, _VP(_ptr(U, self.gauge_shape)))

    def _new(self):
        return torch.empty(self.spinor_shape, dtype=torch.complex128, device=self.device)

    def apply_M(self, m: float, x: torch.Tensor, dag: bool = False, out=None) -> torch.Tensor:
        out = self._new() if out is None else out
        fn = lib().dwf_apply_Mdag if dag else lib().dwf_apply_M
        self._call(fn, float(m), _VP(_ptr(x, self.spinor_shape)), _VP(_ptr(out, self.spinor_shape)))
        return out

    def apply_MdagM(self, m: float, x: torch.Tensor, out=None) -> torch.Tensor:
        out = self._new() if out is None else out
        self._call(lib().dwf_apply_MdagM, float(m), _VP(_ptr(x, self.spinor_shape)),
                   _VP(_ptr(out, self.spinor_shape)))
        return out

    def apply_Mpc(self, m: float, x: torch.Tensor, dag: bool = False, out=None) -> torch.Tensor:
        out = self._new() if out is None else out
        self._call(lib().dwf_apply_Mpc, float(m), int(bool(dag)), _VP(_ptr(x, self.spinor_shape)),
                   _VP(_ptr(out, self.spinor_shape)))
        return out

    def cg(self, m: float, b: torch.Tensor, x0=None, tol=1e-10, max_iter=100000, inner="f64",
           delta=0.1, check_every=10, raise_on_fail=True) -> SolveResult:
        x = torch.zeros_like(b) if x0 is None else x0.clone()
        prm = CGParams(float(tol), int(max_iter), _PREC[inner], float(delta), int(check_every))
        st = Stats()
        with torch.cuda.device(self.device):
            status = lib().dwf_cg(self._h, float(m), _VP(_ptr(b, self.spinor_shape)),
                                  _VP(_ptr(x, self.spinor_shape)), ctypes.byref(prm), ctypes.byref(st))
        if status != 0 and raise_on_fail:
            _check(status, self._h)
        return SolveResult(x, st.as_dict(), status)
