"""Thin Python binding of ``libdwf.so`` (C ABI in ``include/dwf.h``).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  Fields are torch CUDA tensors (complex128, the
boundary layouts of ``dwf.h``); PyTorch provides device memory and streams.
There is no CPU fallback: a missing library or a CPU tensor raises.
"""
from __future__ import annotations

import ctypes
import os
import weakref
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


MADWF_MAX_PASSES = 16


class MadwfParams(ctypes.Structure):
    _fields_ = [("n_dc", ctypes.c_int), ("tol_pv", ctypes.c_double), ("tol_mob", ctypes.c_double),
                ("tol_final", ctypes.c_double), ("inner", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("delta", ctypes.c_double), ("check_every", ctypes.c_int)]


class MadwfStats(ctypes.Structure):
    _fields_ = [("total", Stats), ("pv", Stats), ("mobius", Stats), ("final_cg", Stats),
                ("passes", ctypes.c_int), ("pass_resid", ctypes.c_double * MADWF_MAX_PASSES)]

    def as_dict(self):
        return {"total": self.total.as_dict(), "pv": self.pv.as_dict(), "mobius": self.mobius.as_dict(),
                "final_cg": self.final_cg.as_dict(), "passes": self.passes,
                "pass_resid": [self.pass_resid[i] for i in range(self.passes)]}


DWF_MAX_RHS = 16


class MultiOptions(ctypes.Structure):
    _fields_ = [("use_graph", ctypes.c_int), ("autotune", ctypes.c_int)]


class MultiInfo(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("tune_seconds", ctypes.c_double),
                ("graphs", ctypes.c_int), ("replays", ctypes.c_longlong), ("iterations", ctypes.c_int),
                ("seconds", ctypes.c_double), ("launches", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Quotient(ctypes.Structure):
    _fields_ = [("m1", ctypes.c_double), ("m2", ctypes.c_double)]


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
        "dwf_cg_multi": [H, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                         ctypes.POINTER(CGParams), ctypes.POINTER(MultiOptions), ctypes.POINTER(Stats),
                         ctypes.POINTER(MultiInfo)],
        "madwf_solve": [H, H, ctypes.c_double, _VP, _VP, ctypes.POINTER(MadwfParams), ctypes.POINTER(MadwfStats)],
        "dwf_apply_Mpc_noalloc": [H, ctypes.c_double, ctypes.c_int, _VP, _VP],
        "dwf_host_alloc": [ctypes.c_size_t, ctypes.POINTER(_VP)],
        "dwf_host_free": [_VP],
        "dwf_force": [H, ctypes.c_int, ctypes.POINTER(Quotient), ctypes.POINTER(_VP), ctypes.POINTER(_VP), _VP, _VP,
                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(CGParams), ctypes.POINTER(Stats)],
        "dwf_action": [H, ctypes.c_int, ctypes.POINTER(Quotient), ctypes.POINTER(_VP), ctypes.POINTER(CGParams),
                       ctypes.POINTER(ctypes.c_double)],
        "fgi_link_update": [H, _VP, ctypes.c_double, _VP, _VP],
        "dwf_momentum_update": [H, _VP, ctypes.c_double, _VP],
        "dwf_kinetic": [H, _VP, ctypes.POINTER(ctypes.c_double)],
        "fgi_step": [H, ctypes.c_int, ctypes.POINTER(Quotient), ctypes.POINTER(_VP), _VP, _VP, ctypes.c_double,
                     ctypes.c_int, ctypes.POINTER(CGParams), ctypes.POINTER(Stats), ctypes.POINTER(ctypes.c_int)],
        "dwf_set_kernel_timing": [H, ctypes.c_int],
        "dwf_get_kernel_time": [H, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)],
        "dwf_get_launch_count": [H, ctypes.POINTER(ctypes.c_longlong)],
        "dwf_apply_Mpc_prec": [H, ctypes.c_double, ctypes.c_int, ctypes.c_int, _VP, _VP],
        "dwf_set_wait_limit": [H, ctypes.c_longlong],
        "dwf_heatbath": [H, Quotient, _VP, _VP, ctypes.POINTER(CGParams), ctypes.POINTER(Stats)],
        "dwf_set_fp64_arithmetic": [H, ctypes.c_int],
        "dwf_md_trajectory": [H, ctypes.c_int, ctypes.POINTER(Quotient), ctypes.POINTER(_VP), _VP, _VP,
                              ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(CGParams),
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(Stats), ctypes.POINTER(ctypes.c_int)],
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


def host_empty(shape, dtype=torch.complex128) -> torch.Tensor:
    """A page-locked host tensor from dwf_host_alloc (huge-page backed; see
    include/dwf.h): the host side of copies to and from the GPU.  The memory
    is released when the returned tensor and every view of it are gone."""
    numel = 1
    for n in shape:
        numel *= int(n)
    nbytes = numel * torch.empty((), dtype=dtype).element_size()
    # torch reports registered host memory as pinned only once its own CUDA
    # state is initialised
    torch.cuda.init()
    p = _VP()
    _check(lib().dwf_host_alloc(nbytes, ctypes.byref(p)))
    buf = (ctypes.c_char * nbytes).from_address(p.value)
    weakref.finalize(buf, lib().dwf_host_free, _VP(p.value))
    # torch.frombuffer keeps `buf` alive for as long as the tensor's storage
    return torch.frombuffer(buf, dtype=dtype, count=numel).view(tuple(shape))


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
        """Pack the links (complex128 [4][T][Z][Y][X][3][3] on this lattice's
        GPU) into the library's FP64/FP32/FP16 copies."""
        self._call(lib().dwf_set_gauge, _VP(_ptr(U, self.gauge_shape)))

    def _new(self):
        return torch.empty(self.spinor_shape, dtype=torch.complex128, device=self.device)

    def apply_M(self, m: float, x: torch.Tensor, dag: bool = False, out=None) -> torch.Tensor:
        """D(m) x (or D(m)^+ x) on the whole 5D lattice: D_DW of Sec. 4, Eq. dirac_eq
        (Moebius with this lattice's b, c)."""
        out = self._new() if out is None else out
        fn = lib().dwf_apply_Mdag if dag else lib().dwf_apply_M
        self._call(fn, float(m), _VP(_ptr(x, self.spinor_shape)), _VP(_ptr(out, self.spinor_shape)))
        return out

    def apply_MdagM(self, m: float, x: torch.Tensor, out=None) -> torch.Tensor:
        """D(m)^+ D(m) x on the whole 5D lattice."""
        out = self._new() if out is None else out
        self._call(lib().dwf_apply_MdagM, float(m), _VP(_ptr(x, self.spinor_shape)),
                   _VP(_ptr(out, self.spinor_shape)))
        return out

    def apply_Mpc(self, m: float, x: torch.Tensor, dag: bool = False, out=None) -> torch.Tensor:
        """The even-odd Schur operator M_pc = A - M_eo A^-1 M_oe (or its adjoint) on
        the even sites of x; odd sites of the result are zero."""
        out = self._new() if out is None else out
        self._call(lib().dwf_apply_Mpc, float(m), int(bool(dag)), _VP(_ptr(x, self.spinor_shape)),
                   _VP(_ptr(out, self.spinor_shape)))
        return out

    def apply_Mpc_prec(self, m: float, x: torch.Tensor, prec: str = "f32", dag: bool = False,
                       out=None) -> torch.Tensor:
        """M_pc (or M_pc^+) evaluated with fields stored at `prec` ("f64", "f32",
        "f16") through the launches the solvers' inner iterations use (see
        include/dwf.h, dwf_apply_Mpc_prec)."""
        out = self._new() if out is None else out
        self._call(lib().dwf_apply_Mpc_prec, float(m), int(bool(dag)), _PREC[prec], _VP(_ptr(x, self.spinor_shape)),
                   _VP(_ptr(out, self.spinor_shape)))
        return out

    def set_wait_limit(self, polls: int = -1):
        """Polls of the hop kernel's bounded consumer waits on later launches
        (-1: the default; 0: every wait gives up at once)."""
        self._call(lib().dwf_set_wait_limit, int(polls))

    def set_fp64_arithmetic(self, mode: int = 0):
        """Arithmetic of the hops on FP64 fields (include/dwf.h,
        dwf_set_fp64_arithmetic): 0 FP64, 1 FP32."""
        self._call(lib().dwf_set_fp64_arithmetic, int(mode))

    def apply_Mpc_noalloc(self, m: float, x: torch.Tensor, out: torch.Tensor, dag: bool = False) -> torch.Tensor:
        """apply_Mpc into a caller-provided `out`; the library allocates no
        device memory during the call (for callers whose allocator owns the
        device memory or that may not stall on the driver; see include/dwf.h)."""
        self._call(lib().dwf_apply_Mpc_noalloc, float(m), int(bool(dag)), _VP(_ptr(x, self.spinor_shape)),
                   _VP(_ptr(out, self.spinor_shape)))
        return out

    def cg(self, m: float, b: torch.Tensor, x0=None, tol=1e-10, max_iter=100000, inner="f64",
           delta=0.1, check_every=10, raise_on_fail=True, out=None) -> SolveResult:
        """Solve D(m) x = b (Sec. 4, Eq. dirac_eq) by even-odd CG on the normal
        equations to |b - D(m) x| / |b| <= tol: plain FP64 (inner="f64") or mixed
        precision with FP32 / FP16-stored inner iterations and FP64 reliable
        updates (delta).  x0 is the initial guess (zeros if None).  `out`, if
        given, receives the solution (it is overwritten by the guess first)."""
        if out is None:
            x = torch.zeros_like(b) if x0 is None else x0.clone()
        else:
            x = out
            if x0 is None:
                x.zero_()
            else:
                x.copy_(x0)
        prm = CGParams(float(tol), int(max_iter), _PREC[inner], float(delta), int(check_every))
        st = Stats()
        with torch.cuda.device(self.device):
            status = lib().dwf_cg(self._h, float(m), _VP(_ptr(b, self.spinor_shape)),
                                  _VP(_ptr(x, self.spinor_shape)), ctypes.byref(prm), ctypes.byref(st))
        if status != 0 and raise_on_fail:
            _check(status, self._h)
        return SolveResult(x, st.as_dict(), status)

    def cg_multi(self, masses, bs, x0s=None, tol=1e-10, max_iter=100000, inner="f32", delta=0.1, check_every=10,
                 use_graph=True, autotune=True, raise_on_fail=True):
        """Solve D(m_r) x_r = b_r for a ladder of masses together (see
        include/dwf.h, dwf_cg_multi).  Returns (xs, per-RHS stats, info, status)."""
        n = len(masses)
        if len(bs) != n or (x0s is not None and len(x0s) != n):
            raise ValueError("masses, sources and guesses must have the same length")
        xs = [torch.zeros_like(b) if x0s is None else x0s[i].clone() for i, b in enumerate(bs)]
        prm = CGParams(float(tol), int(max_iter), _PREC[inner], float(delta), int(check_every))
        opt = MultiOptions(int(bool(use_graph)), int(bool(autotune)))
        st = (Stats * n)()
        info = MultiInfo()
        ms = (ctypes.c_double * n)(*[float(m) for m in masses])
        with torch.cuda.device(self.device):
            status = lib().dwf_cg_multi(self._h, n, ms, _ptr_array(bs, self.spinor_shape),
                                        _ptr_array(xs, self.spinor_shape), ctypes.byref(prm), ctypes.byref(opt),
                                        st, ctypes.byref(info))
        if status != 0 and raise_on_fail:
            _check(status, self._h)
        return xs, [st[i].as_dict() for i in range(n)], info.as_dict(), status


def madwf_solve(outer: Lattice, inner: Lattice, m: float, b: torch.Tensor, n_dc=3, tol_pv=1e-8, tol_mob=1e-5,
                tol_final=1e-10, inner_prec="f32", max_iter=100000, delta=0.1, check_every=10,
                raise_on_fail=True, out=None) -> SolveResult:
    """Moebius-accelerated solve of D_DW(m) x = b on `outer` through the Moebius
    lattice `inner` (see include/dwf.h, madwf_solve); `out`, if given,
    receives the solution."""
    x = torch.empty_like(b) if out is None else out
    prm = MadwfParams(int(n_dc), float(tol_pv), float(tol_mob), float(tol_final), _PREC[inner_prec],
                      int(max_iter), float(delta), int(check_every))
    st = MadwfStats()
    with torch.cuda.device(outer.device):
        status = lib().madwf_solve(outer.handle, inner.handle, float(m), _VP(_ptr(b, outer.spinor_shape)),
                                   _VP(_ptr(x, outer.spinor_shape)), ctypes.byref(prm), ctypes.byref(st))
    if status != 0 and raise_on_fail:
        _check(status, outer.handle)
    return SolveResult(x, st.as_dict(), status)


# --------------------------------------------------------------------------- action, force, integrator


def _terms(terms):
    arr = (Quotient * len(terms))(*[Quotient(float(a), float(b)) for a, b in terms])
    return arr


def _ptr_array(ts, shape):
    return (_VP * len(ts))(*[_VP(_ptr(t, shape)) if t is not None else _VP() for t in ts])


def force(lat: Lattice, terms, phis, want_force=True, want_grad=False, X_io=None, tol=1e-12, inner="f64",
          max_iter=100000, delta=0.1, check_every=10):
    """Quotient-action value, force components and/or matrix gradient (see
    include/dwf.h, dwf_force).  Returns (S, F or None, G or None, stats)."""
    V = (4,) + tuple(reversed(lat.dims))
    F = torch.empty(V + (8,), dtype=torch.float64, device=lat.device) if want_force else None
    G = torch.empty(V + (3, 3), dtype=torch.complex128, device=lat.device) if want_grad else None
    S = ctypes.c_double()
    st = Stats()
    prm = CGParams(float(tol), int(max_iter), _PREC[inner], float(delta), int(check_every))
    xio = _ptr_array(X_io, lat.spinor_shape) if X_io is not None else None
    lat._call(lib().dwf_force, len(terms), _terms(terms), _ptr_array(phis, lat.spinor_shape), xio,
              _VP(_ptr(F, dtype=torch.float64)) if F is not None else _VP(),
              _VP(_ptr(G)) if G is not None else _VP(), ctypes.byref(S), ctypes.byref(prm), ctypes.byref(st))
    return S.value, F, G, st.as_dict()


def action_value(lat: Lattice, terms, phis, tol=1e-12, inner="f64", max_iter=100000, delta=0.1,
                 check_every=10) -> float:
    """The quotient action alone (see include/dwf.h, dwf_action)."""
    S = ctypes.c_double()
    prm = CGParams(float(tol), int(max_iter), _PREC[inner], float(delta), int(check_every))
    lat._call(lib().dwf_action, len(terms), _terms(terms), _ptr_array(phis, lat.spinor_shape), ctypes.byref(prm),
              ctypes.byref(S))
    return S.value


def fgi_link_update(lat: Lattice, X: torch.Tensor, coeff: float, U_in: torch.Tensor, U_out=None) -> torch.Tensor:
    """U_out = exp(coeff * X^j T_j) U_in (Sec. 2 force-gradient update)."""
    U_out = torch.empty_like(U_in) if U_out is None else U_out
    lat._call(lib().fgi_link_update, _VP(_ptr(X, dtype=torch.float64)), float(coeff),
              _VP(_ptr(U_in, lat.gauge_shape)), _VP(_ptr(U_out, lat.gauge_shape)))
    return U_out


def momentum_update(lat: Lattice, F: torch.Tensor, coeff: float, p: torch.Tensor):
    """p += coeff * F on su(3) components (the P step of Sec. 2), in place."""
    lat._call(lib().dwf_momentum_update, _VP(_ptr(F, dtype=torch.float64)), float(coeff),
              _VP(_ptr(p, dtype=torch.float64)))


def kinetic(lat: Lattice, p: torch.Tensor) -> float:
    """1/2 sum (p^j)^2 in FP64 (the kinetic part of H, Sec. 2)."""
    T = ctypes.c_double()
    lat._call(lib().dwf_kinetic, _VP(_ptr(p, dtype=torch.float64)), ctypes.byref(T))
    return T.value


def fgi_step(lat: Lattice, terms, phis, U: torch.Tensor, p: torch.Tensor, tau: float, forecast=True, tol=1e-12,
             inner="f64", max_iter=100000):
    """One force-gradient PQPQP step, U and p updated in place.  Returns
    (stats, (iterations of F(U), iterations of F(U')) in the force-gradient step)."""
    st = Stats()
    fg = (ctypes.c_int * 2)()
    prm = CGParams(float(tol), int(max_iter), _PREC[inner], 0.1, 10)
    lat._call(lib().fgi_step, len(terms), _terms(terms), _ptr_array(phis, lat.spinor_shape),
              _VP(_ptr(U, lat.gauge_shape)), _VP(_ptr(p, dtype=torch.float64)), float(tau), int(bool(forecast)),
              ctypes.byref(prm), ctypes.byref(st), fg)
    return st.as_dict(), (fg[0], fg[1])


def heatbath(lat: Lattice, term, eta: torch.Tensor, tol=1e-12, inner="f64", max_iter=100000, delta=0.1):
    """phi = M2^-+ M1^+ eta for the quotient term (m1, m2) (see include/dwf.h,
    dwf_heatbath): the term's action at this gauge field is |eta_e|^2.
    Returns (phi, stats)."""
    phi = torch.empty_like(eta)
    st = Stats()
    prm = CGParams(float(tol), int(max_iter), _PREC[inner], float(delta), 10)
    lat._call(lib().dwf_heatbath, Quotient(float(term[0]), float(term[1])), _VP(_ptr(eta, lat.spinor_shape)),
              _VP(_ptr(phi, lat.spinor_shape)), ctypes.byref(prm), ctypes.byref(st))
    return phi, st.as_dict()


INTEGRATORS = {"fgi": 0, "omelyan": 1}


def md_trajectory(lat: Lattice, terms, phis, U: torch.Tensor, p: torch.Tensor, tau: float, nsteps: int,
                  integrator="fgi", forecast=True, tol=1e-12, inner="f64", max_iter=100000, delta=0.1):
    """A molecular-dynamics trajectory (see include/dwf.h, dwf_md_trajectory); U and p
    are updated in place.  Returns (H0, H1, stats, force evaluations)."""
    H0, H1 = ctypes.c_double(), ctypes.c_double()
    st = Stats()
    nf = ctypes.c_int()
    prm = CGParams(float(tol), int(max_iter), _PREC[inner], float(delta), 10)
    lat._call(lib().dwf_md_trajectory, len(terms), _terms(terms), _ptr_array(phis, lat.spinor_shape),
              _VP(_ptr(U, lat.gauge_shape)), _VP(_ptr(p, dtype=torch.float64)), float(tau), int(nsteps),
              INTEGRATORS[integrator], int(bool(forecast)), ctypes.byref(prm), ctypes.byref(H0), ctypes.byref(H1),
              ctypes.byref(st), ctypes.byref(nf))
    return H0.value, H1.value, st.as_dict(), nf.value


def hamiltonian(lat: Lattice, terms, phis, U: torch.Tensor, p: torch.Tensor, tol=1e-12) -> float:
    """H = 1/2 sum (p^j)^2 + S_f (FP64); sets the lattice's gauge field to U."""
    lat.set_gauge(U)
    S, _, _, _ = force(lat, terms, phis, want_force=False, tol=tol)
    return kinetic(lat, p) + S


class QuotientAction(torch.autograd.Function):
    """S(U) for a set of quotient terms; backward returns the library's
    complex-matrix gradient 2 dS / d conj(U) (torch's convention), computed
    by the adjoint force kernel."""

    @staticmethod
    def forward(ctx, U, lat, terms, phis, tol):
        lat.set_gauge(U.detach())
        S, _, G, _ = force(lat, terms, phis, want_force=False, want_grad=True, tol=tol)
        ctx.save_for_backward(G)
        return torch.tensor(S, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(ctx, gS):
        (G,) = ctx.saved_tensors
        return gS.to(G.dtype) * G, None, None, None, None


def action(lat: Lattice, U: torch.Tensor, terms, phis, tol=1e-12) -> torch.Tensor:
    """Differentiable quotient action (torch.autograd)."""
    return QuotientAction.apply(U, lat, terms, phis, tol)
