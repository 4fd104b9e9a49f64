"""Python binding of the GB300 ADMM / Toeplitz-FFT library (include/fde.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libfde.so``. Tensors are torch CUDA tensors (device memory and the
current stream come from PyTorch); there is no CPU fallback, and importing the
operators raises if the library has not been built.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
from typing import Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfde.so")

FDE_OK, FDE_EINVAL, FDE_ENOMEM, FDE_ECUDA, FDE_ENOCONV = 0, -1, -2, -3, -4
FDE_EBREAKDOWN, FDE_ENONFINITE, FDE_EUNSUPPORTED, FDE_ETIMEOUT = -5, -6, -8, -9
FDE_FP64, FDE_FP32, FDE_MIXED, FDE_MIXED_DF, FDE_MIXED_DFV = 0, 1, 2, 3, 4
FDE_OP_B, FDE_OP_BT, FDE_OP_S = 0, 1, 2


class fde_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nt", ctypes.c_int), ("T", ctypes.c_double),
                ("beta_x", ctypes.c_double), ("beta_y", ctypes.c_double), ("alpha_t", ctypes.c_double),
                ("dp", ctypes.c_double), ("dm", ctypes.c_double), ("ep", ctypes.c_double), ("em", ctypes.c_double),
                ("gamma", ctypes.c_double), ("weights", ctypes.c_int), ("time_step_mode", ctypes.c_int)]


class fde_admm_opts(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("rho", ctypes.c_double), ("tol_admm", ctypes.c_double),
                ("max_admm", ctypes.c_int), ("fixed_iters", ctypes.c_int), ("max_pcg", ctypes.c_int),
                ("inner_tol_mode", ctypes.c_int), ("inner_tol", ctypes.c_double), ("precision", ctypes.c_int),
                ("inner_tol_mixed", ctypes.c_double), ("max_refine", ctypes.c_int), ("algorithm", ctypes.c_int),
                ("c_y", ctypes.c_double), ("c_u", ctypes.c_double), ("inner_solver", ctypes.c_int),
                ("precond", ctypes.c_int), ("warm_start", ctypes.c_int), ("inner_x0", ctypes.c_int)]


class fde_admm_stats(ctypes.Structure):
    _fields_ = [("admm_iters", ctypes.c_int), ("pcg_iters", ctypes.c_int), ("refine_steps", ctypes.c_int),
                ("fp64_matvecs", ctypes.c_int), ("res_eq", ctypes.c_double), ("res_y", ctypes.c_double),
                ("res_u", ctypes.c_double), ("objective", ctypes.c_double), ("max_sub_relres", ctypes.c_double),
                ("recursive_steers", ctypes.c_int), ("copy_in_ms", ctypes.c_double),
                ("copy_out_ms", ctypes.c_double), ("float_steers", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fde_persist_cfg(ctypes.Structure):
    _fields_ = [("group_ctas", ctypes.c_int), ("timeout_s", ctypes.c_double), ("replay", ctypes.c_int),
                ("stall_group", ctypes.c_int), ("schedule", ctypes.c_int)]


class fde_persist_info(ctypes.Structure):
    _fields_ = [("commands", ctypes.c_longlong), ("groups", ctypes.c_int), ("group_ctas", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int), ("smem_bytes", ctypes.c_int), ("timeout_group", ctypes.c_int),
                ("timeout_command", ctypes.c_longlong), ("schedule", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_D = ctypes.c_double
_SIGS = {
    "fde_setup": (ctypes.c_int, [ctypes.POINTER(fde_params), ctypes.POINTER(_P), _P]),
    "fde_destroy": (None, [_P]),
    "fde_size": (ctypes.c_longlong, [_P]),
    "fde_psi": (_D, [_P]),
    "fde_matvec": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(fde_admm_opts), ctypes.c_int, _P, _P, _P]),
    "fde_precond": (ctypes.c_int, [_P, ctypes.POINTER(fde_admm_opts), ctypes.c_int, _P, _P, _P]),
    "fde_admm_solve": (ctypes.c_int, [_P, ctypes.POINTER(fde_admm_opts), _P, _P, _P, _P, _P, _P, _D, _D, _D, _D,
                                      _P, _P, _P, _P, ctypes.POINTER(fde_admm_stats), _P]),
    "fde_admm_solve_host": (ctypes.c_int, [_P, ctypes.POINTER(fde_admm_opts), _P, _P, _P, _P, _P, _P, _D, _D, _D,
                                           _D, _P, _P, _P, _P, ctypes.POINTER(fde_admm_stats), _P]),
    "fde_admm_grad": (ctypes.c_int, [_P, _P, _P, _P, _D, _P, ctypes.POINTER(ctypes.c_double), _P, _P]),
    "fde_admm_get_iterates": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "fde_admm_set_iterates": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "fde_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "fde_last_cuda_error": (ctypes.c_char_p, []),
    "fde_kernel_launches": (ctypes.c_longlong, []),
    "fde_matvec_noalloc": (ctypes.c_int, [ctypes.POINTER(fde_params), ctypes.c_int, _P, _P, _P]),
    "fde_apply_factor": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P]),
    "fde_alu_peak_probe": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), _P]),
    "fde_autotune": (ctypes.c_int, [_P, _P]),
    "fde_tiles": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "fde_set_tiles": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "fde_batch_setup": (ctypes.c_int, [ctypes.POINTER(fde_params), ctypes.c_int, ctypes.POINTER(_P), _P]),
    "fde_batch_destroy": (None, [_P]),
    "fde_batch_instance_size": (ctypes.c_longlong, [_P, ctypes.c_int]),
    "fde_batch_admm_solve": (ctypes.c_int, [_P, ctypes.POINTER(fde_admm_opts), _P, _P, _P, _P, _P, _P, _P,
                                            ctypes.POINTER(fde_admm_stats), _P]),
    "fde_batch_admm_solve_persistent": (ctypes.c_int, [_P, ctypes.POINTER(fde_admm_opts), _P, _P, _P, _P, _P, _P,
                                                       _P, ctypes.POINTER(fde_persist_cfg),
                                                       ctypes.POINTER(fde_admm_stats),
                                                       ctypes.POINTER(fde_persist_info), _P]),
}
EXPORTED = tuple(_SIGS)

_lib = None


def lib() -> ctypes.CDLL:
    """Load libfde.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with python -m paper_1907_13428_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def kernel_launches() -> int:
    """Kernel launches issued by the library so far in this process."""
    return int(lib().fde_kernel_launches())


def alu_peak(precision: int = FDE_FP64) -> float:
    """Measured fused-multiply-add peak of the current GPU in TFLOP/s."""
    v = ctypes.c_double()
    _check(lib().fde_alu_peak_probe(precision, ctypes.byref(v), _stream()), "fde_alu_peak_probe")
    return v.value


class FdeError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = lib().fde_strerror(status).decode()
        if status == FDE_ECUDA:
            msg += ": " + lib().fde_last_cuda_error().decode()
        super().__init__(f"{what}: {msg} ({status})")
        self.status = status


def _tile_prec(dfloat: bool, fp64: bool) -> int:
    if dfloat and fp64:
        raise ValueError("dfloat and fp64 name different passes")
    return FDE_MIXED_DF if dfloat else FDE_FP64 if fp64 else FDE_FP32


def _check(status: int, what: str, allow=(FDE_OK,)):
    if status not in allow:
        raise FdeError(status, what)
    return status


def _stream() -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _host_ptr(t: Optional[torch.Tensor], n: int):
    """Address of a contiguous float64 CPU tensor of n elements (pinned or pageable)."""
    if t is None:
        return None
    if t.is_cuda or not t.is_contiguous() or t.dtype != torch.float64 or t.numel() != n:
        raise ValueError(f"expected a contiguous float64 CPU tensor of {n} elements")
    return ctypes.c_void_p(t.data_ptr())


def _ptr(t: Optional[torch.Tensor], dtype=None, n=None):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("tensors must be contiguous CUDA tensors")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    if n is not None and t.numel() != n:
        raise ValueError(f"expected {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


@dataclasses.dataclass
class AdmmOptions:
    delta: float = 1.0
    rho: float = 1.618
    tol_admm: float = 1e-6
    max_admm: int = 1000
    fixed_iters: bool = False
    max_pcg: int = 1000
    inner_tol_mode: int = 1        # 0: Section 6.1 rule, 1: fixed inner_tol
    inner_tol: float = 1e-10
    precision: int = FDE_FP64
    inner_tol_mixed: float = 1e-4
    max_refine: int = 30
    algorithm: int = 1             # 2: generalized ADMM (Algorithm 2), rho in (0, 1]
    c_y: float = 0.0               # Algorithm 2: R_y = c_y I - J1, c_y >= 1
    c_u: float = 0.0               # Algorithm 2: R_u = c_u I - J2, c_u >= gamma
    inner_solver: int = 0          # 0: PCG on the normal equations, 1: MINRES on the saddle-point system
    precond: int = 0               # 0: S-tilde, 1: matching approximation S-hat (circulant D-tilde)
    warm_start: bool = False       # continue from where the previous solve on the problem ended
    inner_x0: int = 0              # sub-solve initial guess: 0 previous iterate, 1 zero (MATLAB pcg default)

    def c(self) -> fde_admm_opts:
        return fde_admm_opts(self.delta, self.rho, self.tol_admm, self.max_admm, int(self.fixed_iters), self.max_pcg,
                             self.inner_tol_mode, self.inner_tol, self.precision, self.inner_tol_mixed,
                             self.max_refine, self.algorithm, self.c_y, self.c_u, self.inner_solver, self.precond,
                             int(self.warm_start), int(self.inner_x0))


def params_struct(p) -> fde_params:
    """fde_params from any object with the fde_params field names."""
    return fde_params(p.nx, p.ny, p.nt, p.T, p.beta_x, p.beta_y, p.alpha_t, p.dp, p.dm, p.ep, p.em, p.gamma,
                      p.weights, p.time_step_mode)


class Problem:
    """Owner of an fde_problem handle (fde_setup / fde_destroy)."""

    def __init__(self, params):
        self.params = params
        h = ctypes.c_void_p()
        ps = params_struct(params)
        _check(lib().fde_setup(ctypes.byref(ps), ctypes.byref(h), _stream()), "fde_setup")
        self._h = h
        self.N = int(lib().fde_size(h))
        self.shape = (params.nt, params.nx, params.ny)
        self.psi = float(lib().fde_psi(h))

    def close(self):
        if getattr(self, "_h", None):
            lib().fde_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def matvec(self, x: torch.Tensor, op: int = FDE_OP_B, opts: Optional[AdmmOptions] = None,
               out: Optional[torch.Tensor] = None, dfloat: bool = False) -> torch.Tensor:
        """y = op(x); float64 or float32 x. dfloat: float64 B / B^T with the
        transforms in double-float arithmetic (FDE_MIXED_DF)."""
        prec = FDE_FP64 if x.dtype == torch.float64 else FDE_FP32
        if dfloat:
            if x.dtype != torch.float64:
                raise ValueError("dfloat products take float64 vectors")
            prec = FDE_MIXED_DF
        y = torch.empty_like(x) if out is None else out
        o = (opts or AdmmOptions()).c()
        _check(lib().fde_matvec(self._h, op, ctypes.byref(o), prec, _ptr(x, None, self.N), _ptr(y, x.dtype, self.N),
                                _stream()), "fde_matvec")
        return y

    def autotune(self):
        """Pick the float FFT tiles by timing (fde_autotune); returns (rows, axis) threads."""
        _check(lib().fde_autotune(self._h, _stream()), "fde_autotune")
        return self.tiles()

    def set_tiles(self, rows: int = 0, axis: int = 0, dfloat: bool = False, fp64: bool = False):
        """Fix the FFT tiles of the float (or double-float, or double) passes
        (fde_set_tiles; negative = split-halves kernel)."""
        _check(lib().fde_set_tiles(self._h, _tile_prec(dfloat, fp64), rows, axis), "fde_set_tiles")

    def tiles(self, dfloat: bool = False, fp64: bool = False):
        a, c = ctypes.c_int(), ctypes.c_int()
        _check(lib().fde_tiles(self._h, _tile_prec(dfloat, fp64), ctypes.byref(a), ctypes.byref(c)), "fde_tiles")
        return a.value, c.value

    def apply_factor(self, x: torch.Tensor, axis: int, op: int = FDE_OP_B, out=None,
                     dfloat: bool = False) -> torch.Tensor:
        """One Kronecker factor of B along x1 (axis 1) or x2 (axis 2): one kernel
        launch. dfloat: float64 vectors, double-float transform arithmetic."""
        prec = FDE_FP64 if x.dtype == torch.float64 else FDE_FP32
        if dfloat:
            if x.dtype != torch.float64:
                raise ValueError("dfloat products take float64 vectors")
            prec = FDE_MIXED_DF
        y = torch.empty_like(x) if out is None else out
        _check(lib().fde_apply_factor(self._h, axis, op, prec, _ptr(x, None, self.N), _ptr(y, x.dtype, self.N),
                                      _stream()), "fde_apply_factor")
        return y

    def precond(self, r: torch.Tensor, opts: Optional[AdmmOptions] = None,
                out: Optional[torch.Tensor] = None) -> torch.Tensor:
        prec = FDE_FP64 if r.dtype == torch.float64 else FDE_FP32
        z = torch.empty_like(r) if out is None else out
        o = (opts or AdmmOptions()).c()
        _check(lib().fde_precond(self._h, ctypes.byref(o), prec, _ptr(r, None, self.N), _ptr(z, r.dtype, self.N),
                                 _stream()), "fde_precond")
        return z

    def admm_solve(self, opts: AdmmOptions, ybar: torch.Tensor, g=None, ya=None, yb=None, ua=None, ub=None,
                   allow_noconv: bool = False, out=None):
        """Run ADMM. Bounds may be None (unbounded), Python floats or CUDA tensors.
        Returns dict(y, u, p, zu, stats, status)."""
        N = self.N
        dev = ybar.device

        def bound(b, default):
            if b is None:
                return None, default
            if isinstance(b, torch.Tensor):
                return b, default
            return None, float(b)

        ya_t, ya_s = bound(ya, -math.inf)
        yb_t, yb_s = bound(yb, math.inf)
        ua_t, ua_s = bound(ua, -math.inf)
        ub_t, ub_s = bound(ub, math.inf)
        if out is None:
            out = {k: torch.empty(N, dtype=torch.float64, device=dev) for k in ("y", "u", "p", "zu")}
        st = fde_admm_stats()
        o = opts.c()
        s = lib().fde_admm_solve(self._h, ctypes.byref(o), _ptr(ybar, torch.float64, N), _ptr(g, torch.float64, N),
                                 _ptr(ya_t, torch.float64, N), _ptr(yb_t, torch.float64, N),
                                 _ptr(ua_t, torch.float64, N), _ptr(ub_t, torch.float64, N), ya_s, yb_s, ua_s, ub_s,
                                 _ptr(out["y"]), _ptr(out["u"]), _ptr(out["p"]), _ptr(out["zu"]), ctypes.byref(st),
                                 _stream())
        _check(s, "fde_admm_solve", (FDE_OK, FDE_ENOCONV) if allow_noconv else (FDE_OK,))
        res = dict(out)
        res["stats"] = st.as_dict()
        res["status"] = s
        return res

    def admm_solve_host(self, opts: AdmmOptions, ybar: torch.Tensor, g=None, ya=None, yb=None, ua=None, ub=None,
                        allow_noconv: bool = False, out=None, want_p: bool = False, want_zu: bool = False):
        """fde_admm_solve_host: ADMM on host (CPU) float64 tensors; inputs are copied in
        and y, u (and p, z_u if asked) copied out inside the call. Bounds: None, floats or
        CPU tensors. Pinned tensors are moved by a copy kernel. Returns dict(y, u[, p, zu],
        stats, status) with CPU tensors (pinned when allocated here)."""
        N = self.N

        def bound(b, default):
            if b is None or not isinstance(b, torch.Tensor):
                return None, default if b is None else float(b)
            return b, default

        ya_t, ya_s = bound(ya, -math.inf)
        yb_t, yb_s = bound(yb, math.inf)
        ua_t, ua_s = bound(ua, -math.inf)
        ub_t, ub_s = bound(ub, math.inf)
        keys = ["y", "u"] + (["p"] if want_p else []) + (["zu"] if want_zu else [])
        if out is None:
            out = {k: torch.empty(N, dtype=torch.float64, pin_memory=torch.cuda.is_available()) for k in keys}
        st = fde_admm_stats()
        o = opts.c()
        s = lib().fde_admm_solve_host(self._h, ctypes.byref(o), _host_ptr(ybar, N), _host_ptr(g, N),
                                      _host_ptr(ya_t, N), _host_ptr(yb_t, N), _host_ptr(ua_t, N),
                                      _host_ptr(ub_t, N), ya_s, yb_s, ua_s, ub_s, _host_ptr(out["y"], N),
                                      _host_ptr(out["u"], N), _host_ptr(out.get("p"), N),
                                      _host_ptr(out.get("zu"), N), ctypes.byref(st), _stream())
        _check(s, "fde_admm_solve_host", (FDE_OK, FDE_ENOCONV) if allow_noconv else (FDE_OK,))
        res = dict(out)
        res["stats"] = st.as_dict()
        res["status"] = s
        return res

    ITERATES = ("y", "u", "zy", "zu", "p", "wy", "wu")

    def iterates(self, names: Sequence[str] = ITERATES, device=None) -> dict:
        """Iterates the last solve on this problem ended with (fde_admm_get_iterates):
        a dict of CUDA float64 tensors for the requested names among y, u, zy, zu, p,
        wy (state-box multiplier), wu."""
        bad = set(names) - set(self.ITERATES)
        if bad:
            raise ValueError(f"unknown iterates {sorted(bad)}")
        dev = torch.device("cuda") if device is None else device
        out = {k: torch.empty(self.N, dtype=torch.float64, device=dev) for k in names}
        _check(lib().fde_admm_get_iterates(self._h, *[_ptr(out.get(k)) for k in self.ITERATES], _stream()),
               "fde_admm_get_iterates")
        return out

    def set_iterates(self, it: dict):
        """Load the iterates a warm-started solve begins from (fde_admm_set_iterates);
        missing names are zero."""
        bad = set(it) - set(self.ITERATES)
        if bad:
            raise ValueError(f"unknown iterates {sorted(bad)}")
        _check(lib().fde_admm_set_iterates(self._h, *[_ptr(it.get(k), torch.float64, self.N) for k in self.ITERATES],
                                           _stream()), "fde_admm_set_iterates")

    def admm_grad(self, y: torch.Tensor, ybar: torch.Tensor, wy: Optional[torch.Tensor] = None, tol: float = 1e-12):
        """Returns (dJ/dybar [N], dJ/d(d+, d-, e+, e-) [4] float64 CPU tensor, adjoint p [N])."""
        N = self.N
        dJ = torch.empty(N, dtype=torch.float64, device=y.device)
        pv = torch.empty(N, dtype=torch.float64, device=y.device)
        coef = (ctypes.c_double * 4)()
        _check(lib().fde_admm_grad(self._h, _ptr(y, torch.float64, N), _ptr(ybar, torch.float64, N),
                                   _ptr(wy, torch.float64, N), tol, _ptr(dJ), coef, _ptr(pv), _stream()),
               "fde_admm_grad")
        return dJ, torch.tensor(list(coef), dtype=torch.float64), pv


class Batch:
    """Owner of an fde_batch: independent instances solved together in one
    CUDA-graph launch (fde_batch_admm_solve) or in one persistent cooperative
    kernel (fde_batch_admm_solve_persistent)."""

    def __init__(self, params_list):
        self.params = list(params_list)
        n = len(self.params)
        arr = (fde_params * n)(*[params_struct(p) for p in self.params])
        h = ctypes.c_void_p()
        _check(lib().fde_batch_setup(arr, n, ctypes.byref(h), _stream()), "fde_batch_setup")
        self._h = h
        self.sizes = [int(lib().fde_batch_instance_size(h, i)) for i in range(n)]
        self._out = None

    def close(self):
        if getattr(self, "_h", None):
            lib().fde_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def admm_solve(self, opts: AdmmOptions, ybars, ya=None, yb=None, ua=None, ub=None, out=None):
        """ybars: list of CUDA float64 tensors (N_i); bounds: None or lists of floats.
        Returns (ys, us, stats list). Output tensors are reused between calls so that
        the captured graph can be replayed."""
        n = len(self.sizes)
        if out is None:
            if self._out is None:
                self._out = ([torch.empty(N, dtype=torch.float64, device=ybars[0].device) for N in self.sizes],
                             [torch.empty(N, dtype=torch.float64, device=ybars[0].device) for N in self.sizes])
            out = self._out
        ys, us = out
        P = ctypes.c_void_p
        yb_ptrs = (P * n)(*[_ptr(t, torch.float64, N).value for t, N in zip(ybars, self.sizes)])
        y_ptrs = (P * n)(*[t.data_ptr() for t in ys])
        u_ptrs = (P * n)(*[t.data_ptr() for t in us])

        def arr(v):
            return None if v is None else (ctypes.c_double * n)(*[float(a) for a in v])

        st = (fde_admm_stats * n)()
        o = opts.c()
        s = lib().fde_batch_admm_solve(self._h, ctypes.byref(o), yb_ptrs, arr(ya), arr(yb), arr(ua), arr(ub), y_ptrs,
                                       u_ptrs, st, _stream())
        _check(s, "fde_batch_admm_solve")
        return ys, us, [x.as_dict() for x in st]

    def admm_solve_persistent(self, opts: AdmmOptions, ybars, ya=None, yb=None, ua=None, ub=None, out=None,
                              group_ctas: int = 0, timeout_s: float = 0.0, replay: bool = False,
                              stall_group: int = 0, schedule: int = 0, check: bool = True):
        """The same batch solve run by one persistent cooperative kernel
        (fde_batch_admm_solve_persistent; FDE_MIXED only). schedule 0: lockstep
        over the instances, 1: instance groups of group_ctas CTAs taking
        instances from a queue. replay=True issues the recorded launches one by
        one instead (reference executor). Returns (ys, us, stats list, info dict,
        status); with check=True a failing status raises FdeError."""
        n = len(self.sizes)
        if out is None:
            if self._out is None:
                self._out = ([torch.empty(N, dtype=torch.float64, device=ybars[0].device) for N in self.sizes],
                             [torch.empty(N, dtype=torch.float64, device=ybars[0].device) for N in self.sizes])
            out = self._out
        ys, us = out
        P = ctypes.c_void_p
        yb_ptrs = (P * n)(*[_ptr(t, torch.float64, N).value for t, N in zip(ybars, self.sizes)])
        y_ptrs = (P * n)(*[t.data_ptr() for t in ys])
        u_ptrs = (P * n)(*[t.data_ptr() for t in us])

        def arr(v):
            return None if v is None else (ctypes.c_double * n)(*[float(a) for a in v])

        st = (fde_admm_stats * n)()
        info = fde_persist_info()
        cfg = fde_persist_cfg(int(group_ctas), float(timeout_s), int(bool(replay)), int(stall_group), int(schedule))
        o = opts.c()
        s = lib().fde_batch_admm_solve_persistent(self._h, ctypes.byref(o), yb_ptrs, arr(ya), arr(yb), arr(ua),
                                                  arr(ub), y_ptrs, u_ptrs, ctypes.byref(cfg), st,
                                                  ctypes.byref(info), _stream())
        if check:
            _check(s, "fde_batch_admm_solve_persistent")
        return ys, us, [x.as_dict() for x in st], info.as_dict(), s


class FdeAdmmFn(torch.autograd.Function):
    """J*(ybar, d+, d-, e+, e-): optimal value of the ADMM problem. The backward
    pass is the library's adjoint (fde_admm_grad): gradient of J* with respect
    to the desired state and the four diffusion coefficients. The adjoint
    equation B^T p = -J1 (y* - ybar) - w_y* takes the state-box multiplier w_y*
    of the converged solve (fde_admm_get_iterates), so active state bounds are
    accounted for. The problem handle lives as long as the autograd graph, so a
    second backward (retain_graph) works."""

    @staticmethod
    def forward(ctx, ybar, coef, params, opts, bounds):
        q = dataclasses.replace(params, dp=float(coef[0]), dm=float(coef[1]), ep=float(coef[2]), em=float(coef[3]))
        prob = Problem(q)
        r = prob.admm_solve(opts, ybar.contiguous().view(-1), **bounds)
        state_box = bounds.get("ya") is not None or bounds.get("yb") is not None
        wy = prob.iterates(("wy",), device=ybar.device)["wy"] if state_box else None
        ctx.prob = prob
        ctx.wy = wy
        ctx.save_for_backward(r["y"], ybar)
        return torch.tensor(r["stats"]["objective"], dtype=torch.float64, device=ybar.device)

    @staticmethod
    def backward(ctx, gout):
        y, ybar = ctx.saved_tensors
        dJ, dcoef, _ = ctx.prob.admm_grad(y, ybar.contiguous().view(-1), wy=ctx.wy)
        return (gout * dJ.view_as(ybar), gout.cpu() * dcoef, None, None, None)


def solve_objective(ybar: torch.Tensor, coef: torch.Tensor, params, opts: AdmmOptions, bounds: dict):
    """Differentiable optimal value (see FdeAdmmFn)."""
    return FdeAdmmFn.apply(ybar, coef, params, opts, bounds)
