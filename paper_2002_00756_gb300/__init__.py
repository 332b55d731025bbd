"""Python binding of libmgsolve.so, the GB300 column multigrid solver (C ABI in include/mgsolve.h).

Argument marshalling only: every step of the solve runs in the library's CUDA kernels.
Vectors are torch CUDA tensors of dtype float64 (contiguous); host inputs (background
factors, level heights, mixed-system weights) are numpy arrays.  Calls are issued on the
current torch CUDA stream unless a stream is given.

The library must have been built (``paper_2002_00756_gb300.build.build()`` or
``__graft_entry__.build()``); there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from .build import LIB as _LIB_PATH

MG_OK, MG_ERR_ARG, MG_ERR_CUDA, MG_ERR_NOMEM = 0, -1, -2, -3
MG_ERR_NOT_CONVERGED, MG_ERR_BREAKDOWN, MG_ERR_TIMEOUT, MG_ERR_UNSUPPORTED = -4, -5, -6, -7
MG_FP64, MG_FP32, MG_FP32_BF16COEF, MG_FP32_P64 = 0, 1, 2, 3
PRECISIONS = {"fp64": MG_FP64, "fp32": MG_FP32, "fp32_bf16": MG_FP32_BF16COEF, "fp32_p64": MG_FP32_P64}


class MGError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        extra = f" [{load().mg_last_cuda_error().decode()}]" if status == MG_ERR_CUDA else ""
        super().__init__(f"{what}: {status_string(status)} ({status}){extra}")


class _Mesh(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nlev", ctypes.c_int32), ("radius", ctypes.c_double),
                ("cs_dt", ctypes.c_double), ("z_interfaces", ctypes.POINTER(ctypes.c_double))]


class _Params(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("omega", ctypes.c_double), ("n_pre", ctypes.c_int32),
                ("n_post", ctypes.c_int32), ("n_coarse", ctypes.c_int32),
                ("vcycle_precision", ctypes.c_int32), ("gcr_restart", ctypes.c_int32),
                ("max_iter", ctypes.c_int32)]


class _Mixed(ctypes.Structure):
    _fields_ = [("beta_up", ctypes.POINTER(ctypes.c_double)), ("beta_dn", ctypes.POINTER(ctypes.c_double)),
                ("eps", ctypes.c_double), ("consistent", ctypes.c_int32), ("coriolis_f0", ctypes.c_double)]


class _PSolver(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("eps", ctypes.c_double), ("omega", ctypes.c_double),
                ("sweeps", ctypes.c_int32), ("max_iter", ctypes.c_int32)]


# pressure solvers K_H(A_H, P_H, eps_H) of the Schur-complement step (Table 1 of the paper)
PRESSURE_SOLVERS = {"mg": 0, "jacobi": 1, "bicgstab_jacobi": 2, "bicgstab_mg": 3}


class _KRec(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("level", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("bytes", ctypes.c_double), ("ms", ctypes.c_double)]


KERNEL_KINDS = ("sweep", "restrict", "prolong", "apply", "convert", "dot", "gcr_dots", "gcr_orth",
                "gcr_update", "mixed")


class _Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("rel_res", ctypes.c_double), ("ms", ctypes.c_double)]


_lib = None

_VP, _DP, _I32, _D = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
_SIGS = {
    "mg_setup": [ctypes.POINTER(_Mesh), ctypes.POINTER(_Params), ctypes.POINTER(ctypes.c_double),
                 ctypes.POINTER(_Mixed), ctypes.POINTER(ctypes.c_void_p)],
    "mg_setup_coeffs": [ctypes.POINTER(_Mesh), ctypes.POINTER(_Params), ctypes.POINTER(ctypes.c_double),
                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_void_p)],
    "mg_set_coefficients": [_VP, _DP, _VP],
    "mg_setup_9pt": [ctypes.POINTER(_Mesh), ctypes.POINTER(_Params), ctypes.POINTER(ctypes.c_double), _D,
                     ctypes.POINTER(ctypes.c_void_p)],
    "mg_set_pressure_solver": [_VP, ctypes.POINTER(_PSolver)],
    "helmholtz_solve": [_VP, _DP, _DP, ctypes.POINTER(ctypes.c_double), _VP],
    "mg_inner_stats": [_VP, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)],
    "mg_ensemble_create": [_VP, _I32, _VP, _VP, _D, ctypes.POINTER(ctypes.c_void_p)],
    "mg_ensemble_solve": [_VP, ctypes.POINTER(_Info), ctypes.POINTER(ctypes.c_int32), _VP],
    "mg_ensemble_destroy": [_VP],
    "mg_destroy": [_VP],
    "mg_sizes": [_VP, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
    "helmholtz_apply": [_VP, _DP, _DP, _VP],
    "vcycle": [_VP, _DP, _DP, _VP],
    "pressure_solve": [_VP, _DP, _DP, _D, ctypes.POINTER(_Info), _VP],
    "pressure_solve_adjoint": [_VP, _DP, _DP, _D, ctypes.POINTER(_Info), _VP],
    "helmholtz_coefficient_gradient": [_VP, _DP, _DP, _DP, _VP],
    "ensemble_pressure_solve": [_VP, _I32, _VP, _VP, _D, ctypes.POINTER(_Info), ctypes.POINTER(ctypes.c_int32),
                                _VP],
    "mixed_solve": [_VP, _DP, _DP, _DP, _DP, _D, ctypes.POINTER(_Info), _VP],
    "mg_level_apply": [_VP, _I32, _DP, _DP, _VP],
    "mg_smooth": [_VP, _I32, _DP, _DP, _DP, _I32, _VP],
    "mg_smooth_noalloc": [_VP, _I32, _DP, _DP, _DP, _I32, _VP],
    "mg_residual_restrict": [_VP, _I32, _DP, _DP, _DP, _VP],
    "mg_prolong_add": [_VP, _I32, _DP, _DP, _VP],
    "mixed_apply": [_VP, _DP, _DP, _DP, _DP, _VP],
    "mixed_apply_transpose": [_VP, _DP, _DP, _DP, _DP, _VP],
    "mixed_solve_adjoint": [_VP, _DP, _DP, _DP, _DP, _D, ctypes.POINTER(_Info), _VP],
    "mixed_coefficient_gradient": [_VP, _DP, _DP, _DP, _DP, _DP, _DP, _VP],
    "mg_autotune": [_VP, ctypes.POINTER(ctypes.c_int32), _VP],
    "schur_precond": [_VP, _DP, _DP, _DP, _DP, _VP],
    "mg_profile_start": [_VP, _I32, _I32, _I32],
    "mg_profile_stop": [_VP, ctypes.POINTER(_KRec), _I32, ctypes.POINTER(ctypes.c_int32)],
}


def library_path() -> str:
    return _LIB_PATH


def load() -> ctypes.CDLL:
    """Load libmgsolve.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"{_LIB_PATH} is missing: build it with paper_2002_00756_gb300.build.build()")
        lib = ctypes.CDLL(_LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = None if name in ("mg_destroy", "mg_ensemble_destroy") else ctypes.c_int
        lib.mg_status_string.argtypes = [ctypes.c_int]
        lib.mg_status_string.restype = ctypes.c_char_p
        lib.mg_last_cuda_error.argtypes = []
        lib.mg_last_cuda_error.restype = ctypes.c_char_p
        lib.mg_inject_alloc_failure.argtypes = [ctypes.c_int64]
        lib.mg_inject_alloc_failure.restype = ctypes.c_int64
        lib.mg_live_allocations.argtypes = []
        lib.mg_live_allocations.restype = ctypes.c_int64
        _lib = lib
    return _lib


def status_string(status: int) -> str:
    return load().mg_status_string(int(status)).decode()


mg_status_string = status_string


def _raw_ptr(t, n: int | None = None, name: str = "vector"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} elements, expected {n}")
    return ctypes.c_void_p(t.data_ptr())


def _ptr(h, t, n: int | None = None, name: str = "vector"):
    """Device pointer of a vector argument of a call on handle h: a contiguous float64 tensor on
    the GPU the handle was set up on."""
    p = _raw_ptr(t, n, name)
    if t.device.index != h.device:
        raise ValueError(f"{name} is on cuda:{t.device.index}, the handle on cuda:{h.device}")
    return p


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _host(a, n: int, name: str):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).ravel())
    if a.size != n:
        raise ValueError(f"{name} has {a.size} values, expected {n}")
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class SolveInfo:
    status: int
    iters: int
    rel_res: float
    ms: float

    @property
    def converged(self) -> bool:
        return self.status == MG_OK


class Handle:
    """An mg_setup handle (owns the multigrid hierarchy and workspace on one GPU)."""

    def __init__(self, ptr: int, n: int, nlev: int, levels: int, ncol: int, ncell: int, nu: int, device: int = 0):
        self._ptr = ctypes.c_void_p(ptr)
        self.device = device
        self.n, self.nlev, self.levels = n, nlev, levels
        self.ncol, self.ncell, self.nu = ncol, ncell, nu

    def level_cells(self, level: int) -> int:
        return self.nlev * 6 * (self.n >> level) ** 2

    @property
    def ptr(self):
        if not self._ptr:
            raise ValueError("handle was destroyed")
        return self._ptr

    def destroy(self):
        if self._ptr:
            load().mg_destroy(self._ptr)
            self._ptr = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def _check(st: int, what: str):
    if st != MG_OK:
        raise MGError(st, what)


def mg_setup(n: int, nlev: int, z_interfaces, g, *, radius: float = 6371.0e3, cs_dt: float = 340.0 * 600.0,
             levels: int = 4, omega: float = 0.8, n_pre: int = 2, n_post: int = 2, n_coarse: int = 4,
             precision: str | int = "fp64", gcr_restart: int = 5, max_iter: int = 200,
             beta_up=None, beta_dn=None, eps: float = 0.0, consistent_mass: bool = False,
             coriolis_f0: float = 0.0, coeffs=None, gamma2: float = 0.0) -> Handle:
    """Build the hierarchy on the current CUDA device (see mg_setup in mgsolve.h).  With
    ``coeffs`` (host array of 6 N couplings a[s, k, c], s = E, W, N, S, up, down) the finest
    operator is the caller's and g only shapes the coarse levels (mg_setup_coeffs).  With
    ``gamma2`` > 0 the operator is the 9-cell stencil (mg_setup_9pt)."""
    import torch
    device = torch.cuda.current_device()   # (also makes sure the device context exists)
    lib = load()
    ncol = 6 * n * n
    z, zp = _host(z_interfaces, nlev + 1, "z_interfaces")
    gg, gp = _host(g, nlev * ncol, "g")
    mesh = _Mesh(n, nlev, radius, cs_dt, zp)
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    prm = _Params(levels, omega, n_pre, n_post, n_coarse, prec, gcr_restart, max_iter)
    mixed = None
    keep = [z, gg]
    if beta_up is not None:
        bu, bup = _host(beta_up, (nlev + 1) * ncol, "beta_up")
        bd, bdp = _host(beta_dn, (nlev + 1) * ncol, "beta_dn")
        keep += [bu, bd]
        mixed = _Mixed(bup, bdp, eps, int(bool(consistent_mass)), coriolis_f0)
    out = ctypes.c_void_p()
    if gamma2 > 0.0:
        if mixed is not None or coeffs is not None:
            raise ValueError("the 9-cell stencil is a pressure-system handle built from g")
        _check(lib.mg_setup_9pt(ctypes.byref(mesh), ctypes.byref(prm), gp, gamma2, ctypes.byref(out)), "mg_setup_9pt")
    elif coeffs is not None:
        if mixed is not None:
            raise ValueError("caller-supplied coefficients define a pressure-only handle (no mixed data)")
        cc, cp = _host(coeffs, 6 * nlev * ncol, "coeffs")
        keep.append(cc)
        st = lib.mg_setup_coeffs(ctypes.byref(mesh), ctypes.byref(prm), cp, gp, ctypes.byref(out))
        _check(st, "mg_setup_coeffs")
    else:
        st = lib.mg_setup(ctypes.byref(mesh), ctypes.byref(prm), gp,
                          ctypes.byref(mixed) if mixed is not None else None, ctypes.byref(out))
        _check(st, "mg_setup")
    nc, nn, nu = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib.mg_sizes(out, ctypes.byref(nc), ctypes.byref(nn), ctypes.byref(nu)), "mg_sizes")
    del keep
    return Handle(out.value, n, nlev, levels, nc.value, nn.value, nu.value, device)


def mg_set_coefficients(h: Handle, coeffs, stream=None):
    """Replace the finest-level operator by the couplings ``coeffs`` (float64 CUDA tensor of
    6 N values, the layout of helmholtz_coefficient_gradient); see mg_set_coefficients."""
    _check(load().mg_set_coefficients(h.ptr, _ptr(h, coeffs, 6 * h.ncell, "coeffs"), _stream(stream)),
           "mg_set_coefficients")


def mg_setup_config(cfg, inp: dict, precision: str | int = "fp64", levels: int | None = None,
                    mixed: bool | None = None, max_iter: int = 200, **kw) -> Handle:
    """mg_setup for a synthetic workload (a ``synthetic.Config`` and its input arrays)."""
    mixed = cfg.mixed if mixed is None else mixed
    extra = {}
    if mixed:
        # Coriolis factor tau_u dt 2 Omega of Eq. M2muCdef, tau_u = 1/2 (Sec. 3.3)
        extra = dict(beta_up=inp["beta_up"], beta_dn=inp["beta_dn"], eps=cfg.eps,
                     consistent_mass=cfg.consistent_mass, coriolis_f0=0.5 * cfg.dt * 2.0 * cfg.rotation)
    if getattr(cfg, "gamma2", 0.0) > 0.0 and "gamma2" not in kw:
        kw["gamma2"] = cfg.gamma2
    return mg_setup(cfg.n, cfg.nlev, inp["z_if"], inp["g"], radius=cfg.radius, cs_dt=cfg.cs * cfg.dt,
                    levels=levels or cfg.levels, omega=cfg.omega, n_pre=cfg.n_pre, n_post=cfg.n_post,
                    n_coarse=cfg.n_coarse, precision=precision, gcr_restart=cfg.gcr_restart,
                    max_iter=max_iter, **extra, **kw)


def mg_destroy(h: Handle):
    h.destroy()


def helmholtz_apply(h: Handle, x, y, stream=None):
    _check(load().helmholtz_apply(h.ptr, _ptr(h, x, h.ncell, "x"), _ptr(h, y, h.ncell, "y"), _stream(stream)),
           "helmholtz_apply")


def vcycle(h: Handle, b, x, stream=None):
    _check(load().vcycle(h.ptr, _ptr(h, b, h.ncell, "b"), _ptr(h, x, h.ncell, "x"), _stream(stream)), "vcycle")


def _solve_status(st: int, info: _Info, what: str) -> SolveInfo:
    if st not in (MG_OK, MG_ERR_NOT_CONVERGED, MG_ERR_BREAKDOWN):
        raise MGError(st, what)
    return SolveInfo(st, info.iters, info.rel_res, info.ms)


def pressure_solve(h: Handle, b, x, tol: float = 1e-8, stream=None) -> SolveInfo:
    info = _Info()
    st = load().pressure_solve(h.ptr, _ptr(h, b, h.ncell, "b"), _ptr(h, x, h.ncell, "x"), tol, ctypes.byref(info),
                               _stream(stream))
    return _solve_status(st, info, "pressure_solve")


def pressure_solve_adjoint(h: Handle, g, lam, tol: float = 1e-8, stream=None) -> SolveInfo:
    """lam = H^-T g (see pressure_solve_adjoint in mgsolve.h)."""
    info = _Info()
    st = load().pressure_solve_adjoint(h.ptr, _ptr(h, g, h.ncell, "g"), _ptr(h, lam, h.ncell, "lambda"), tol,
                                       ctypes.byref(info), _stream(stream))
    return _solve_status(st, info, "pressure_solve_adjoint")


def helmholtz_coefficient_gradient(h: Handle, lam, x, grad, stream=None):
    """grad (6 N, E/W/N/S/up/down blocks) = dL/da = -lam_i (x_i - x_j), see mgsolve.h."""
    _check(load().helmholtz_coefficient_gradient(h.ptr, _ptr(h, lam, h.ncell, "lambda"), _ptr(h, x, h.ncell, "x"),
                                                 _ptr(h, grad, 6 * h.ncell, "grad"), _stream(stream)),
           "helmholtz_coefficient_gradient")


def _pressure_solve_function():
    import torch

    class PressureSolve(torch.autograd.Function):
        """x = H(a)^-1 b with dL/db = lam = H^-T dL/dx and, when the couplings a are an input,
        dL/da = -lam_i (x_i - x_j) (helmholtz_coefficient_gradient); every step in the library."""

        @staticmethod
        def forward(ctx, b, coeffs, h, tol):
            if coeffs is not None:
                mg_set_coefficients(h, coeffs.detach().contiguous())
            x = torch.zeros_like(b)
            info = pressure_solve(h, b.contiguous(), x, tol=tol)
            if not info.converged:
                raise MGError(info.status, "pressure_solve")
            ctx.h, ctx.tol = h, tol
            if coeffs is not None:
                ctx.save_for_backward(x, coeffs)
            ctx.has_coeffs = coeffs is not None
            return x

        @staticmethod
        def backward(ctx, gx):
            if ctx.has_coeffs:
                x, coeffs = ctx.saved_tensors
                # the handle holds one operator: the one this forward pass solved with
                mg_set_coefficients(ctx.h, coeffs.detach().contiguous())
            lam = torch.zeros_like(gx)
            info = pressure_solve_adjoint(ctx.h, gx.contiguous(), lam, tol=ctx.tol)
            if not info.converged:
                raise MGError(info.status, "pressure_solve_adjoint")
            gcoef = None
            if ctx.has_coeffs and ctx.needs_input_grad[1]:
                gcoef = torch.empty(6 * ctx.h.ncell, dtype=lam.dtype, device=lam.device)
                helmholtz_coefficient_gradient(ctx.h, lam, x, gcoef)
            return lam, gcoef, None, None

    return PressureSolve


def solve(h: Handle, b, tol: float = 1e-8, coeffs=None):
    """Differentiable pressure solve: x = H^-1 b as a torch operation (float64 CUDA tensor b);
    its backward pass is the adjoint solve.  With ``coeffs`` (6 N couplings, float64 CUDA
    tensor) the finest operator is set to them first and the backward pass also gives dL/dcoeffs;
    they must describe a flux-symmetric operator (see mg_setup_coeffs)."""
    global _PS
    if _PS is None:
        _PS = _pressure_solve_function()
    return _PS.apply(b, coeffs, h, tol)


_PS = None


def ensemble_pressure_solve(handles, bs, xs, tol: float = 1e-8, stream=None) -> list[SolveInfo]:
    """Independent pressure solves, one per handle, with interleaved iterations (see
    ensemble_pressure_solve in mgsolve.h); returns each member's SolveInfo."""
    n = len(handles)
    if len(bs) != n or len(xs) != n:
        raise ValueError("one b and one x per handle")
    hs = (ctypes.c_void_p * n)(*[h.ptr for h in handles])
    bp = (ctypes.c_void_p * n)(*[_ptr(h, b, h.ncell, "b").value for b, h in zip(bs, handles)])
    xp = (ctypes.c_void_p * n)(*[_ptr(h, x, h.ncell, "x").value for x, h in zip(xs, handles)])
    infos = (_Info * max(n, 1))()
    sts = (ctypes.c_int32 * max(n, 1))()
    st = load().ensemble_pressure_solve(hs, n, bp, xp, tol, infos, sts, _stream(stream))
    if st not in (MG_OK, MG_ERR_NOT_CONVERGED, MG_ERR_BREAKDOWN):
        raise MGError(st, "ensemble_pressure_solve")
    return [SolveInfo(sts[i], infos[i].iters, infos[i].rel_res, infos[i].ms) for i in range(n)]


class Ensemble:
    """An mg_ensemble: every member's pressure solve recorded into one CUDA graph (see
    mg_ensemble_create in mgsolve.h).  The b and x tensors are bound at creation; solve() runs
    all members with one graph launch and returns each member's SolveInfo."""

    def __init__(self, handles, bs, xs, tol: float = 1e-8):
        n = len(handles)
        if n < 1 or len(bs) != n or len(xs) != n:
            raise ValueError("one b and one x per handle, at least one member")
        self.handles, self.bs, self.xs = list(handles), list(bs), list(xs)   # keep them alive
        hs = (ctypes.c_void_p * n)(*[h.ptr for h in handles])
        bp = (ctypes.c_void_p * n)(*[_ptr(h, b, h.ncell, "b").value for b, h in zip(bs, handles)])
        xp = (ctypes.c_void_p * n)(*[_ptr(h, x, h.ncell, "x").value for x, h in zip(xs, handles)])
        out = ctypes.c_void_p()
        _check(load().mg_ensemble_create(hs, n, bp, xp, tol, ctypes.byref(out)), "mg_ensemble_create")
        self._ptr = out

    def solve(self, stream=None) -> list[SolveInfo]:
        n = len(self.handles)
        infos = (_Info * n)()
        sts = (ctypes.c_int32 * n)()
        st = load().mg_ensemble_solve(self._ptr, infos, sts, _stream(stream))
        if st not in (MG_OK, MG_ERR_NOT_CONVERGED, MG_ERR_BREAKDOWN):
            raise MGError(st, "mg_ensemble_solve")
        return [SolveInfo(sts[i], infos[i].iters, infos[i].rel_res, infos[i].ms) for i in range(n)]

    def destroy(self):
        if self._ptr:
            load().mg_ensemble_destroy(self._ptr)
            self._ptr = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def mixed_solve(h: Handle, rhs_u, rhs_p, u, p, tol: float = 1e-8, stream=None) -> SolveInfo:
    info = _Info()
    st = load().mixed_solve(h.ptr, _ptr(h, rhs_u, h.nu, "rhs_u"), _ptr(h, rhs_p, h.ncell, "rhs_p"),
                            _ptr(h, u, h.nu, "u"), _ptr(h, p, h.ncell, "p"), tol, ctypes.byref(info), _stream(stream))
    return _solve_status(st, info, "mixed_solve")


def mixed_solve_adjoint(h: Handle, g_u, g_p, lam_u, lam_p, tol: float = 1e-8, stream=None) -> SolveInfo:
    """[lam_u; lam_p] = A^-T [g_u; g_p] (see mixed_solve_adjoint in mgsolve.h)."""
    info = _Info()
    st = load().mixed_solve_adjoint(h.ptr, _ptr(h, g_u, h.nu, "g_u"), _ptr(h, g_p, h.ncell, "g_p"),
                                    _ptr(h, lam_u, h.nu, "lam_u"), _ptr(h, lam_p, h.ncell, "lam_p"), tol,
                                    ctypes.byref(info), _stream(stream))
    return _solve_status(st, info, "mixed_solve_adjoint")


def mixed_coefficient_gradient(h: Handle, lam_u, u, p, grad_g, grad_beta_up, grad_beta_dn, stream=None):
    """dL/dg (N), dL/dbeta_up, dL/dbeta_dn ((nlev+1) ncol) from lam_u = (A^-T dL/d(u, p))_u and
    the solution (u, p); see mixed_coefficient_gradient in mgsolve.h."""
    nv = (h.nlev + 1) * h.ncol
    _check(load().mixed_coefficient_gradient(h.ptr, _ptr(h, lam_u, h.nu, "lam_u"), _ptr(h, u, h.nu, "u"),
                                             _ptr(h, p, h.ncell, "p"), _ptr(h, grad_g, h.ncell, "grad_g"),
                                             _ptr(h, grad_beta_up, nv, "grad_beta_up"),
                                             _ptr(h, grad_beta_dn, nv, "grad_beta_dn"), _stream(stream)),
           "mixed_coefficient_gradient")


def mg_autotune(h: Handle, stream=None) -> list[tuple[int, int, int]]:
    """Pick the fastest sweep and restriction launch shapes per level (see mg_autotune in
    mgsolve.h); returns (sweep threads per block, restriction levels per thread, copy ring)
    per level."""
    ch = (ctypes.c_int32 * (3 * h.levels))()
    _check(load().mg_autotune(h.ptr, ch, _stream(stream)), "mg_autotune")
    return [(ch[3 * l], ch[3 * l + 1], ch[3 * l + 2]) for l in range(h.levels)]


def mixed_apply_transpose(h: Handle, u, p, yu, yp, stream=None):
    _check(load().mixed_apply_transpose(h.ptr, _ptr(h, u, h.nu, "u"), _ptr(h, p, h.ncell, "p"), _ptr(h, yu, h.nu, "yu"),
                                        _ptr(h, yp, h.ncell, "yp"), _stream(stream)), "mixed_apply_transpose")


def _mixed_solve_function():
    import torch

    class MixedSolve(torch.autograd.Function):
        """[u; p] = A^-1 [rhs_u; rhs_p] with dL/drhs = A^-T dL/d[u; p] (both solves in the library)."""

        @staticmethod
        def forward(ctx, rhs_u, rhs_p, h, tol):
            u, p = torch.zeros_like(rhs_u), torch.zeros_like(rhs_p)
            info = mixed_solve(h, rhs_u.contiguous(), rhs_p.contiguous(), u, p, tol=tol)
            if not info.converged:
                raise MGError(info.status, "mixed_solve")
            ctx.h, ctx.tol = h, tol
            return u, p

        @staticmethod
        def backward(ctx, gu, gp):
            # (autograd materialises an unused output's gradient as zeros)
            gu, gp = gu.contiguous(), gp.contiguous()
            lu, lp = torch.zeros_like(gu), torch.zeros_like(gp)
            info = mixed_solve_adjoint(ctx.h, gu, gp, lu, lp, tol=ctx.tol)
            if not info.converged:
                raise MGError(info.status, "mixed_solve_adjoint")
            return lu, lp, None, None

    return MixedSolve


def solve_mixed(h: Handle, rhs_u, rhs_p, tol: float = 1e-8):
    """Differentiable mixed solve: (u, p) = A^-1 (rhs_u, rhs_p) as a torch operation (float64
    CUDA tensors); its backward pass is mixed_solve_adjoint."""
    global _MS
    if _MS is None:
        _MS = _mixed_solve_function()
    return _MS.apply(rhs_u, rhs_p, h, tol)


_MS = None


def mg_set_pressure_solver(h: Handle, kind: str = "mg", eps: float = 1e-2, omega: float = 0.8, sweeps: int = 10,
                           max_iter: int = 200):
    """Pressure solver of the Schur-complement step and of helmholtz_solve: "mg" (one V-cycle),
    "jacobi" (line relaxation, `sweeps` block-Jacobi sweeps with `omega`), "bicgstab_jacobi"
    (BiCGStab to eps preconditioned by the block-Jacobi sweeps) or "bicgstab_mg" (BiCGStab to eps
    preconditioned by one V-cycle); see mg_set_pressure_solver in mgsolve.h."""
    ps = _PSolver(PRESSURE_SOLVERS[kind], eps, omega, sweeps, max_iter)
    _check(load().mg_set_pressure_solver(h.ptr, ctypes.byref(ps)), "mg_set_pressure_solver")


@dataclass
class InnerInfo:
    status: int
    iterations: float

    @property
    def converged(self) -> bool:
        return self.status == MG_OK


def helmholtz_solve(h: Handle, b, x, stream=None) -> InnerInfo:
    """x = K_H(A_H, P_H, eps_H) b with the handle's pressure solver, from x = 0."""
    it = ctypes.c_double()
    st = load().helmholtz_solve(h.ptr, _ptr(h, b, h.ncell, "b"), _ptr(h, x, h.ncell, "x"), ctypes.byref(it),
                                _stream(stream))
    if st not in (MG_OK, MG_ERR_NOT_CONVERGED, MG_ERR_BREAKDOWN):
        raise MGError(st, "helmholtz_solve")
    return InnerInfo(st, it.value)


def mg_inner_stats(h: Handle) -> tuple[int, float]:
    """(BiCGStab pressure solves, their iterations) since the last call; resets both."""
    n, it = ctypes.c_int64(), ctypes.c_double()
    _check(load().mg_inner_stats(h.ptr, ctypes.byref(n), ctypes.byref(it)), "mg_inner_stats")
    return n.value, it.value


def mg_level_apply(h: Handle, level: int, x, y, stream=None):
    n = h.level_cells(level)
    _check(load().mg_level_apply(h.ptr, level, _ptr(h, x, n, "x"), _ptr(h, y, n, "y"), _stream(stream)), "mg_level_apply")


def mg_smooth(h: Handle, level: int, b, x_in, x_out, sweeps: int, stream=None):
    n = h.level_cells(level)
    xin = None if x_in is None else _ptr(h, x_in, n, "x_in")
    _check(load().mg_smooth(h.ptr, level, _ptr(h, b, n, "b"), xin, _ptr(h, x_out, n, "x_out"), sweeps, _stream(stream)),
           "mg_smooth")


MG_NOALLOC_MAX_CELLS = 1 << 21


def mg_smooth_noalloc(h: Handle, level: int, b, x_in, x_out, sweeps: int, stream=None):
    """mg_smooth for callers that cannot allocate device memory at this point (real-time
    loops, frameworks whose memory pool owns the device, fixed memory budgets): the
    library keeps the intermediate iterate in a fixed 16 MiB device array, so this call
    allocates nothing.  Levels above MG_NOALLOC_MAX_CELLS cells are rejected; overlapping
    calls race on the shared array.  The first call on a device must precede any capture."""
    n = h.level_cells(level)
    xin = None if x_in is None else _ptr(h, x_in, n, "x_in")
    _check(load().mg_smooth_noalloc(h.ptr, level, _ptr(h, b, n, "b"), xin, _ptr(h, x_out, n, "x_out"), sweeps,
                                    _stream(stream)), "mg_smooth_noalloc")


def mg_residual_restrict(h: Handle, level: int, b, x, bc, stream=None):
    n, nc = h.level_cells(level), h.level_cells(level + 1)
    _check(load().mg_residual_restrict(h.ptr, level, _ptr(h, b, n, "b"), _ptr(h, x, n, "x"), _ptr(h, bc, nc, "bc"),
                                       _stream(stream)), "mg_residual_restrict")


def mg_prolong_add(h: Handle, level: int, xc, x, stream=None):
    n, nc = h.level_cells(level), h.level_cells(level + 1)
    _check(load().mg_prolong_add(h.ptr, level, _ptr(h, xc, nc, "xc"), _ptr(h, x, n, "x"), _stream(stream)),
           "mg_prolong_add")


def mixed_apply(h: Handle, u, p, yu, yp, stream=None):
    _check(load().mixed_apply(h.ptr, _ptr(h, u, h.nu, "u"), _ptr(h, p, h.ncell, "p"), _ptr(h, yu, h.nu, "yu"),
                              _ptr(h, yp, h.ncell, "yp"), _stream(stream)), "mixed_apply")


def schur_precond(h: Handle, ru, rp, u, p, stream=None):
    _check(load().schur_precond(h.ptr, _ptr(h, ru, h.nu, "ru"), _ptr(h, rp, h.ncell, "rp"), _ptr(h, u, h.nu, "u"),
                                _ptr(h, p, h.ncell, "p"), _stream(stream)), "schur_precond")


def mg_profile_start(h: Handle, capacity: int = 65536, kind: str | None = None, level: int | None = None):
    """Record the kernel launches of the following calls with CUDA events (all of them, or
    only those of one kind, e.g. "sweep", and / or one multigrid level)."""
    k = -1 if kind is None else KERNEL_KINDS.index(kind)
    _check(load().mg_profile_start(h.ptr, capacity, k, -1 if level is None else level), "mg_profile_start")
    h._prof_cap = capacity


def mg_profile_stop(h: Handle) -> list[dict]:
    """Stop recording; returns one dict per timed launch (kind, level, bytes, ms)."""
    cap = getattr(h, "_prof_cap", 65536)
    recs = (_KRec * cap)()
    cnt = ctypes.c_int32()
    _check(load().mg_profile_stop(h.ptr, recs, cap, ctypes.byref(cnt)), "mg_profile_stop")
    return [dict(kind=KERNEL_KINDS[r.kind], level=r.level, variant=r.variant, bytes=r.bytes, ms=r.ms)
            for r in recs[:min(cnt.value, cap)]]
