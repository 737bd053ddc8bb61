"""Python binding of libgsis (include/gsis.h): argument marshalling only.

Device arrays are torch tensors (float64, contiguous, on the current CUDA
device); host arrays (mesh spacings, quadrature) are numpy arrays.  Every
computation happens in the CUDA library; if it is not built or cannot be
loaded, every call raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

GSIS_OK = 0
GSIS_ERR_ARG = -1
GSIS_ERR_CUDA = -2
GSIS_ERR_MAXITER = -3
GSIS_ERR_DIVERGED = -4
GSIS_ERR_STALLED = -5
GSIS_ERR_DEVICE_TIMEOUT = -6
GSIS_ERR_WORKSPACE = -7

SCHEME_SI = 0
SCHEME_GSIS = 1
FP64 = 0
FP32_SWEEP = 1

_P = ctypes.POINTER(ctypes.c_double)


class GsisError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"gsis status {status}: {message}")
        self.status = status


class Mesh(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("dx", _P), ("dy", _P)]


class Quadrature(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("mu", _P), ("eta", _P), ("w", _P)]


KERNEL_CLASSES = ("setup", "sweep", "moments", "hot_rhs", "synth", "update")


class KernelStats(ctypes.Structure):
    _fields_ = [("kernels", ctypes.c_longlong), ("groups", ctypes.c_longlong),
                ("timed", ctypes.c_longlong), ("total_ms", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("synth_inner_iters", ctypes.c_longlong),
                ("err", ctypes.c_double), ("synth_relres", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [
        ("scheme", ctypes.c_int), ("precision", ctypes.c_int), ("tol", ctypes.c_double),
        ("max_iter", ctypes.c_int), ("fixed_iters", ctypes.c_int), ("synth_rtol", ctypes.c_double),
        ("synth_max_iter", ctypes.c_int), ("cfl_p", ctypes.c_double), ("beta", ctypes.c_double),
        ("check_every", ctypes.c_int), ("stall_window", ctypes.c_int), ("wait_limit_s", ctypes.c_double),
        ("spatial_order", ctypes.c_int), ("limiter", ctypes.c_int),
    ]


class Problem(ctypes.Structure):
    _fields_ = [
        ("mesh", Mesh), ("quad", Quadrature),
        ("sigma_a", ctypes.c_void_p), ("sigma_s", ctypes.c_void_p), ("q", ctypes.c_void_p),
        ("inflow", ctypes.c_void_p), ("rho", ctypes.c_void_p), ("F", ctypes.c_void_p),
        ("iters", ctypes.c_int), ("err", ctypes.c_double), ("status", ctypes.c_int),
    ]


class BatchTuning(ctypes.Structure):
    _fields_ = [("sweep_order", ctypes.c_int), ("sweep_dynamic", ctypes.c_int),
                ("synth_cells_per_cta", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


ORDER_PROBLEM, ORDER_BAND, ORDER_LONGEST, ORDER_BAND_LONGEST = 0, 1, 2, 3

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load the in-tree libgsis.so (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"libgsis is not built ({_build.LIB}); run __graft_entry__.build()")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    vp, sz = ctypes.c_void_p, ctypes.c_size_t
    Mp, Qp, Op = ctypes.POINTER(Mesh), ctypes.POINTER(Quadrature), ctypes.POINTER(Options)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.gsis_default_options.argtypes = [Op]
    lib.gsis_default_options.restype = None
    lib.gsis_quadrature_level_symmetric.argtypes = [ctypes.c_int, _P, _P, _P, ip]
    lib.gsis_workspace_bytes.argtypes = [Mp, Qp, Op, ctypes.POINTER(sz)]
    lib.gsis_solve.argtypes = [Mp, Qp, Op, vp, vp, vp, vp, vp, vp, vp, _P, ip, _P, vp, sz, vp]
    lib.gsis_transport_sweep.argtypes = [Mp, Qp, Op, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    lib.gsis_synthetic_step.argtypes = [Mp, Op, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, ip, vp, sz, vp]
    lib.gsis_transport_sweep_static.argtypes = [Mp, Qp, Op, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.gsis_transport_sweep_static.restype = ctypes.c_int
    lib.gsis_adjoint_workspace_bytes.argtypes = [Mp, Qp, Op, ctypes.POINTER(sz)]
    lib.gsis_adjoint_workspace_bytes.restype = ctypes.c_int
    lib.gsis_adjoint.argtypes = [Mp, Qp, Op, vp, vp, vp, vp, vp, vp, vp, vp, ip, _P, vp, sz, vp]
    lib.gsis_adjoint.restype = ctypes.c_int
    lib.gsis_last_solve_info.argtypes = [ctypes.POINTER(SolveInfo)]
    lib.gsis_last_solve_info.restype = ctypes.c_int
    lib.gsis_profile_enable.argtypes = [ctypes.c_int]
    lib.gsis_profile_enable.restype = ctypes.c_int
    lib.gsis_profile_read.argtypes = [ctypes.POINTER(KernelStats), ctypes.c_int]
    lib.gsis_profile_read.restype = ctypes.c_int
    lib.gsis_status_string.argtypes = [ctypes.c_int]
    lib.gsis_status_string.restype = ctypes.c_char_p
    lib.gsis_last_error.argtypes = []
    lib.gsis_last_error.restype = ctypes.c_char_p
    Pp, Tp, dp = ctypes.POINTER(Problem), ctypes.POINTER(BatchTuning), ctypes.POINTER(ctypes.c_double)
    lib.gsis_default_batch_tuning.argtypes = [Tp]
    lib.gsis_default_batch_tuning.restype = None
    lib.gsis_batch_workspace_bytes.argtypes = [Pp, ctypes.c_int, Op, ctypes.POINTER(sz)]
    lib.gsis_batch_workspace_bytes.restype = ctypes.c_int
    lib.gsis_solve_batch.argtypes = [Pp, ctypes.c_int, Op, Tp, vp, sz, vp]
    lib.gsis_solve_batch.restype = ctypes.c_int
    lib.gsis_batch_autotune.argtypes = [Pp, ctypes.c_int, Op, ctypes.c_int, Tp, dp, dp, vp, sz, vp]
    lib.gsis_batch_autotune.restype = ctypes.c_int
    for name in ("gsis_quadrature_level_symmetric", "gsis_workspace_bytes", "gsis_solve",
                 "gsis_transport_sweep", "gsis_synthetic_step"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().gsis_status_string(status).decode()


def last_error() -> str:
    return load().gsis_last_error().decode()


def _raise(rc: int, hard=(GSIS_ERR_ARG, GSIS_ERR_CUDA, GSIS_ERR_WORKSPACE, GSIS_ERR_DEVICE_TIMEOUT)):
    if rc in hard:
        raise GsisError(rc, last_error() or status_string(rc))
    return rc


def profile_enable(enable: bool = True) -> None:
    """gsis_profile_enable: reset the per-class counters; time later launches."""
    _raise(load().gsis_profile_enable(1 if enable else 0))


def profile_read() -> dict:
    """gsis_profile_read: {class: dict(kernels, groups, timed, total_ms)}."""
    arr = (KernelStats * len(KERNEL_CLASSES))()
    _raise(load().gsis_profile_read(arr, len(KERNEL_CLASSES)))
    return {n: dict(kernels=a.kernels, groups=a.groups, timed=a.timed, total_ms=a.total_ms)
            for n, a in zip(KERNEL_CLASSES, arr)}


def default_options(**kw) -> Options:
    o = Options()
    load().gsis_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def quadrature_level_symmetric(order: int):
    lib = load()
    K = ctypes.c_int(0)
    _raise(lib.gsis_quadrature_level_symmetric(order, None, None, None, ctypes.byref(K)))
    mu, eta, w = (np.zeros(K.value) for _ in range(3))
    _raise(lib.gsis_quadrature_level_symmetric(order, _hp(mu), _hp(eta), _hp(w), ctypes.byref(K)))
    return mu, eta, w


def _hp(a: np.ndarray):
    return a.ctypes.data_as(_P)


def _host(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _dev(t, n=None, name="array"):
    """Device pointer of a float64 contiguous CUDA tensor (or None)."""
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if n is not None and t.numel() < n:
        raise ValueError(f"{name} has {t.numel()} elements, needs {n}")
    return ctypes.c_void_p(t.data_ptr())


class _Args:
    """Keeps the host arrays alive while the C structs point at them."""

    def __init__(self, dx, dy, mu=None, eta=None, w=None):
        self.dx, self.dy = _host(dx), _host(dy)
        self.mesh = Mesh(len(self.dx), len(self.dy), _hp(self.dx), _hp(self.dy))
        self.quad = None
        if mu is not None:
            self.mu, self.eta, self.w = _host(mu), _host(eta), _host(w)
            self.quad = Quadrature(len(self.mu), _hp(self.mu), _hp(self.eta), _hp(self.w))


def workspace_bytes(dx, dy, mu=None, eta=None, w=None, options: Options | None = None) -> int:
    a = _Args(dx, dy, mu, eta, w)
    o = options or default_options()
    n = ctypes.c_size_t(0)
    _raise(load().gsis_workspace_bytes(ctypes.byref(a.mesh), ctypes.byref(a.quad) if a.quad else None,
                                       ctypes.byref(o), ctypes.byref(n)))
    return int(n.value)


def _workspace(nbytes, workspace, device):
    import torch
    if workspace is None or workspace.numel() < nbytes:
        workspace = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device)
    return workspace


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def solve(dx, dy, mu, eta, w, sigma_a, sigma_s, q, inflow=None, options: Options | None = None,
          want_P=True, workspace=None, stream=None):
    """gsis_solve: returns dict(rho, F, P, iters, err, history, status, workspace)."""
    import torch
    a = _Args(dx, dy, mu, eta, w)
    o = options or default_options()
    N, K = a.mesh.nx * a.mesh.ny, a.quad.K
    dev = sigma_a.device
    rho = torch.empty(N, dtype=torch.float64, device=dev)
    F = torch.empty(2 * N, dtype=torch.float64, device=dev)
    P = torch.empty(3 * N, dtype=torch.float64, device=dev) if want_P else None
    nh = max(o.max_iter, o.fixed_iters, 1)
    hist = np.zeros(nh)
    iters, err = ctypes.c_int(0), ctypes.c_double(0.0)
    nbytes = workspace_bytes(a.dx, a.dy, a.mu, a.eta, a.w, o)
    workspace = _workspace(nbytes, workspace, dev)
    rc = load().gsis_solve(
        ctypes.byref(a.mesh), ctypes.byref(a.quad), ctypes.byref(o),
        _dev(sigma_a, N, "sigma_a"), _dev(sigma_s, N, "sigma_s"), _dev(q, N, "q"),
        _dev(inflow, 2 * (a.mesh.nx + a.mesh.ny) * K, "inflow"),
        _dev(rho), _dev(F), _dev(P), _hp(hist), ctypes.byref(iters), ctypes.byref(err),
        ctypes.c_void_p(workspace.data_ptr()), ctypes.c_size_t(workspace.numel()), _stream(stream))
    _raise(rc)
    info = SolveInfo()
    load().gsis_last_solve_info(ctypes.byref(info))
    return dict(rho=rho, F=F, P=P, iters=iters.value, err=err.value, history=hist[:iters.value],
                status=rc, workspace=workspace, synth_inner_iters=int(info.synth_inner_iters),
                synth_relres=info.synth_relres)


def transport_sweep(dx, dy, mu, eta, w, sigma_a, sigma_s, q, rho_in, inflow=None,
                    options: Options | None = None, want_P=True, workspace=None, stream=None):
    """gsis_transport_sweep: returns dict(rho, F, P, bflux)."""
    import torch
    a = _Args(dx, dy, mu, eta, w)
    o = options or default_options()
    N, K = a.mesh.nx * a.mesh.ny, a.quad.K
    dev = sigma_a.device
    rho = torch.empty(N, dtype=torch.float64, device=dev)
    F = torch.empty(2 * N, dtype=torch.float64, device=dev)
    P = torch.empty(3 * N, dtype=torch.float64, device=dev) if want_P else None
    fb = torch.empty(2 * (a.mesh.nx + a.mesh.ny), dtype=torch.float64, device=dev)
    nbytes = workspace_bytes(a.dx, a.dy, a.mu, a.eta, a.w, o)
    workspace = _workspace(nbytes, workspace, dev)
    rc = load().gsis_transport_sweep(
        ctypes.byref(a.mesh), ctypes.byref(a.quad), ctypes.byref(o),
        _dev(sigma_a, N, "sigma_a"), _dev(sigma_s, N, "sigma_s"), _dev(q, N, "q"),
        _dev(inflow, 2 * (a.mesh.nx + a.mesh.ny) * K, "inflow"), _dev(rho_in, N, "rho_in"),
        _dev(rho), _dev(F), _dev(P), _dev(fb), ctypes.c_void_p(workspace.data_ptr()),
        ctypes.c_size_t(workspace.numel()), _stream(stream))
    _raise(rc)
    return dict(rho=rho, F=F, P=P, bflux=fb, workspace=workspace)


def transport_sweep_static(dx, dy, mu, eta, w, sigma_a, sigma_s, q, rho_in, inflow=None,
                           options: Options | None = None, want_P=True, stream=None):
    """gsis_transport_sweep_static: the kinetic step with the library's static
    device scratch (no workspace, no device allocation by the library);
    returns dict(rho, F, P, bflux)."""
    import torch
    a = _Args(dx, dy, mu, eta, w)
    o = options or default_options()
    N, K = a.mesh.nx * a.mesh.ny, a.quad.K
    dev = sigma_a.device
    rho = torch.empty(N, dtype=torch.float64, device=dev)
    F = torch.empty(2 * N, dtype=torch.float64, device=dev)
    P = torch.empty(3 * N, dtype=torch.float64, device=dev) if want_P else None
    fb = torch.empty(2 * (a.mesh.nx + a.mesh.ny), dtype=torch.float64, device=dev)
    rc = load().gsis_transport_sweep_static(
        ctypes.byref(a.mesh), ctypes.byref(a.quad), ctypes.byref(o),
        _dev(sigma_a, N, "sigma_a"), _dev(sigma_s, N, "sigma_s"), _dev(q, N, "q"),
        _dev(inflow, 2 * (a.mesh.nx + a.mesh.ny) * K, "inflow"), _dev(rho_in, N, "rho_in"),
        _dev(rho), _dev(F), _dev(P), _dev(fb), _stream(stream))
    _raise(rc)
    return dict(rho=rho, F=F, P=P, bflux=fb)


def synthetic_step(dx, dy, sigma_a, sigma_s, q, rho_half, F_half, bflux, rho_guess=None,
                   options: Options | None = None, workspace=None, stream=None):
    """gsis_synthetic_step: returns dict(rho, hot, rhs, synth_iters)."""
    import torch
    a = _Args(dx, dy)
    o = options or default_options()
    N = a.mesh.nx * a.mesh.ny
    dev = sigma_a.device
    rho = torch.empty(N, dtype=torch.float64, device=dev)
    hot = torch.empty(2 * N, dtype=torch.float64, device=dev)
    rhs = torch.empty(N, dtype=torch.float64, device=dev)
    it = ctypes.c_int(0)
    nbytes = workspace_bytes(a.dx, a.dy, options=o)
    workspace = _workspace(nbytes, workspace, dev)
    rc = load().gsis_synthetic_step(
        ctypes.byref(a.mesh), ctypes.byref(o), _dev(sigma_a, N, "sigma_a"), _dev(sigma_s, N, "sigma_s"),
        _dev(q, N, "q"), _dev(rho_half, N, "rho_half"), _dev(F_half, 2 * N, "F_half"),
        _dev(bflux, 2 * (a.mesh.nx + a.mesh.ny), "bflux"), _dev(rho_guess, N, "rho_guess"),
        _dev(rho), _dev(hot), _dev(rhs), ctypes.byref(it), ctypes.c_void_p(workspace.data_ptr()),
        ctypes.c_size_t(workspace.numel()), _stream(stream))
    _raise(rc)
    return dict(rho=rho, hot=hot, rhs=rhs, synth_iters=it.value, workspace=workspace)


def adjoint_workspace_bytes(dx, dy, mu, eta, w, options: Options | None = None) -> int:
    a = _Args(dx, dy, mu, eta, w)
    o = options or default_options()
    n = ctypes.c_size_t(0)
    _raise(load().gsis_adjoint_workspace_bytes(ctypes.byref(a.mesh), ctypes.byref(a.quad), ctypes.byref(o),
                                               ctypes.byref(n)))
    return int(n.value)


def adjoint(dx, dy, mu, eta, w, sigma_a, sigma_s, q, rho_star, dJ_drho, inflow=None,
            options: Options | None = None, workspace=None, stream=None):
    """gsis_adjoint: gradient of J(rho*) with respect to sigma_a, sigma_s given
    dJ/drho; returns dict(grad_sigma_a, grad_sigma_s, iters, err, status, workspace)."""
    import torch
    a = _Args(dx, dy, mu, eta, w)
    o = options or default_options()
    N, K = a.mesh.nx * a.mesh.ny, a.quad.K
    dev = sigma_a.device
    gsa = torch.empty(N, dtype=torch.float64, device=dev)
    gss = torch.empty(N, dtype=torch.float64, device=dev)
    iters, err = ctypes.c_int(0), ctypes.c_double(0.0)
    nbytes = adjoint_workspace_bytes(a.dx, a.dy, a.mu, a.eta, a.w, o)
    workspace = _workspace(nbytes, workspace, dev)
    rc = load().gsis_adjoint(
        ctypes.byref(a.mesh), ctypes.byref(a.quad), ctypes.byref(o),
        _dev(sigma_a, N, "sigma_a"), _dev(sigma_s, N, "sigma_s"), _dev(q, N, "q"),
        _dev(inflow, 2 * (a.mesh.nx + a.mesh.ny) * K, "inflow"), _dev(rho_star, N, "rho_star"),
        _dev(dJ_drho, N, "dJ_drho"), _dev(gsa), _dev(gss), ctypes.byref(iters), ctypes.byref(err),
        ctypes.c_void_p(workspace.data_ptr()), ctypes.c_size_t(workspace.numel()), _stream(stream))
    _raise(rc)
    return dict(grad_sigma_a=gsa, grad_sigma_s=gss, iters=iters.value, err=err.value, status=rc,
                workspace=workspace)


def _autograd_function():
    import torch

    class GsisSolve(torch.autograd.Function):
        """rho* = GSIS solution as a differentiable function of (sigma_a, sigma_s):
        forward = gsis_solve, backward = gsis_adjoint with dJ/drho = grad_output."""

        @staticmethod
        def forward(ctx, sigma_a, sigma_s, q, host, inflow, options):
            dx, dy, mu, eta, w = host
            r = solve(dx, dy, mu, eta, w, sigma_a.detach().contiguous(), sigma_s.detach().contiguous(),
                      q.detach().contiguous(), inflow=inflow, options=options, want_P=False)
            rho = r["rho"]
            ctx.host, ctx.inflow, ctx.options = host, inflow, options
            ctx.save_for_backward(sigma_a, sigma_s, q, rho)
            return rho

        @staticmethod
        def backward(ctx, grad_rho):
            sigma_a, sigma_s, q, rho = ctx.saved_tensors
            dx, dy, mu, eta, w = ctx.host
            out = adjoint(dx, dy, mu, eta, w, sigma_a.detach().contiguous(), sigma_s.detach().contiguous(),
                          q.detach().contiguous(), rho, grad_rho.detach().to(torch.float64).contiguous(),
                          inflow=ctx.inflow, options=ctx.options)
            return out["grad_sigma_a"], out["grad_sigma_s"], None, None, None, None

    return GsisSolve


_GsisSolve = None


def solve_differentiable(dx, dy, mu, eta, w, sigma_a, sigma_s, q, inflow=None, options: Options | None = None):
    """rho* (device [N]) of gsis_solve, differentiable with respect to sigma_a and
    sigma_s through torch.autograd (the backward pass is gsis_adjoint)."""
    global _GsisSolve
    if _GsisSolve is None:
        _GsisSolve = _autograd_function()
    return _GsisSolve.apply(sigma_a, sigma_s, q, (dx, dy, mu, eta, w), inflow, options)


# ------------------------------------------------------------------ batches
def default_batch_tuning(**kw) -> BatchTuning:
    t = BatchTuning()
    load().gsis_default_batch_tuning(ctypes.byref(t))
    for k, v in kw.items():
        if not hasattr(t, k):
            raise KeyError(k)
        setattr(t, k, v)
    return t


class _Batch:
    """C records of a list of problems; each problem is a mapping with dx, dy,
    mu, eta, w (host arrays) and sigma_a, sigma_s, q, optional inflow
    (float64 CUDA tensors).  Keeps every host array alive."""

    def __init__(self, problems, with_outputs=True):
        import torch
        if not problems:
            raise ValueError("empty batch")
        self.args = [_Args(p["dx"], p["dy"], p["mu"], p["eta"], p["w"]) for p in problems]
        self.arr = (Problem * len(problems))()
        self.rho, self.F = [], []
        for i, (p, a) in enumerate(zip(problems, self.args)):
            N, K = a.mesh.nx * a.mesh.ny, a.quad.K
            r = self.arr[i]
            r.mesh, r.quad = a.mesh, a.quad
            r.sigma_a = _dev(p["sigma_a"], N, "sigma_a")
            r.sigma_s = _dev(p["sigma_s"], N, "sigma_s")
            r.q = _dev(p["q"], N, "q")
            r.inflow = _dev(p.get("inflow"), 2 * (a.mesh.nx + a.mesh.ny) * K, "inflow")
            dev = p["sigma_a"].device
            rho = torch.empty(N, dtype=torch.float64, device=dev) if with_outputs else None
            F = torch.empty(2 * N, dtype=torch.float64, device=dev) if with_outputs else None
            r.rho = _dev(rho)
            r.F = _dev(F)
            self.rho.append(rho)
            self.F.append(F)
        self.device = problems[0]["sigma_a"].device


def batch_workspace_bytes(problems, options: Options | None = None) -> int:
    b = _Batch(problems, with_outputs=False)
    o = options or default_options()
    n = ctypes.c_size_t(0)
    _raise(load().gsis_batch_workspace_bytes(b.arr, len(problems), ctypes.byref(o), ctypes.byref(n)))
    return int(n.value)


def solve_batch(problems, options: Options | None = None, tuning: BatchTuning | None = None,
                workspace=None, stream=None):
    """gsis_solve_batch: returns dict(results=[dict(rho, F, iters, err, status)], status, workspace)."""
    b = _Batch(problems)
    o = options or default_options()
    workspace = _workspace(batch_workspace_bytes(problems, o), workspace, b.device)
    rc = load().gsis_solve_batch(b.arr, len(problems), ctypes.byref(o), ctypes.byref(tuning) if tuning else None,
                                 ctypes.c_void_p(workspace.data_ptr()), ctypes.c_size_t(workspace.numel()),
                                 _stream(stream))
    _raise(rc)
    res = [dict(rho=b.rho[i], F=b.F[i], iters=b.arr[i].iters, err=b.arr[i].err, status=b.arr[i].status)
           for i in range(len(problems))]
    return dict(results=res, status=rc, workspace=workspace)


def batch_autotune(problems, options: Options | None = None, trial_iters: int = 3, workspace=None, stream=None):
    """gsis_batch_autotune: returns dict(tuning, ms_per_iter, class_ms, workspace)."""
    b = _Batch(problems, with_outputs=False)
    o = options or default_options()
    workspace = _workspace(batch_workspace_bytes(problems, o), workspace, b.device)
    t = BatchTuning()
    ms = ctypes.c_double(0.0)
    cls = (ctypes.c_double * len(KERNEL_CLASSES))()
    _raise(load().gsis_batch_autotune(b.arr, len(problems), ctypes.byref(o), trial_iters, ctypes.byref(t),
                                      ctypes.byref(ms), cls, ctypes.c_void_p(workspace.data_ptr()),
                                      ctypes.c_size_t(workspace.numel()), _stream(stream)))
    return dict(tuning=t, ms_per_iter=ms.value, class_ms=dict(zip(KERNEL_CLASSES, list(cls))),
                workspace=workspace)


# ------------------------------------------------------------ time-dependent
class TimeParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("c", ctypes.c_double), ("a", ctypes.c_double),
                ("cv", ctypes.c_double), ("nsteps", ctypes.c_int), ("predictor", ctypes.c_int)]


def _td_load():
    lib = load()
    if not getattr(lib, "_td_bound", False):
        vp, sz = ctypes.c_void_p, ctypes.c_size_t
        Mp, Qp, Op = ctypes.POINTER(Mesh), ctypes.POINTER(Quadrature), ctypes.POINTER(Options)
        lib.gsis_td_workspace_bytes.argtypes = [Mp, Qp, Op, ctypes.POINTER(sz)]
        lib.gsis_td_workspace_bytes.restype = ctypes.c_int
        lib.gsis_td_solve.argtypes = [Mp, Qp, Op, ctypes.POINTER(TimeParams), vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                      ctypes.POINTER(ctypes.c_int), _P, vp, sz, vp]
        lib.gsis_td_solve.restype = ctypes.c_int
        lib._td_bound = True
    return lib


def td_workspace_bytes(dx, dy, mu, eta, w, options: Options | None = None) -> int:
    a = _Args(dx, dy, mu, eta, w)
    o = options or default_options()
    n = ctypes.c_size_t(0)
    _raise(_td_load().gsis_td_workspace_bytes(ctypes.byref(a.mesh), ctypes.byref(a.quad), ctypes.byref(o),
                                              ctypes.byref(n)))
    return int(n.value)


def td_solve(dx, dy, mu, eta, w, sigma_a, sigma_s, q, rho0, T0, dt, nsteps, c=1.0, a=1.0, cv=1.0,
             inflow=None, options: Options | None = None, workspace=None, stream=None, predictor=0):
    """gsis_td_solve: returns dict(rho, T, F, step_iters, step_err, status, workspace).
    predictor: first iterate of each step (0 previous step, 1 linear, 2
    quadratic extrapolation in time; gsis_time_params)."""
    import torch
    args = _Args(dx, dy, mu, eta, w)
    o = options or default_options()
    N, K = args.mesh.nx * args.mesh.ny, args.quad.K
    dev = sigma_a.device
    rho = torch.empty(N, dtype=torch.float64, device=dev)
    T = torch.empty(N, dtype=torch.float64, device=dev)
    F = torch.empty(2 * N, dtype=torch.float64, device=dev)
    its = (ctypes.c_int * nsteps)()
    errs = np.zeros(nsteps)
    tp = TimeParams(dt, c, a, cv, nsteps, predictor)
    workspace = _workspace(td_workspace_bytes(args.dx, args.dy, args.mu, args.eta, args.w, o), workspace, dev)
    rc = _td_load().gsis_td_solve(
        ctypes.byref(args.mesh), ctypes.byref(args.quad), ctypes.byref(o), ctypes.byref(tp),
        _dev(sigma_a, N, "sigma_a"), _dev(sigma_s, N, "sigma_s"), _dev(q, N, "q"),
        _dev(inflow, 2 * (args.mesh.nx + args.mesh.ny) * K, "inflow"), _dev(rho0, N, "rho0"), _dev(T0, N, "T0"),
        _dev(rho), _dev(T), _dev(F), its, _hp(errs), ctypes.c_void_p(workspace.data_ptr()),
        ctypes.c_size_t(workspace.numel()), _stream(stream))
    _raise(rc)
    return dict(rho=rho, T=T, F=F, step_iters=np.array(list(its)), step_err=errs, status=rc, workspace=workspace)


def _td_adj_load():
    lib = _td_load()
    if not getattr(lib, "_td_adj_bound", False):
        vp, sz = ctypes.c_void_p, ctypes.c_size_t
        Mp, Qp, Op = ctypes.POINTER(Mesh), ctypes.POINTER(Quadrature), ctypes.POINTER(Options)
        Tp = ctypes.POINTER(TimeParams)
        lib.gsis_td_adjoint_workspace_bytes.argtypes = [Mp, Qp, Op, Tp, ctypes.c_int, ctypes.POINTER(sz)]
        lib.gsis_td_adjoint_workspace_bytes.restype = ctypes.c_int
        lib.gsis_td_adjoint.argtypes = [Mp, Qp, Op, Tp, ctypes.c_int] + [vp] * 14 + [ctypes.POINTER(ctypes.c_int),
                                                                                     vp, sz, vp]
        lib.gsis_td_adjoint.restype = ctypes.c_int
        lib._td_adj_bound = True
    return lib


def td_adjoint_workspace_bytes(dx, dy, mu, eta, w, dt, nsteps, checkpoint_every, c=1.0, a=1.0, cv=1.0,
                               options: Options | None = None) -> int:
    ar = _Args(dx, dy, mu, eta, w)
    o = options or default_options()
    tp = TimeParams(dt, c, a, cv, nsteps)
    n = ctypes.c_size_t(0)
    _raise(_td_adj_load().gsis_td_adjoint_workspace_bytes(ctypes.byref(ar.mesh), ctypes.byref(ar.quad),
                                                          ctypes.byref(o), ctypes.byref(tp),
                                                          int(checkpoint_every), ctypes.byref(n)))
    return int(n.value)


def td_adjoint(dx, dy, mu, eta, w, sigma_a, sigma_s, q, rho0, T0, dt, nsteps, dJ_drho=None, dJ_dT=None,
               checkpoint_every=None, c=1.0, a=1.0, cv=1.0, inflow=None, options: Options | None = None,
               workspace=None, stream=None, predictor=0):
    """gsis_td_adjoint: gradient of dJ_drho . rho^N + dJ_dT . T^N after a
    time-dependent GSIS run with respect to sigma_a, sigma_s, rho^0, T^0.
    checkpoint_every defaults to ceil(sqrt(nsteps)).  Returns dict(grad_sigma_a,
    grad_sigma_s, grad_rho0, grad_T0, rho, T, adj_iters, status, workspace)."""
    import math as _m

    import torch
    ar = _Args(dx, dy, mu, eta, w)
    o = options or default_options()
    N, K = ar.mesh.nx * ar.mesh.ny, ar.quad.K
    if checkpoint_every is None:
        checkpoint_every = max(1, _m.isqrt(nsteps - 1) + 1 if nsteps > 1 else 1)
    dev = sigma_a.device
    out = {k: torch.empty(N, dtype=torch.float64, device=dev)
           for k in ("rho", "T", "grad_sigma_a", "grad_sigma_s", "grad_rho0", "grad_T0")}
    its = (ctypes.c_int * nsteps)()
    tp = TimeParams(dt, c, a, cv, nsteps, predictor)
    workspace = _workspace(td_adjoint_workspace_bytes(ar.dx, ar.dy, ar.mu, ar.eta, ar.w, dt, nsteps,
                                                      checkpoint_every, c, a, cv, o), workspace, dev)
    rc = _td_adj_load().gsis_td_adjoint(
        ctypes.byref(ar.mesh), ctypes.byref(ar.quad), ctypes.byref(o), ctypes.byref(tp), int(checkpoint_every),
        _dev(sigma_a, N, "sigma_a"), _dev(sigma_s, N, "sigma_s"), _dev(q, N, "q"),
        _dev(inflow, 2 * (ar.mesh.nx + ar.mesh.ny) * K, "inflow"), _dev(rho0, N, "rho0"), _dev(T0, N, "T0"),
        _dev(dJ_drho, N, "dJ_drho"), _dev(dJ_dT, N, "dJ_dT"), _dev(out["rho"]), _dev(out["T"]),
        _dev(out["grad_sigma_a"]), _dev(out["grad_sigma_s"]), _dev(out["grad_rho0"]), _dev(out["grad_T0"]), its,
        ctypes.c_void_p(workspace.data_ptr()), ctypes.c_size_t(workspace.numel()), _stream(stream))
    _raise(rc)
    out.update(adj_iters=np.array(list(its)), status=rc, workspace=workspace, checkpoint_every=checkpoint_every)
    return out


def _peak_load():
    lib = load()
    if not getattr(lib, "_peak_bound", False):
        for f in (lib.gsis_measure_fp64_fma, lib.gsis_measure_fp32_fma):
            f.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
            f.restype = ctypes.c_int
        lib._peak_bound = True
    return lib


def measure_fp64_fma(stream=None) -> float:
    """gsis_measure_fp64_fma: the device's FP64 FMA rate in GFLOP/s."""
    g = ctypes.c_double(0.0)
    _raise(_peak_load().gsis_measure_fp64_fma(ctypes.byref(g), _stream(stream)))
    return float(g.value)


def measure_fp32_fma(stream=None) -> float:
    """gsis_measure_fp32_fma: the device's FP32 FMA rate in GFLOP/s."""
    g = ctypes.c_double(0.0)
    _raise(_peak_load().gsis_measure_fp32_fma(ctypes.byref(g), _stream(stream)))
    return float(g.value)
