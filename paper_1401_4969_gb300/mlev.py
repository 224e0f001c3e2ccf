"""Python binding of the mlev C ABI (include/mlev.h): argument marshalling only.

Every step of the solve runs in the CUDA kernels of libmlev.so; this module only
loads the library, passes host arrays and torch-owned device pointers, and turns
status codes into exceptions. There is no CPU fallback: if the library or a CUDA
device is missing, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import _build

MLEV_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENOCONV", -5: "ETIMEOUT", -6: "EUNSUPPORTED",
          -7: "ESTATE"}
KAPPA_ONE, KAPPA_PER_COARSE_CELL, KAPPA_PER_FINE_ELEM = 0, 1, 2
GLUE_PAPER = 0
PREC_FP64, PREC_MIXED = 0, 1
MAX_LEVELS = 10

EXPORTS = ["mlev_opts_default", "mlev_create", "mlev_destroy", "mlev_last_error", "mlev_set_domain",
           "mlev_set_partition", "mlev_set_levels", "mlev_set_forms", "mlev_workspace_size", "mlev_problem_info",
           "mlev_solve", "mlev_solve_host", "mlev_profile_read", "mlev_solve_noalloc", "mlev_grad_workspace_size",
           "mlev_grad_kappa", "mlev_set_eigenpairs"]
MAX_EIGENPAIRS = 8
NOALLOC_WORKSPACE_BYTES = 32 << 20
GRAD_FINE_ELEM, GRAD_COARSE_CELL = 0, 1


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("vcycles", C.c_int), ("refine_passes", C.c_int),
                ("strip_vcycles", C.c_int), ("pre_smooth", C.c_int), ("post_smooth", C.c_int),
                ("coarse_sweeps", C.c_int), ("level1_max_iter", C.c_int), ("level1_tol", C.c_double),
                ("rr_max_iter", C.c_int), ("use_graph", C.c_int), ("omega", C.c_double),
                ("check_residuals", C.c_int), ("profile", C.c_int), ("fused", C.c_int), ("tail_nodes", C.c_int),
                ("reg_depths", C.c_int), ("reserved", C.c_int)]


class KernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int), ("ms", C.c_double), ("bytes", C.c_double)]


class Report(C.Structure):
    _fields_ = [("levels", C.c_int), ("batch", C.c_int), ("lambda_", C.c_double * (MAX_LEVELS + 1)),
                ("level1_iters", C.c_int), ("level1_residual", C.c_double),
                ("rr_iters", C.c_int * (MAX_LEVELS + 1)), ("local_residual", C.c_double * (MAX_LEVELS + 1)),
                ("strip_residual", C.c_double * (MAX_LEVELS + 1)), ("n_fine", C.c_longlong),
                ("n_local_fine", C.c_longlong), ("n_strip_fine", C.c_longlong), ("n_coarse", C.c_int),
                ("kernel_launches", C.c_int), ("status_flags", C.c_int), ("h2d_bytes", C.c_longlong),
                ("d2h_bytes", C.c_longlong)]

    def as_dict(self) -> dict:
        n = self.levels
        return {"levels": n, "batch": self.batch, "lambda_levels": [self.lambda_[k] for k in range(1, n + 1)],
                "level1_iters": self.level1_iters, "level1_residual": self.level1_residual,
                "rr_iters": [self.rr_iters[k] for k in range(2, n + 1)],
                "local_residual": [self.local_residual[k] for k in range(2, n + 1)],
                "strip_residual": [self.strip_residual[k] for k in range(2, n + 1)], "n_fine": self.n_fine,
                "n_local_fine": self.n_local_fine, "n_strip_fine": self.n_strip_fine, "n_coarse": self.n_coarse,
                "kernel_launches": self.kernel_launches, "status_flags": self.status_flags,
                "h2d_bytes": self.h2d_bytes, "d2h_bytes": self.d2h_bytes}


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load libmlev.so (building it in-tree first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"mlev CUDA library not found at {path}")
    lib = C.CDLL(path)
    P, I, D, VP, SZ = C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_size_t
    lib.mlev_opts_default.argtypes = [C.POINTER(Opts)]
    lib.mlev_opts_default.restype = None
    lib.mlev_create.argtypes = [C.POINTER(P), I]
    lib.mlev_destroy.argtypes = [P]
    lib.mlev_destroy.restype = None
    lib.mlev_last_error.argtypes = [P]
    lib.mlev_last_error.restype = C.c_char_p
    lib.mlev_set_domain.argtypes = [P, I, I, D, D, D, VP]
    lib.mlev_set_partition.argtypes = [P, I, VP, VP, D, I]
    lib.mlev_set_levels.argtypes = [P, I]
    lib.mlev_set_forms.argtypes = [P, I, I, VP, I]
    lib.mlev_set_eigenpairs.argtypes = [P, I]
    lib.mlev_workspace_size.argtypes = [P, C.POINTER(Opts), C.POINTER(SZ)]
    lib.mlev_problem_info.argtypes = [P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                      C.POINTER(C.c_longlong), C.POINTER(C.c_int)]
    lib.mlev_solve.argtypes = [P, C.POINTER(Opts), VP, SZ, VP, VP, VP, C.POINTER(Report)]
    lib.mlev_solve_host.argtypes = [P, C.POINTER(Opts), VP, SZ, VP, VP, VP, VP, C.POINTER(Report)]
    lib.mlev_profile_read.argtypes = [P, C.POINTER(KernelStat), I, C.POINTER(I)]
    lib.mlev_solve_noalloc.argtypes = [P, C.POINTER(Opts), VP, VP, VP, C.POINTER(Report)]
    lib.mlev_grad_workspace_size.argtypes = [P, C.POINTER(Opts), C.POINTER(SZ)]
    lib.mlev_grad_kappa.argtypes = [P, C.POINTER(Opts), VP, SZ, VP, VP, I, VP, VP, C.POINTER(Report)]
    for name in ("mlev_create", "mlev_set_domain", "mlev_set_partition", "mlev_set_levels", "mlev_set_forms",
                 "mlev_set_eigenpairs",
                 "mlev_workspace_size", "mlev_problem_info", "mlev_solve", "mlev_solve_host", "mlev_profile_read",
                 "mlev_solve_noalloc", "mlev_grad_workspace_size", "mlev_grad_kappa"):
        getattr(lib, name).restype = I
    _lib = lib
    return lib


class MlevError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mlev {ERRORS.get(code, code)}: {msg}")
        self.code = code


def default_opts(**kw) -> Opts:
    o = Opts()
    load().mlev_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class Solver:
    """One mlev context: geometry, partition, levels and forms of a (batched) problem.

    ``problem`` is any object with the attributes of ``workloads.Problem``: ncx, ncy,
    x0, y0, H, cell_in, cell_owner, overlap, delta, levels, batch, kappa_kind, kappa.
    """

    def __init__(self, problem, device: int = 0, kappa_device=None, eigenpairs: int = 1):
        """device = -1 gives a planning-only context (set-up, validation, sizes; no solves);
        eigenpairs = q computes the q smallest eigenpairs of every problem (outputs gain a
        dimension q after the batch one)."""
        import torch

        if device >= 0 and not torch.cuda.is_available():
            raise RuntimeError("mlev needs a CUDA device; there is no CPU fallback")
        self.lib = load()
        self.device = device
        self.problem = problem
        h = C.c_void_p()
        rc = self.lib.mlev_create(C.byref(h), device)
        if rc != MLEV_OK:
            raise MlevError(rc, "mlev_create failed")
        self.h = h
        p = problem
        self._cell_in = np.ascontiguousarray(p.cell_in, dtype=np.uint8)
        self._owner = np.ascontiguousarray(p.cell_owner, dtype=np.int32)
        self._overlap = np.ascontiguousarray(p.overlap, dtype=np.int32)
        self._check(self.lib.mlev_set_domain(h, p.ncx, p.ncy, p.x0, p.y0, p.H, _ptr(self._cell_in)))
        self._check(self.lib.mlev_set_partition(h, int(self._overlap.size), _ptr(self._owner), _ptr(self._overlap),
                                                float(p.delta), GLUE_PAPER))
        self._check(self.lib.mlev_set_levels(h, p.levels))
        self.kappa_device = kappa_device
        if p.kappa_kind == KAPPA_ONE:
            self._check(self.lib.mlev_set_forms(h, p.batch, KAPPA_ONE, None, 0))
        elif kappa_device is not None:
            assert kappa_device.is_cuda and kappa_device.dtype == torch.float64 and kappa_device.is_contiguous()
            self._check(self.lib.mlev_set_forms(h, p.batch, p.kappa_kind, C.c_void_p(kappa_device.data_ptr()), 1))
        else:
            self._kappa = np.ascontiguousarray(p.kappa, dtype=np.float64)
            self._check(self.lib.mlev_set_forms(h, p.batch, p.kappa_kind, _ptr(self._kappa), 0))
        self.q = int(eigenpairs)
        self._check(self.lib.mlev_set_eigenpairs(h, self.q))
        self._ws = None

    def _check(self, rc: int):
        if rc != MLEV_OK:
            raise MlevError(rc, self.lib.mlev_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.mlev_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        nf, nl, ns, nc = C.c_longlong(), C.c_longlong(), C.c_longlong(), C.c_int()
        self._check(self.lib.mlev_problem_info(self.h, C.byref(nf), C.byref(nl), C.byref(ns), C.byref(nc)))
        return {"n_fine": nf.value, "n_local_fine": nl.value, "n_strip_fine": ns.value, "n_coarse": nc.value}

    def workspace_bytes(self, opts: Opts) -> int:
        b = C.c_size_t()
        self._check(self.lib.mlev_workspace_size(self.h, C.byref(opts), C.byref(b)))
        return b.value

    def grad_workspace_bytes(self, opts: Opts) -> int:
        b = C.c_size_t()
        self._check(self.lib.mlev_grad_workspace_size(self.h, C.byref(opts), C.byref(b)))
        return b.value

    def workspace(self, opts: Opts, grad: bool = False):
        import torch

        need = self.grad_workspace_bytes(opts) if grad else self.workspace_bytes(opts)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device=f"cuda:{self.device}")
            assert self._ws.data_ptr() % 256 == 0
        return self._ws

    def grid_shape(self):
        p = self.problem
        return ((p.ncy << p.levels) + 1, (p.ncx << p.levels) + 1)

    def alloc_outputs(self, want_u: bool = False):
        import torch

        dev = f"cuda:{self.device}"
        lead = (self.problem.batch,) if self.q == 1 else (self.problem.batch, self.q)
        lam = torch.empty(lead, dtype=torch.float64, device=dev)
        u = torch.empty((*lead, *self.grid_shape()), dtype=torch.float64, device=dev) if want_u else None
        return lam, u

    def solve_into(self, opts: Opts, lam, u=None, stream=None, report: bool = False):
        """mlev_solve on caller-provided device outputs; returns the report dict or None."""
        import torch

        ws = self.workspace(opts)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        rep = Report() if report else None
        rc = self.lib.mlev_solve(self.h, C.byref(opts), C.c_void_p(ws.data_ptr()), ws.numel(),
                                 C.c_void_p(s.cuda_stream), C.c_void_p(lam.data_ptr()),
                                 C.c_void_p(u.data_ptr()) if u is not None else None,
                                 C.byref(rep) if rep is not None else None)
        self._check(rc)
        return rep.as_dict() if rep is not None else None

    def solve_noalloc(self, opts: Opts, lam, u=None, stream=None, report: bool = False):
        """mlev_solve_noalloc: like solve_into but with the library's fixed workspace (no allocation)."""
        import torch

        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        rep = Report() if report else None
        rc = self.lib.mlev_solve_noalloc(self.h, C.byref(opts), C.c_void_p(s.cuda_stream), C.c_void_p(lam.data_ptr()),
                                         C.c_void_p(u.data_ptr()) if u is not None else None,
                                         C.byref(rep) if rep is not None else None)
        self._check(rc)
        return rep.as_dict() if rep is not None else None

    def solve(self, opts: Opts | None = None, want_u: bool = False, report: bool = True):
        opts = opts or default_opts()
        lam, u = self.alloc_outputs(want_u)
        rep = self.solve_into(opts, lam, u, report=report)
        return lam, u, rep

    def solve_host(self, opts: Opts, lam_host: np.ndarray, u_host: np.ndarray | None = None,
                   kappa_host: np.ndarray | None = None, stream=None, report: bool = False):
        """mlev_solve_host: host inputs/outputs, copies inside the call (synchronizes)."""
        import torch

        ws = self.workspace(opts)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        rep = Report() if report else None
        rc = self.lib.mlev_solve_host(self.h, C.byref(opts), C.c_void_p(ws.data_ptr()), ws.numel(),
                                      C.c_void_p(s.cuda_stream),
                                      _ptr(kappa_host) if kappa_host is not None else None, _ptr(lam_host),
                                      _ptr(u_host) if u_host is not None else None,
                                      C.byref(rep) if rep is not None else None)
        self._check(rc)
        return rep.as_dict() if rep is not None else None


    def grad_shape(self, layout: int):
        p = self.problem
        if layout == GRAD_COARSE_CELL:
            return (p.batch, p.ncy, p.ncx)
        return (p.batch, p.ncy << p.levels, p.ncx << p.levels, 2)

    def grad_kappa(self, opts: Opts | None = None, dlambda=None, layout: int | None = None, stream=None,
                   report: bool = False):
        """mlev_grad_kappa: (dkappa, lambda, report) with dkappa = dlambda_b * dlambda_{h_n}/dkappa on the
        device. ``layout`` defaults to per coarse cell for a per-cell kappa, else per finest triangle."""
        import torch

        opts = opts or default_opts()
        p = self.problem
        if layout is None:
            layout = GRAD_COARSE_CELL if p.kappa_kind == KAPPA_PER_COARSE_CELL else GRAD_FINE_ELEM
        dev = f"cuda:{self.device}"
        if dlambda is None:
            dlambda = torch.ones(p.batch, dtype=torch.float64, device=dev)
        assert dlambda.is_cuda and dlambda.dtype == torch.float64 and dlambda.is_contiguous()
        assert dlambda.numel() == p.batch
        ws = self.workspace(opts, grad=True)
        dk = torch.empty(self.grad_shape(layout), dtype=torch.float64, device=dev)
        lam = torch.empty(p.batch, dtype=torch.float64, device=dev)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        rep = Report() if report else None
        rc = self.lib.mlev_grad_kappa(self.h, C.byref(opts), C.c_void_p(ws.data_ptr()), ws.numel(),
                                      C.c_void_p(s.cuda_stream), C.c_void_p(dlambda.data_ptr()), layout,
                                      C.c_void_p(dk.data_ptr()), C.c_void_p(lam.data_ptr()),
                                      C.byref(rep) if rep is not None else None)
        self._check(rc)
        return dk, lam, (rep.as_dict() if rep is not None else None)

    def set_kappa(self, kappa):
        """Copy new coefficient values into the device buffer this solver was created with
        (``kappa_device``); the next solve reads them."""
        if self.kappa_device is None:
            raise MlevError(-7, "set_kappa needs a solver created with kappa_device")
        self.kappa_device.copy_(kappa.reshape(self.kappa_device.shape))


def kappa_solver(problem, device: int = 0) -> Solver:
    """A Solver whose coefficient lives in a device buffer (initialised from problem.kappa),
    as ``LambdaFn`` needs."""
    import torch

    if problem.kappa_kind == KAPPA_ONE:
        raise MlevError(-1, "the problem has no coefficient array (kappa_kind ONE)")
    buf = torch.tensor(np.ascontiguousarray(problem.kappa, dtype=np.float64), device=f"cuda:{device}")
    return Solver(problem, device=device, kappa_device=buf)


def _autograd_function():
    import torch

    class LambdaFn(torch.autograd.Function):
        """lambda_{h_n}[b] of Algorithm 4.2 as a differentiable function of the coefficient.

        ``LambdaFn.apply(kappa, solver, opts)``: kappa has the shape of the solver's problem
        kappa ([B][ncy][ncx] per coarse cell or [B][fny][fnx][2] per finest triangle) and
        lives on the solver's device; ``solver`` comes from ``kappa_solver``. The backward
        pass is mlev_grad_kappa with the incoming gradient as upstream weights.
        """

        @staticmethod
        def forward(ctx, kappa, solver, opts):
            solver.set_kappa(kappa.detach())
            lam, _ = solver.alloc_outputs()
            solver.solve_into(opts, lam)
            ctx.solver, ctx.opts = solver, opts
            ctx.save_for_backward(kappa.detach().clone())
            return lam

        @staticmethod
        def backward(ctx, g):
            (kappa,) = ctx.saved_tensors
            ctx.solver.set_kappa(kappa)
            dk, _, _ = ctx.solver.grad_kappa(ctx.opts, g.detach().to(torch.float64).contiguous())
            return dk.reshape(kappa.shape), None, None

    return LambdaFn


def __getattr__(name):
    if name == "LambdaFn":
        fn = _autograd_function()
        globals()["LambdaFn"] = fn
        return fn
    raise AttributeError(name)


def eigensolve(problem, opts: Opts | None = None, want_u: bool = False, device: int = 0):
    """One-call solve: (lambda [B], u [B, ny+1, nx+1] or None, report)."""
    s = Solver(problem, device=device)
    try:
        return s.solve(opts, want_u=want_u)
    finally:
        s.close()


def profile_read(solver: "Solver") -> list[dict]:
    """Per-kernel-family statistics of the solver's last solve run with opts.profile = 1."""
    arr = (KernelStat * 64)()
    cnt = C.c_int()
    solver._check(solver.lib.mlev_profile_read(solver.h, arr, 64, C.byref(cnt)))
    return [{"name": arr[i].name.decode(), "launches": arr[i].launches, "ms": arr[i].ms, "bytes": arr[i].bytes}
            for i in range(min(cnt.value, 64))]
