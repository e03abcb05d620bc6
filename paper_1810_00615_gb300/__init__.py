"""GB300 all-at-once solver: MPW block-circulant preconditioned GMRES.

Python binding of libaao.so (include/aao.h).  PyTorch supplies device memory
and the current CUDA stream; every step of the solve runs in the library's
CUDA kernels.  Goddard & Wathen, "A note on parallel preconditioning for
all-at-once evolutionary PDEs": Section 2 defines the all-at-once systems and
the preconditioners, Section 3 the Fourier diagonalisation applied here.

    >>> aao = AllAtOnce(n=4095, ell=4096, tau=1/4096)        # heat equation
    >>> b = aao.build_rhs(u0)                                  # [M u0; 0; ...]
    >>> U, info = aao.solve(b, restart=30, rtol=1e-10)         # FP32 precond
"""
from __future__ import annotations

import ctypes as C
import weakref
from typing import Optional

import numpy as np
import torch

from . import _build
from ._capi import (AAO_ECUDA, AAO_EINVAL, AAO_ENOCONV, AAO_ENUMERIC, AAO_EUNSUPPORTED,
                    AAO_HEAT, AAO_HEAT_LITERAL, AAO_OK, AAO_PREC_FP32, AAO_PREC_FP32_REFINED, AAO_PREC_FP64,
                    AAO_SPACE_DST, AAO_SPACE_TRIDIAG,
                    AAO_WAVE_BD2, AAO_WAVE_BD4, AAOError, SolveInfo, check, lib)

__all__ = ["AllAtOnce", "AAOSolve", "SolveInfo", "AAOError", "lib", "build",
           "AAO_HEAT", "AAO_WAVE_BD2", "AAO_WAVE_BD4", "AAO_HEAT_LITERAL", "AAO_PREC_FP32", "AAO_PREC_FP32_REFINED", "AAO_PREC_FP64",
           "AAO_SPACE_TRIDIAG", "AAO_SPACE_DST", "AAO_OK", "AAO_ENOCONV", "AAO_EINVAL", "AAO_ECUDA", "AAO_ENUMERIC",
           "AAO_EUNSUPPORTED"]

EQUATIONS = {"heat": AAO_HEAT, "wave_bd2": AAO_WAVE_BD2, "heat_literal": AAO_HEAT_LITERAL,
             "wave_bd4": AAO_WAVE_BD4}


def build(force: bool = False) -> str:
    """Compile libaao.so for sm_103a (in-tree) and return its path."""
    return _build.build(force=force)


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dev_f64(t: torch.Tensor, numel: int, name: str, dtype=torch.float64) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype:
        raise TypeError(f"{name} must be a CUDA {str(dtype).replace('torch.', '')} tensor")
    if not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{name} must be contiguous with {numel} elements")
    return t


class AllAtOnce:
    """One all-at-once system (n spatial nodes, ell time steps) on one GPU.

    equation: "heat" (implicit Euler, A0 = M + tau kappa K, A1 = -M),
    "wave_bd2" (A0 = M + tau^2 K, A1 = -2M, A2 = M), "wave_bd4" (A0 = 2M +
    tau^2 K, A1 = -5M, A2 = 4M, A3 = -M after two BD2 start-up rows;
    preconditioned by R_BD4) or "heat_literal" (the printed A0 = K + tau M).  precision: "fp32", "fp32_refined" (FP32 with
    one refinement sweep, FP64-like accuracy) or "fp64" for the
    preconditioner; the outer GMRES is FP64 either way.
    """

    # every live instance (for workspace guard checks after a test or a run)
    _live: "weakref.WeakSet[AllAtOnce]" = weakref.WeakSet()

    def __init__(self, n: int, ell: int, tau: Optional[float] = None, equation="heat",
                 kappa: float = 1.0, precision: str = "fp32", restart: int = 30,
                 device=None, space: str = "tridiag"):
        self.lib = lib()
        self.n, self.ell = int(n), int(ell)
        self.N = self.n * self.ell
        self.tau = float(tau) if tau is not None else 1.0 / self.ell
        self.equation = EQUATIONS[equation] if isinstance(equation, str) else int(equation)
        self.device = torch.device(device) if device is not None else torch.device("cuda")
        self._ctx = C.c_void_p()
        with torch.cuda.device(self.device):
            check(self.lib.aao_create(self.n, self.ell, self.tau, self.equation,
                                      C.byref(self._ctx)), "aao_create")
        self.kappa = 1.0
        if kappa != 1.0:
            self.set_kappa(kappa)
        self.set_precision(precision)
        self.space = "tridiag"
        if space != "tridiag":
            self.set_space_solver(space)
        self._ws = None
        self._restart = 0
        self.ensure_workspace(restart)
        AllAtOnce._live.add(self)

    # ------------------------------------------------------------ settings
    def __del__(self):
        ctx = getattr(self, "_ctx", None)
        if ctx is not None and ctx.value:
            self.lib.aao_destroy(ctx)
            self._ctx = None

    def set_kappa(self, kappa: float):
        check(self.lib.aao_set_kappa(self._ctx, float(kappa)), "aao_set_kappa", self._ctx)
        self.kappa = float(kappa)

    def set_steps(self, taus: Optional[np.ndarray]):
        if taus is None:
            check(self.lib.aao_set_steps(self._ctx, None), "aao_set_steps", self._ctx)
            return
        arr = np.ascontiguousarray(taus, dtype=np.float64)
        if arr.size != self.ell:
            raise ValueError("need ell steps")
        check(self.lib.aao_set_steps(self._ctx, arr.ctypes.data), "aao_set_steps", self._ctx)

    def set_precision(self, precision: str):
        p = {"fp32": AAO_PREC_FP32, "fp64": AAO_PREC_FP64,
             "fp32_refined": AAO_PREC_FP32_REFINED}[precision]
        check(self.lib.aao_set_precision(self._ctx, p), "aao_set_precision", self._ctx)
        self.precision = precision

    def set_space_solver(self, space: str):
        sv = {"tridiag": AAO_SPACE_TRIDIAG, "dst": AAO_SPACE_DST}[space]
        check(self.lib.aao_set_space_solver(self._ctx, sv), "aao_set_space_solver", self._ctx)
        self.space = space

    def workspace_bytes(self, restart: int) -> int:
        return int(self.lib.aao_workspace_bytes(self._ctx, int(restart)))

    def ensure_workspace(self, restart: int):
        if self._ws is not None and restart <= self._restart:
            return
        nbytes = self.workspace_bytes(restart)
        if nbytes == 0:
            raise ValueError("bad restart length")
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        off = (-ws.data_ptr()) % 256
        self._ws = ws
        check(self.lib.aao_set_workspace(self._ctx, ws.data_ptr() + off, nbytes),
              "aao_set_workspace", self._ctx)
        self._restart = restart

    # -------------------------------------------------------------- kernels
    def _out(self, out):
        if out is None:
            return torch.empty(self.ell, self.n, dtype=torch.float64, device=self.device)
        return _dev_f64(out, self.N, "out")

    def precond_apply(self, x, transpose=False, out=None, stream=None):
        """y = P^{-1} x (or P^{-T} x)."""
        x = _dev_f64(x, self.N, "x")
        y = self._out(out)
        check(self.lib.aao_precond_apply(self._ctx, x.data_ptr(), y.data_ptr(),
                                         int(bool(transpose)), _stream(stream)),
              "aao_precond_apply", self._ctx)
        return y

    def neumann_apply(self, x, terms: int, transpose=False, out=None, stream=None):
        """y = Q_i^{-1} x with i = terms (Neumann series of Section 2)."""
        x = _dev_f64(x, self.N, "x")
        y = self._out(out)
        check(self.lib.aao_neumann_apply(self._ctx, int(terms), x.data_ptr(), y.data_ptr(),
                                         int(bool(transpose)), _stream(stream)),
              "aao_neumann_apply", self._ctx)
        return y

    def matvec(self, x, transpose=False, out=None, sub=None, stream=None):
        """y = A x (or A^T x) in FP64; with sub, y = A x - sub (fused)."""
        x = _dev_f64(x, self.N, "x")
        y = self._out(out)
        if sub is not None:
            sub = _dev_f64(sub, self.N, "sub")
            check(self.lib.aao_matvec_sub(self._ctx, x.data_ptr(), sub.data_ptr(), y.data_ptr(),
                                          int(bool(transpose)), _stream(stream)),
                  "aao_matvec_sub", self._ctx)
            return y
        check(self.lib.aao_matvec(self._ctx, x.data_ptr(), y.data_ptr(), int(bool(transpose)),
                                  _stream(stream)), "aao_matvec", self._ctx)
        return y

    def matvec_f32(self, x, transpose=False, out=None, sub=None, stream=None):
        """y = A x (or A^T x) of an FP32 x, in FP64; with sub, y = A x - sub
        (the shifted-Arnoldi product the mixed solver forms)."""
        x = _dev_f64(x, self.N, "x", torch.float32)
        sp = _dev_f64(sub, self.N, "sub").data_ptr() if sub is not None else None
        y = self._out(out)
        check(self.lib.aao_matvec_f32(self._ctx, x.data_ptr(), sp, y.data_ptr(),
                                      int(bool(transpose)), _stream(stream)),
              "aao_matvec_f32", self._ctx)
        return y

    def matvec_dots(self, x, v, v0=None, transpose=False, out=None, stream=None):
        """w = A x - v (or A^T x - v) and its Arnoldi dots in one pass:
        returns (w, [v0 . w,] v . w, w . w) (synchronises)."""
        self.ensure_workspace(self._restart)
        x = _dev_f64(x, self.N, "x")
        v = _dev_f64(v, self.N, "v")
        v0p = _dev_f64(v0, self.N, "v0").data_ptr() if v0 is not None else None
        w = self._out(out)
        d = (C.c_double * 3)()
        check(self.lib.aao_matvec_dots(self._ctx, x.data_ptr(), v.data_ptr(), v0p, w.data_ptr(),
                                       int(bool(transpose)), d, _stream(stream)),
              "aao_matvec_dots", self._ctx)
        return w, [d[q] for q in range(3 if v0 is not None else 2)]

    def residual(self, x, b, transpose=False, out=None, stream=None):
        """r = A x - b (or A^T x - b) and ||r||^2 in one pass (synchronises)."""
        self.ensure_workspace(self._restart)
        x = _dev_f64(x, self.N, "x")
        b = _dev_f64(b, self.N, "b")
        r = self._out(out)
        nrm = C.c_double()
        check(self.lib.aao_residual(self._ctx, x.data_ptr(), b.data_ptr(), r.data_ptr(),
                                    int(bool(transpose)), C.byref(nrm), _stream(stream)),
              "aao_residual", self._ctx)
        return r, float(nrm.value)

    def circulant_residual_f32(self, z, x, transpose=False, out=None, stream=None):
        """r = P z - x (or P^T z - x) for an FP32 z, in FP64: the residual of
        the refined FP32 preconditioner apply."""
        z = _dev_f64(z, self.N, "z", torch.float32)
        x = _dev_f64(x, self.N, "x")
        r = self._out(out)
        check(self.lib.aao_circulant_residual_f32(self._ctx, z.data_ptr(), x.data_ptr(),
                                                  r.data_ptr(), int(bool(transpose)),
                                                  _stream(stream)),
              "aao_circulant_residual_f32", self._ctx)
        return r

    def build_rhs(self, u0, v0=None, out=None, stream=None):
        u0 = _dev_f64(u0, self.n, "u0")
        vp = None
        if v0 is not None:
            vp = _dev_f64(v0, self.n, "v0").data_ptr()
        b = self._out(out)
        check(self.lib.aao_build_rhs(self._ctx, u0.data_ptr(), vp, b.data_ptr(),
                                     _stream(stream)), "aao_build_rhs", self._ctx)
        return b

    def _solve(self, fn, name, b, x0, restart, rtol, maxit, precond, history, stream):
        self.ensure_workspace(restart)
        b = _dev_f64(b, self.N, "b")
        if x0 is None:
            # x0 = 0 without a fill: the solver never reads x and writes it whole
            x = torch.empty(self.ell, self.n, dtype=torch.float64, device=self.device)
            guess = 1
        else:
            x = _dev_f64(x0, self.N, "x0").clone()
            guess = 0
        check(self.lib.aao_set_initial_guess(self._ctx, guess), "aao_set_initial_guess",
              self._ctx)
        info = SolveInfo()
        hist = None
        if history:
            hist = (C.c_double * int(history))()
            info.history = C.cast(hist, C.POINTER(C.c_double))
            info.history_cap = int(history)
        st = fn(self._ctx, b.data_ptr(), x.data_ptr(), int(restart), float(rtol), int(maxit),
                int(precond), C.byref(info), _stream(stream))
        check(st, name, self._ctx, allow_noconv=True)
        out = {"status": st, "iters": info.iters, "restarts": info.restarts,
               "relres_true": info.relres_true, "relres_est": info.relres_est,
               "converged": st == AAO_OK}
        if hist is not None:
            out["history"] = [hist[i] for i in range(info.history_len)]
        return x, out

    def solve(self, b, x0=None, restart=30, rtol=1e-10, maxit=300, precond=1, history=0,
              stream=None):
        """Flexible GMRES on A x = b; precond 0 none, 1 P, i >= 2 Neumann Q_i."""
        return self._solve(self.lib.aao_gmres_solve, "aao_gmres_solve", b, x0, restart, rtol,
                           maxit, precond, history, stream)

    def adjoint_solve(self, g, x0=None, restart=30, rtol=1e-10, maxit=300, precond=1,
                      history=0, stream=None):
        """Flexible GMRES on A^T lam = g with P^{-T}."""
        return self._solve(self.lib.aao_adjoint_solve, "aao_adjoint_solve", g, x0, restart,
                           rtol, maxit, precond, history, stream)

    def adjoint_grads(self, lam, U, stream=None):
        """(M lam_1, -sum_t tau_t lam_t^T K u_t) for the heat equation."""
        lam = _dev_f64(lam, self.N, "lam")
        U = _dev_f64(U, self.N, "U")
        g_u0 = torch.empty(self.n, dtype=torch.float64, device=self.device)
        gk = C.c_double()
        check(self.lib.aao_adjoint_grads(self._ctx, lam.data_ptr(), U.data_ptr(),
                                         g_u0.data_ptr(), C.byref(gk), _stream(stream)),
              "aao_adjoint_grads", self._ctx)
        return g_u0, gk.value

    def profile(self, on: bool = True):
        """Bracket every kernel of this context with CUDA events (or stop)."""
        check(self.lib.aao_profile_enable(self._ctx, int(bool(on))), "aao_profile_enable",
              self._ctx)

    def profile_read(self, reset: bool = False):
        """{class: (milliseconds, launches)} since the last reset."""
        from ._capi import KERNEL_CLASSES
        ms = (C.c_double * len(KERNEL_CLASSES))()
        nl = (C.c_int64 * len(KERNEL_CLASSES))()
        check(self.lib.aao_profile_read(self._ctx, ms, nl, int(bool(reset))),
              "aao_profile_read", self._ctx)
        return {k: (ms[i], nl[i]) for i, k in enumerate(KERNEL_CLASSES)}

    def kernel_launches(self) -> int:
        return int(self.lib.aao_kernel_launches(self._ctx))

    def workspace_check(self) -> int:
        """Number of damaged 8-byte guard words around the workspace's regions
        and basis vectors (0: no kernel wrote outside its region)."""
        bad = C.c_int64(0)
        with torch.cuda.device(self.device):
            check(self.lib.aao_workspace_check(self._ctx, C.byref(bad)), "aao_workspace_check",
                  self._ctx)
        return int(bad.value)

    @classmethod
    def live_instances(cls):
        return list(cls._live)

    def solve_host(self, u0: torch.Tensor, v0: Optional[torch.Tensor] = None, out=None,
                   restart=30, rtol=1e-10, maxit=300, precond=1, stream=None):
        """End-to-end solve from host initial data to a host solution U."""
        self.ensure_workspace(restart)
        u0 = u0.contiguous()
        if u0.dtype != torch.float64 or u0.is_cuda or u0.numel() != self.n:
            raise TypeError("u0 must be a CPU float64 tensor of n elements")
        vp = None
        if v0 is not None:
            v0 = v0.contiguous()
            vp = v0.data_ptr()
        if out is None:
            out = torch.empty(self.ell, self.n, dtype=torch.float64, pin_memory=True)
        info = SolveInfo()
        st = self.lib.aao_solve_host(self._ctx, u0.data_ptr(), vp, out.data_ptr(), int(restart),
                                     float(rtol), int(maxit), int(precond), C.byref(info),
                                     _stream(stream))
        check(st, "aao_solve_host", self._ctx, allow_noconv=True)
        return out, {"status": st, "iters": info.iters, "relres_true": info.relres_true}


class AAOSolve(torch.autograd.Function):
    """U = A(kappa)^{-1} [M u0; 0; ...] for the heat equation, differentiable in
    u0 and kappa by the adjoint system A^T lam = dL/dU (solved by flexible
    GMRES with P^{-T} on the GPU).

    forward(u0 [n] CUDA float64, kappa [] float64, solver: AllAtOnce, rtol)
    returns U [ell, n].
    """

    @staticmethod
    def forward(ctx, u0, kappa, solver: AllAtOnce, rtol: float = 1e-12, restart: int = 30):
        k = float(kappa.item()) if isinstance(kappa, torch.Tensor) else float(kappa)
        if k != solver.kappa:
            solver.set_kappa(k)
        b = solver.build_rhs(u0.detach().contiguous())
        U, info = solver.solve(b, rtol=rtol, restart=restart)
        if not info["converged"]:
            raise AAOError(AAO_ENOCONV, "AAOSolve.forward")
        ctx.solver = solver
        ctx.rtol = rtol
        ctx.restart = restart
        ctx.kappa_is_tensor = isinstance(kappa, torch.Tensor)
        ctx.kappa_device = kappa.device if ctx.kappa_is_tensor else None
        ctx.save_for_backward(U)
        return U

    @staticmethod
    def backward(ctx, gU):
        (U,) = ctx.saved_tensors
        solver = ctx.solver
        lam, info = solver.adjoint_solve(gU.contiguous().to(torch.float64), rtol=ctx.rtol,
                                         restart=ctx.restart)
        if not info["converged"]:
            raise AAOError(AAO_ENOCONV, "AAOSolve.backward")
        g_u0, g_k = solver.adjoint_grads(lam, U)
        gk = torch.tensor(g_k, dtype=torch.float64, device=ctx.kappa_device) \
            if ctx.kappa_is_tensor else None
        return g_u0, gk, None, None, None
