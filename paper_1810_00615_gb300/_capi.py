"""ctypes declarations of the C ABI in include/aao.h (argument marshalling only).

Every entry point named here is implemented in libaao.so; nothing in this
package computes any part of the solve on the host.  If the library is
missing or was built elsewhere, ``lib()`` builds it with nvcc (the CUDA
toolkit is required) or raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import threading

from . import _build

AAO_HEAT, AAO_WAVE_BD2, AAO_HEAT_LITERAL, AAO_WAVE_BD4 = 0, 1, 2, 3
AAO_PREC_FP64, AAO_PREC_FP32, AAO_PREC_FP32_REFINED = 0, 1, 2
AAO_SPACE_TRIDIAG, AAO_SPACE_DST = 0, 1
AAO_GUESS_GIVEN, AAO_GUESS_ZERO = 0, 1
AAO_OK, AAO_ENOCONV = 0, 1
AAO_EINVAL, AAO_ENOMEM, AAO_ECUDA, AAO_ENUMERIC, AAO_EUNSUPPORTED = -1, -2, -3, -4, -5
KERNEL_CLASSES = ["fft_forward", "tridiag", "fft_inverse", "matvec", "dots", "update",
                  "combine", "other", "refine", "fft_forward_solve",
                  "fft_inverse_solve"]


class SolveInfo(C.Structure):
    _fields_ = [
        ("iters", C.c_int),
        ("restarts", C.c_int),
        ("relres_true", C.c_double),
        ("relres_est", C.c_double),
        ("history", C.POINTER(C.c_double)),
        ("history_cap", C.c_int),
        ("history_len", C.c_int),
    ]


# name -> (restype, argtypes)
SIGNATURES = {
    "aao_create": (C.c_int, [C.c_int64, C.c_int64, C.c_double, C.c_int, C.POINTER(C.c_void_p)]),
    "aao_destroy": (None, [C.c_void_p]),
    "aao_set_kappa": (C.c_int, [C.c_void_p, C.c_double]),
    "aao_set_steps": (C.c_int, [C.c_void_p, C.c_void_p]),
    "aao_set_precision": (C.c_int, [C.c_void_p, C.c_int]),
    "aao_set_space_solver": (C.c_int, [C.c_void_p, C.c_int]),
    "aao_set_initial_guess": (C.c_int, [C.c_void_p, C.c_int]),
    "aao_workspace_bytes": (C.c_size_t, [C.c_void_p, C.c_int]),
    "aao_set_workspace": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "aao_precond_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "aao_neumann_apply": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                    C.c_void_p]),
    "aao_matvec": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "aao_matvec_sub": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                 C.c_void_p]),
    "aao_matvec_f32": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                 C.c_void_p]),
    "aao_circulant_residual_f32": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_int, C.c_void_p]),
    "aao_residual": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                               C.POINTER(C.c_double), C.c_void_p]),
    "aao_matvec_dots": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_int, C.POINTER(C.c_double), C.c_void_p]),
    "aao_build_rhs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "aao_gmres_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                                  C.c_int, C.c_int, C.POINTER(SolveInfo), C.c_void_p]),
    "aao_adjoint_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                                    C.c_int, C.c_int, C.POINTER(SolveInfo), C.c_void_p]),
    "aao_adjoint_grads": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.POINTER(C.c_double), C.c_void_p]),
    "aao_solve_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                 C.c_double, C.c_int, C.c_int, C.POINTER(SolveInfo),
                                 C.c_void_p]),
    "aao_profile_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "aao_profile_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                   C.c_int]),
    "aao_kernel_launches": (C.c_int64, [C.c_void_p]),
    "aao_precond_apply_static": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                           C.c_void_p]),
    "aao_check_conversions": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                        C.c_void_p]),
    "aao_workspace_check": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "aao_strerror": (C.c_char_p, [C.c_int]),
    "aao_last_error": (C.c_char_p, [C.c_void_p]),
}

_lock = threading.Lock()
_lib = None


def lib(build_if_needed: bool = True) -> C.CDLL:
    """Load libaao.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not _build.is_current():
            if not build_if_needed:
                raise RuntimeError("libaao.so is not built for this machine; run build()")
            _build.build()
        handle = C.CDLL(_build.LIB)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
        return _lib


class AAOError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = lib().aao_strerror(status).decode()
        super().__init__(f"{where}: {msg} ({status}){': ' + detail if detail else ''}")


def check(status: int, where: str, ctx=None, allow_noconv: bool = False) -> int:
    if status == AAO_OK or (allow_noconv and status == AAO_ENOCONV):
        return status
    detail = lib().aao_last_error(ctx).decode() if ctx else ""
    raise AAOError(status, where, detail)
