"""The allocation-free preconditioner apply (aao_precond_apply_static).

Some callers cannot allocate device memory where they apply the
preconditioner: code recorded into a CUDA graph by stream capture, plug-ins
that must stay off the host program's allocator, runtimes that forbid
allocation after start-up.  For them the library keeps its frequency-domain
scratch in a fixed 32 MiB array of its own.  These tests call that entry
point through the C ABI and check it against the oracle (Section 3: P^{-1}
through the sine (x) Fourier eigenbasis, and P applied from its definition
for the backward error), on two calls in a row (the second reuses the shared
scratch left by the first), in both precisions and both orientations, over
the transform lengths that take different kernels (short, radix-16,
mixed-radix, the longest), a wave form, the DST-in-space solver and the
largest FP32 system that fits.  The file is named so that pytest collects it
last.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import precond
from tests._helpers import (U32, U64, backward_error, bw_tol, fp32_tol, kappa, need_gpu,
                            oracle_system, rand_block, rel_max, to_dev, to_host)

pytestmark = pytest.mark.gpu


def _stream(torch):
    return C.c_void_p(int(torch.cuda.current_stream().cuda_stream))


def _static_apply(torch, lib, a, X, transpose):
    got = torch.empty_like(X)
    st = lib.aao_precond_apply_static(a._ctx, C.c_void_p(X.data_ptr()),
                                      C.c_void_p(got.data_ptr()), transpose, _stream(torch))
    return st, got


CASES = [  # (kind, n, ell, space)
    ("heat", 63, 16, "tridiag"),
    ("heat", 63, 256, "tridiag"),
    ("heat", 127, 1024, "tridiag"),
    ("heat", 31, 4096, "tridiag"),
    ("heat", 47, 96, "tridiag"),          # mixed radix
    ("wave_bd2", 63, 256, "tridiag"),
    ("heat", 255, 256, "dst"),
    ("heat", 1023, 512, "tridiag"),
]


@pytest.mark.parametrize("kind,n,ell,space", CASES)
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("transpose", [0, 1])
def test_static_scratch_apply_matches_oracle(kind, n, ell, space, prec, transpose):
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    from paper_1810_00615_gb300 import _capi
    lib = _capi.lib()
    S = oracle_system(kind, n, ell)
    a = AllAtOnce(n, ell, 1.0 / ell, equation=kind, precision=prec, restart=1, space=space)
    u = U64 if prec == "fp64" else U32
    before = a.kernel_launches()
    for call in range(2):      # the second call reuses the scratch of the first
        Xh = rand_block(n, ell, 500 + 7 * call + n)
        st, got = _static_apply(torch, lib, a, to_dev(torch, Xh), transpose)
        assert st == _capi.AAO_OK, lib.aao_last_error(a._ctx)
        torch.cuda.synchronize()
        Y = to_host(got)
        want = precond.circulant_inverse_spectral(S, Xh, transpose=bool(transpose))
        assert backward_error(S, Xh, Y, bool(transpose)) <= bw_tol(n, ell, u)
        tol = (max(1e-10, 4 * kappa(S) * U64) if prec == "fp64"
               else max(fp32_tol(n, ell), kappa(S) * U32 if kind != "heat" else 0.0))
        if tol < 1e-2:
            assert rel_max(Y, want) <= tol
    # every launch is counted by the context, as for the workspace apply
    assert a.kernel_launches() > before


def test_static_scratch_largest_fp32_system():
    """n = 4095, ell = 1024 in FP32: (513 x 4096) complex64 = 16.8 MB of the
    32 MiB array."""
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    from paper_1810_00615_gb300 import _capi
    lib = _capi.lib()
    n, ell = 4095, 1024
    S = oracle_system("heat", n, ell)
    a = AllAtOnce(n, ell, 1.0 / ell, precision="fp32", restart=1)
    for call in range(2):
        Xh = rand_block(n, ell, 900 + call)
        st, got = _static_apply(torch, lib, a, to_dev(torch, Xh), 0)
        assert st == _capi.AAO_OK, lib.aao_last_error(a._ctx)
        torch.cuda.synchronize()
        Y = to_host(got)
        assert rel_max(Y, precond.circulant_inverse_spectral(S, Xh)) <= fp32_tol(n, ell)
        assert backward_error(S, Xh, Y) <= bw_tol(n, ell, U32)


def test_static_scratch_rejects_systems_that_do_not_fit():
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    from paper_1810_00615_gb300 import _capi
    lib = _capi.lib()
    n, ell = 4095, 4096         # spectrum 2049 x 4096 x 8 bytes = 64 MiB
    a = AllAtOnce(n, ell, 1.0 / ell, precision="fp32", restart=1)
    X = torch.zeros(ell, n, dtype=torch.float64, device="cuda")
    st, _ = _static_apply(torch, lib, a, X, 0)
    assert st == _capi.AAO_EINVAL
    assert b"static scratch" in lib.aao_last_error(a._ctx)
