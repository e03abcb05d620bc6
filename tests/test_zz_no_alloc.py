"""The allocation-free preconditioner apply (aao_precond_apply_static).

Some callers cannot allocate device memory where they apply the
preconditioner: code recorded into a CUDA graph by stream capture, plug-ins
that must stay off the host program's allocator, runtimes that forbid
allocation after start-up.  For them the library keeps its frequency-domain
scratch in a fixed 32 MiB array of its own.  This test calls that entry point
through the C ABI and checks it against the workspace-based
aao_precond_apply, on two calls in a row (the second reuses the shared
scratch left by the first), in both precisions and both orientations.  The
file is named so that pytest collects it last.
"""
import ctypes as C

import pytest

from tests._helpers import need_gpu, rand_block, rel_max, to_dev, to_host

pytestmark = pytest.mark.gpu


def _stream(torch):
    return C.c_void_p(int(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("transpose", [0, 1])
def test_static_scratch_apply_matches_workspace_apply(prec, transpose):
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    from paper_1810_00615_gb300 import _capi
    lib = _capi.lib()
    n, ell = 1023, 512          # spectrum 257 x 1024 complex: well inside 32 MiB
    a = AllAtOnce(n, ell, 1.0 / ell, precision=prec, restart=1)
    tol = 1e-10 if prec == "fp64" else 1e-5
    for call in range(2):      # the second call reuses the scratch of the first
        X = to_dev(torch, rand_block(n, ell, 500 + call))
        want = a.precond_apply(X, transpose=bool(transpose))
        got = torch.empty_like(X)
        st = lib.aao_precond_apply_static(a._ctx, C.c_void_p(X.data_ptr()),
                                          C.c_void_p(got.data_ptr()), transpose, _stream(torch))
        assert st == _capi.AAO_OK, lib.aao_last_error(a._ctx)
        torch.cuda.synchronize()
        assert rel_max(to_host(got), to_host(want)) <= tol


def test_static_scratch_rejects_systems_that_do_not_fit():
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    from paper_1810_00615_gb300 import _capi
    lib = _capi.lib()
    n, ell = 4095, 4096         # spectrum 2049 x 4096 x 8 bytes = 64 MiB
    a = AllAtOnce(n, ell, 1.0 / ell, precision="fp32", restart=1)
    X = torch.zeros(ell, n, dtype=torch.float64, device="cuda")
    Y = torch.empty_like(X)
    st = lib.aao_precond_apply_static(a._ctx, C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr()),
                                      0, _stream(torch))
    assert st == _capi.AAO_EINVAL
    assert b"static scratch" in lib.aao_last_error(a._ctx)
