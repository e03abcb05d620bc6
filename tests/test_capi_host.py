"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every entry point that include/aao.h declares, and
rejects invalid arguments before touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "aao.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(aao_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1810_00615_gb300 import _capi
    return _capi.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["aao_create", "aao_precond_apply", "aao_neumann_apply", "aao_matvec",
                     "aao_gmres_solve", "aao_adjoint_solve", "aao_destroy"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_1810_00615_gb300 import _capi
    assert set(_capi.SIGNATURES) == set(declared_functions())


def test_create_rejects_bad_arguments_without_a_device(lib):
    from paper_1810_00615_gb300 import _capi as K
    ctx = C.c_void_p()
    assert lib.aao_create(0, 64, 1 / 64, K.AAO_HEAT, C.byref(ctx)) == K.AAO_EINVAL
    assert lib.aao_create(63, 64, 0.0, K.AAO_HEAT, C.byref(ctx)) == K.AAO_EINVAL
    assert lib.aao_create(63, 64, -1.0, K.AAO_HEAT, C.byref(ctx)) == K.AAO_EINVAL
    assert lib.aao_create(63, 64, 1 / 64, 7, C.byref(ctx)) == K.AAO_EINVAL
    assert lib.aao_create(63, 49, 1 / 49, K.AAO_HEAT, C.byref(ctx)) == K.AAO_EUNSUPPORTED  # 7^2
    assert lib.aao_create(63, 14, 1 / 14, K.AAO_HEAT, C.byref(ctx)) == K.AAO_EUNSUPPORTED
    assert lib.aao_create(63, 8192, 1 / 8192, K.AAO_HEAT, C.byref(ctx)) == K.AAO_EUNSUPPORTED
    assert lib.aao_create(1 << 20, 64, 1 / 64, K.AAO_HEAT, C.byref(ctx)) == K.AAO_EUNSUPPORTED
    assert lib.aao_create(63, 64, 1 / 64, K.AAO_HEAT, None) == K.AAO_EINVAL
    assert not ctx.value


def test_null_context_calls_are_rejected(lib):
    from paper_1810_00615_gb300 import _capi as K
    assert lib.aao_set_kappa(None, 1.0) == K.AAO_EINVAL
    assert lib.aao_precond_apply(None, None, None, 0, None) == K.AAO_EINVAL
    assert lib.aao_matvec(None, None, None, 0, None) == K.AAO_EINVAL
    assert lib.aao_matvec_f32(None, None, None, None, 0, None) == K.AAO_EINVAL
    assert lib.aao_matvec_sub(None, None, None, None, 0, None) == K.AAO_EINVAL
    assert lib.aao_gmres_solve(None, None, None, 30, 1e-10, 10, 1, None, None) == K.AAO_EINVAL
    assert lib.aao_set_space_solver(None, K.AAO_SPACE_DST) == K.AAO_EINVAL
    assert lib.aao_circulant_residual_f32(None, None, None, None, 0, None) == K.AAO_EINVAL
    assert lib.aao_residual(None, None, None, None, 0, None, None) == K.AAO_EINVAL
    assert lib.aao_matvec_dots(None, None, None, None, None, 0, None, None) == K.AAO_EINVAL
    assert lib.aao_set_initial_guess(None, 0) == K.AAO_EINVAL
    assert lib.aao_workspace_bytes(None, 30) == 0
    lib.aao_destroy(None)


def test_strerror_texts(lib):
    for code in (0, 1, -1, -2, -3, -4, -5):
        assert lib.aao_strerror(code)
    assert lib.aao_strerror(99) == b"unknown status"
