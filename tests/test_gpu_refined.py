"""The refined FP32 preconditioner (AAO_PREC_FP32_REFINED): z0 = P32^{-1} x,
r = P z0 - x in compensated FP32, z = z0 - P32^{-1} r.

Its residual is P z - x = -dr + dP d (dr the rounding of r, dP the backward
error of the FP32 apply of the correction d), so its backward error is about
the FP32 one times ||d|| / ||z||: the product of two FP32 apply errors.
Every case asserts that bound (tests._helpers.refined_bw_tol, with ||d|| /
||z|| measured against the plain FP32 apply of the same input), and an
element-wise error against the oracle where the forward bound
32 t^2 + 4 kappa 2^-53 (t the FP32 element-wise bound, kappa 2^-24 for the
wave forms) stays below 1e-2; above that a forward bound pins nothing."""
import numpy as np
import pytest

import synthetic as syn
from oracle import precond, system
from tests._helpers import (U32, U64, backward_error, bw_tol, fp32_tol, kappa, need_gpu,
                            oracle_system, rand_block, refined_bw_tol, rel_max, to_dev, to_host)

pytestmark = pytest.mark.gpu

ELEMENTWISE_MAX = 1e-2


def refined_tol(S, kind, n, ell):
    t = fp32_tol(n, ell)
    if kind.startswith("wave"):
        t = max(t, kappa(S) * U32)
    return 32 * t * t + 4 * kappa(S) * U64


SHAPES = [(1, 1), (2, 4), (15, 16), (17, 16), (33, 64), (100, 128), (255, 256), (257, 32),
          (64, 1024), (130, 2)]


@pytest.mark.parametrize("n,ell", SHAPES)
@pytest.mark.parametrize("kind", ["heat", "wave_bd2", "heat_literal", "wave_bd4"])
@pytest.mark.parametrize("transpose", [False, True])
def test_refined_apply_matches_oracle(n, ell, kind, transpose):
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    S = oracle_system(kind, n, ell)
    X = rand_block(n, ell, 2000 + n + ell)
    want = precond.circulant_inverse(S, X, transpose=transpose)
    a = AllAtOnce(n, ell, 1.0 / ell, equation=kind, precision="fp32_refined", restart=1)
    got = to_host(a.precond_apply(to_dev(torch, X), transpose=transpose))
    err = rel_max(got, want)
    tol = refined_tol(S, kind, n, ell)
    if tol < ELEMENTWISE_MAX:
        assert err <= tol
    a.set_precision("fp32")
    z0 = to_host(a.precond_apply(to_dev(torch, X), transpose=transpose))
    d = np.linalg.norm(z0 - got) / max(np.linalg.norm(got), 1e-300)
    eta = backward_error(S, X, got, transpose)
    assert eta <= refined_bw_tol(n, ell, d), (eta, d)
    # and the plain apply it refines is within the FP32 backward bound
    assert backward_error(S, X, z0, transpose) <= bw_tol(n, ell, U32)


@pytest.mark.parametrize("transpose", [False, True])
def test_refined_apply_full_size(transpose):
    """n = 4095, ell = 4096: against the spectral oracle, and the residual
    P z - x with P applied from its definition."""
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n, ell = 4095, 4096
    S = oracle_system("heat", n, ell)
    X = rand_block(n, ell, 12)
    a = AllAtOnce(n, ell, 1.0 / ell, precision="fp32_refined", restart=1)
    Y = to_host(a.precond_apply(to_dev(torch, X), transpose=transpose))
    want = precond.circulant_inverse_spectral(S, X, transpose=transpose)
    assert rel_max(Y, want) <= refined_tol(S, "heat", n, ell)
    R = precond.circulant_matvec(S, Y, transpose=transpose) - X
    assert np.linalg.norm(R) / np.linalg.norm(X) <= 1e-7


@pytest.mark.parametrize("transpose", [False, True])
def test_refined_neumann_matches_oracle(transpose):
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n, ell = 63, 128
    taus = syn.time_steps(ell, 0.9, syn.rng(5))
    S = oracle_system("heat", n, ell, taus=taus)
    X = rand_block(n, ell, 8)
    a = AllAtOnce(n, ell, 1.0 / ell, precision="fp32_refined", restart=1)
    a.set_steps(taus)
    tol = 3 * refined_tol(oracle_system("heat", n, ell), "heat", n, ell)
    for terms in (1, 2, 3):
        want = precond.neumann_inverse(S, X, terms, transpose=transpose)
        got = to_host(a.neumann_apply(to_dev(torch, X), terms, transpose=transpose))
        assert rel_max(got, want) <= tol, terms


@pytest.mark.parametrize("kind", ["heat", "wave_bd2"])
def test_refined_solve_takes_the_fp64_iteration_count(kind):
    """The refined apply is accurate enough that FGMRES needs the iterations
    of the FP64 preconditioner (FP32 alone needs about two more)."""
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n, ell = (1023, 1024) if kind == "heat" else (511, 512)
    S = oracle_system(kind, n, ell)
    if kind == "heat":
        B = system.rhs_heat(S, syn.heat_initial(n, modes=8))
    else:
        u0, v0 = syn.wave_initial(n, modes=16)
        B = system.rhs_bd2(S, u0, v0)
    want = system.forward_substitution(S, B)
    its = {}
    for prec in ("fp64", "fp32_refined"):
        a = AllAtOnce(n, ell, 1.0 / ell, equation=kind, precision=prec, restart=30)
        x, info = a.solve(to_dev(torch, B), rtol=1e-10)
        assert info["relres_true"] <= 1e-10
        assert rel_max(to_host(x), want) <= 1e-8
        its[prec] = info["iters"]
    assert its["fp32_refined"] <= its["fp64"] + 1


def test_refined_solve_full_size():
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n, ell = 4095, 4096
    a = AllAtOnce(n, ell, 1.0 / ell, precision="fp32_refined", restart=30)
    b = a.build_rhs(to_dev(torch, syn.heat_initial(n, modes=8)))
    x, info = a.solve(b, rtol=1e-10)
    assert info["relres_true"] <= 1e-10
    assert info["iters"] <= 3
    # sampled rows against time stepping
    S = oracle_system("heat", n, ell)
    U = system.forward_substitution(S, to_host(b))
    assert rel_max(to_host(x)[::512], U[::512]) <= 1e-8


def test_refined_adjoint_matches_fp64():
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n, ell = 255, 256
    G = to_dev(torch, rand_block(n, ell, 31))
    out = {}
    for prec in ("fp64", "fp32_refined"):
        a = AllAtOnce(n, ell, 1.0 / ell, precision=prec, restart=30)
        lam, info = a.adjoint_solve(G, rtol=1e-10)
        assert info["relres_true"] <= 1e-10
        out[prec] = to_host(lam)
    assert rel_max(out["fp32_refined"], out["fp64"]) <= 1e-8


def test_static_scratch_apply_rejects_refined_mode():
    torch = need_gpu()
    import ctypes as C
    from paper_1810_00615_gb300 import AllAtOnce, _capi
    lib = _capi.lib()
    n, ell = 63, 64
    a = AllAtOnce(n, ell, 1.0 / ell, precision="fp32_refined", restart=1)
    X = to_dev(torch, rand_block(n, ell, 3))
    Y = torch.empty_like(X)
    st = lib.aao_precond_apply_static(a._ctx, C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr()),
                                      0, C.c_void_p(int(torch.cuda.current_stream().cuda_stream)))
    assert st == _capi.AAO_EINVAL
    assert b"refined" in lib.aao_last_error(a._ctx)
