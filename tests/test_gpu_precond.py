"""Parity of the CUDA preconditioner applies (aao_precond_apply,
aao_neumann_apply) with the oracle (Sections 2 and 3).

Two measures, both against the oracle:
* Backward error eta = ||P y - x|| / (||P|| ||y|| + ||x||), P applied from
  its definition (tests._helpers.backward_error).  It is asserted for every
  case: FP32 within bw_tol(n, ell, 2^-24), FP64 within bw_tol(n, ell,
  2^-53), whatever the condition number of P.
* Element-wise (max-norm relative) error against the oracle's inverse, with
  a tolerance from the arithmetic:
  - FP64: both sides are backward stable, so they agree to eps64 times the
    condition number kappa of the circulant (max|lam| / min|lam| over its
    sine (x) Fourier symbols): max(1e-10, 4 kappa 2^-53).
  - FP32, heat: the blocks are shifted Laplacians with a non-negative row
    excess; in excess form no step subtracts two O(1) numbers to get a
    small one, so each mode keeps O(2^-24) relative accuracy through input
    rounding, the FFT, the chunk Thomas and the separator levels
    (tests._helpers.fp32_tol).
  - FP32, BD2 / BD4: the blocks (1 - w_k)^2 M + tau^2 K (BD4: times
    (2 - w_k) on M) are indefinite and come close to singular, so the
    forward error is of order kappa 2^-24.  That comparison is made only
    where kappa 2^-24 < 1e-2; above, a forward bound pins nothing and the
    backward error carries the check.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import precond
from tests._helpers import (U32, U64, backward_error, bw_tol, fp32_tol, kappa, need_gpu,
                            oracle_system, rand_block, refined_bw_tol, rel_max, to_dev, to_host)

pytestmark = pytest.mark.gpu

ELEMENTWISE_MAX = 1e-2   # element-wise tolerances at or above this pin nothing


def tol_for(S, kind, prec, n, ell):
    if prec == "fp64":
        return max(1e-10, 4 * kappa(S) * U64)
    if kind.startswith("wave"):
        return max(fp32_tol(n, ell), kappa(S) * U32)
    return fp32_tol(n, ell)


def check_apply(S, kind, prec, n, ell, X, got, want, transpose):
    """Backward error always; element-wise error where its bound is tight."""
    u = U64 if prec == "fp64" else U32
    eta = backward_error(S, X, got, transpose)
    assert eta <= bw_tol(n, ell, u), ("backward", eta)
    tol = tol_for(S, kind, prec, n, ell)
    if tol < ELEMENTWISE_MAX:
        assert rel_max(got, want) <= tol, ("elementwise", rel_max(got, want), tol)


SHAPES = [(1, 1), (1, 2), (2, 4), (3, 8), (15, 16), (16, 16), (17, 16), (31, 32), (33, 64),
          (63, 64), (100, 128), (255, 256), (257, 32), (64, 1024), (130, 2)]


@pytest.mark.parametrize("n,ell", SHAPES)
@pytest.mark.parametrize("kind", ["heat", "wave_bd2", "wave_bd4"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("transpose", [False, True])
def test_precond_matches_oracle(n, ell, kind, prec, transpose):
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    S = oracle_system(kind, n, ell)
    X = rand_block(n, ell, 1000 + n + ell)
    want = precond.circulant_inverse(S, X, transpose=transpose)
    a = AllAtOnce(n, ell, 1.0 / ell, equation=kind, precision=prec, restart=1)
    got = to_host(a.precond_apply(to_dev(torch, X), transpose=transpose))
    torch.cuda.synchronize()
    check_apply(S, kind, prec, n, ell, X, got, want, transpose)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_precond_kappa_and_literal(prec):
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n, ell = 47, 64
    X = rand_block(n, ell, 7)
    a = AllAtOnce(n, ell, 1.0 / ell, precision=prec, kappa=0.37, restart=1)
    want = precond.circulant_inverse(oracle_system("heat", n, ell, kappa=0.37), X)
    assert rel_max(to_host(a.precond_apply(to_dev(torch, X))), want) <= (
        1e-10 if prec == "fp64" else fp32_tol(n, ell))
    b = AllAtOnce(n, ell, 1.0 / ell, equation="heat_literal", precision=prec, restart=1)
    want = precond.circulant_inverse(oracle_system("heat_literal", n, ell), X)
    assert rel_max(to_host(b.precond_apply(to_dev(torch, X))), want) <= (
        1e-10 if prec == "fp64" else fp32_tol(n, ell))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("transpose", [False, True])
def test_neumann_matches_oracle(prec, transpose):
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n, ell = 63, 128
    taus = syn.time_steps(ell, 0.9, syn.rng(5))
    S = oracle_system("heat", n, ell, taus=taus)
    X = rand_block(n, ell, 8)
    a = AllAtOnce(n, ell, 1.0 / ell, precision=prec, restart=1)
    a.set_steps(taus)
    for terms in (1, 2, 3):
        want = precond.neumann_inverse(S, X, terms, transpose=transpose)
        got = to_host(a.neumann_apply(to_dev(torch, X), terms, transpose=transpose))
        tol = 1e-10 if prec == "fp64" else 3 * fp32_tol(n, ell)
        assert rel_max(got, want) <= tol, terms


def test_neumann_uniform_steps_equals_circulant():
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n, ell = 31, 64
    X = to_dev(torch, rand_block(n, ell, 9))
    a = AllAtOnce(n, ell, 1.0 / ell, restart=1)
    p = a.precond_apply(X)
    for terms in (1, 2, 3):
        assert torch.equal(a.neumann_apply(X, terms), p)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("transpose", [False, True])
def test_precond_full_size_matches_spectral_oracle(prec, transpose):
    """n = 4095, ell = 4096 (the benchmark size and launch configuration):
    the GPU apply against the oracle's sine (x) Fourier route on a random
    block vector; plus the residual P y - x with P applied from its
    definition (FP64 only: in FP32 the rounding of y alone gives a residual
    of order kappa 2^-24 / sqrt(n ell) ~ 1e-4, whatever the method)."""
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n, ell = 4095, 4096
    S = oracle_system("heat", n, ell)
    X = rand_block(n, ell, 11)
    a = AllAtOnce(n, ell, 1.0 / ell, precision=prec, restart=1)
    Y = to_host(a.precond_apply(to_dev(torch, X), transpose=transpose))
    want = precond.circulant_inverse_spectral(S, X, transpose=transpose)
    check_apply(S, "heat", prec, n, ell, X, Y, want, transpose)
    if prec == "fp64":
        R = precond.circulant_matvec(S, Y, transpose=transpose) - X
        assert np.linalg.norm(R) / np.linalg.norm(X) <= 1e-11


@pytest.mark.parametrize("j,k", [(1, 0), (1, 1), (3, 7), (100, 2048), (4095, 1)])
def test_precond_full_size_sine_fourier_mode(j, k):
    """P^{-1} maps s_j (x) cos(2 pi k t/ell) to Re(s_j e^{2 pi i k t/ell} /
    (a0_j + w_k a1_j)): an exact closed form at the benchmark size.

    For a mode with a large symbol the rounding of the input and of the FFT
    leaks into the smoothest mode, whose symbol is smaller by
    r = |lam_jk| / min|lam| (up to 7e6 here): the attainable accuracy is
    r eps, so the tolerance is max(1e-10, 4 r 2^-53) in FP64 and
    max(2e-5, 4 r 2^-24) in FP32 (FP32 is skipped where that exceeds 1e-2)."""
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n, ell = 4095, 4096
    tau = 1.0 / ell
    h = 1.0 / (n + 1)
    th = j * np.pi * h
    m = (h / 6) * (4 + 2 * np.cos(th))
    kk = (2 / h) * (1 - np.cos(th))
    a0, a1 = m + tau * kk, -m
    t = np.arange(ell)
    ph = np.exp(2j * np.pi * k * t / ell)
    s = np.sin(j * np.pi * syn.grid(n))
    X = (ph[:, None] * s[None, :]).real
    w = np.exp(-2j * np.pi * k / ell)
    want = ((ph / (a0 + w * a1))[:, None] * s[None, :]).real
    from oracle import system as osys
    lam = np.abs(precond.sine_fourier_symbols(osys.heat(n, ell, tau)))
    r = abs(a0 + w * a1) / lam.min()
    cases = [("fp64", max(1e-10, 4 * r * U64))]
    if 4 * r * U32 < ELEMENTWISE_MAX:
        cases.append(("fp32", max(2e-5, 4 * r * U32)))
    for prec, tol in cases:
        a = AllAtOnce(n, ell, tau, precision=prec, restart=1)
        got = to_host(a.precond_apply(to_dev(torch, X)))
        assert rel_max(got, want) <= tol, prec


def test_precond_rejects_aliasing_and_missing_workspace():
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce, AAOError
    a = AllAtOnce(15, 16, 1 / 16, restart=1)
    X = to_dev(torch, rand_block(15, 16, 1))
    with pytest.raises(AAOError):
        a.precond_apply(X, out=X)


@pytest.mark.parametrize("n,ell", [(16383, 16), (32767, 8), (65535, 16)])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("transpose", [False, True])
def test_precond_long_rows_cluster_form(n, ell, prec, transpose):
    """Rows longer than one CTA holds (the n = 65535 workload's spatial size)
    are solved by a cluster of CTAs sharing the separator system through
    distributed shared memory; checked against the oracle's sine (x) Fourier
    route."""
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    S = oracle_system("heat", n, ell)
    X = rand_block(n, ell, 77 + n)
    a = AllAtOnce(n, ell, 1.0 / ell, precision=prec, restart=1)
    got = to_host(a.precond_apply(to_dev(torch, X), transpose=transpose))
    want = precond.circulant_inverse_spectral(S, X, transpose=transpose)
    check_apply(S, "heat", prec, n, ell, X, got, want, transpose)


@pytest.mark.parametrize("ell", [256, 512, 1024, 2048, 4096])
@pytest.mark.parametrize("n", [1, 2, 3, 64, 127, 130])
@pytest.mark.parametrize("prec", ["fp32", "fp32_refined"])
@pytest.mark.parametrize("transpose", [False, True])
def test_precond_four_step_lengths_match_oracle(ell, n, prec, transpose):
    """ell = 256 ... 4096 (the four-step FP32 transforms, factors 16/32/64),
    at column counts that leave ragged 32-column blocks; the refined mode
    also runs the inverse with its base (z0 - P^{-1} r)."""
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    S = oracle_system("heat", n, ell)
    X = rand_block(n, ell, 4000 + n)
    want = precond.circulant_inverse_spectral(S, X, transpose=transpose)
    a = AllAtOnce(n, ell, 1.0 / ell, precision=prec, restart=1)
    got = to_host(a.precond_apply(to_dev(torch, X), transpose=transpose))
    t = fp32_tol(n, ell)
    tol = t if prec == "fp32" else 32 * t * t + 4 * kappa(S) * U64
    assert rel_max(got, want) <= tol
    eta = backward_error(S, X, got, transpose)
    if prec == "fp32":
        assert eta <= bw_tol(n, ell, U32)
    else:
        a.set_precision("fp32")
        z0 = to_host(a.precond_apply(to_dev(torch, X), transpose=transpose))
        d = np.linalg.norm(z0 - got) / max(np.linalg.norm(got), 1e-300)
        assert eta <= refined_bw_tol(n, ell, d)


@pytest.mark.parametrize("kind,n,ell", [("wave_bd2", 1023, 1024), ("wave_bd2", 8191, 2048),
                                        ("wave_bd4", 1023, 1024), ("wave_bd4", 255, 256)])
@pytest.mark.parametrize("prec", ["fp32", "fp32_refined", "fp64"])
def test_wave_apply_backward_error_at_scale(kind, n, ell, prec):
    """The wave circulants R_BD2 / R_BD4 at the wave workload's size (n =
    8191, ell = 2048, kappa 2e9) and below it, where kappa 2^-24 exceeds 1
    and only the backward error can pin the FP32 apply: FP32 and FP64 within
    bw_tol; the refined apply within the product bound refined_bw_tol (its
    correction measured against the plain FP32 apply of the same input)."""
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    S = oracle_system(kind, n, ell)
    X = rand_block(n, ell, 6100 + n)
    a = AllAtOnce(n, ell, 1.0 / ell, equation=kind, precision=prec, restart=1)
    for tr in (False, True):
        got = to_host(a.precond_apply(to_dev(torch, X), transpose=tr))
        eta = backward_error(S, X, got, tr)
        if prec == "fp32_refined":
            a.set_precision("fp32")
            z0 = to_host(a.precond_apply(to_dev(torch, X), transpose=tr))
            a.set_precision("fp32_refined")
            d = np.linalg.norm(z0 - got) / np.linalg.norm(got)
            assert eta <= refined_bw_tol(n, ell, d), (tr, eta, d)
            # the refinement gains: its backward error is far below FP32's
            assert eta <= 1e-3 * bw_tol(n, ell, U32), (tr, eta)
        else:
            assert eta <= bw_tol(n, ell, U64 if prec == "fp64" else U32), (tr, eta)
        if n * ell > 4_000_000:
            break


def test_short_workspace_is_rejected_before_any_launch():
    """A workspace shorter than the layout needs is refused by
    aao_set_workspace, and a solve asking for a longer restart than the
    workspace holds returns AAO_EINVAL without launching a kernel; the guard
    words of the workspace stay intact throughout."""
    torch = need_gpu()
    import ctypes as C
    from paper_1810_00615_gb300 import AllAtOnce, _capi
    lib = _capi.lib()
    n, ell = 63, 64
    a = AllAtOnce(n, ell, 1.0 / ell, restart=2)
    need0 = a.workspace_bytes(0)
    buf = torch.empty(need0, dtype=torch.uint8, device="cuda")
    base = buf.data_ptr() + (-buf.data_ptr()) % 256
    assert lib.aao_set_workspace(a._ctx, C.c_void_p(base), need0 - 4096) == _capi.AAO_EINVAL
    b = a.build_rhs(to_dev(torch, syn.heat_initial(n)))
    x = torch.zeros_like(b)
    before = a.kernel_launches()
    st = lib.aao_gmres_solve(a._ctx, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), 20,
                             1e-10, 100, 1, None,
                             C.c_void_p(int(torch.cuda.current_stream().cuda_stream)))
    assert st == _capi.AAO_EINVAL
    assert a.kernel_launches() == before
    assert a.workspace_check() == 0
