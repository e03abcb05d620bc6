"""The DST-in-space form of the per-frequency solves (AAO_SPACE_DST): the
spatial blocks cM_k M + cK K diagonalised by DST-I as well (Section 3 with
the textbook sine eigenpairs of the uniform P1 matrices), against the
oracle's dense-DFT + banded-LU route.

Tolerances: FP64 and FP32 as for the tridiagonal form (test_gpu_precond: the
oracle itself is accurate only to kappa eps64).  What the DST form adds is
per-mode accuracy: a single sine (x) Fourier mode comes back divided by its
symbol to the transforms' rounding, 2^-24 times a few log2(n) in FP32, even
on the near-singular modes of R_BD4 where elimination loses kappa_k 2^-24."""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import precond, system
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


SHAPES = [(15, 16), (15, 1), (31, 2), (63, 64), (127, 8), (255, 256), (511, 32), (1023, 1024),
          (4095, 16), (63, 768)]


@pytest.mark.parametrize("n,ell", SHAPES)
@pytest.mark.parametrize("kind", ["heat", "wave_bd2", "wave_bd4", "heat_literal"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("transpose", [False, True])
def test_dst_apply_matches_oracle(n, ell, kind, prec, transpose):
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    S = oracle_system(kind, n, ell)
    X = rand_block(n, ell, 3000 + n + ell)
    want = (precond.circulant_inverse(S, X, transpose=transpose) if n * ell * ell <= 2 ** 26
            else precond.circulant_inverse_spectral(S, X, transpose=transpose))
    a = AllAtOnce(n, ell, 1.0 / ell, equation=kind, precision=prec, restart=1, space="dst")
    got = to_host(a.precond_apply(to_dev(torch, X), transpose=transpose))
    assert backward_error(S, X, got, transpose) <= bw_tol(n, ell, U64 if prec == "fp64" else U32)
    tol = tol_for(S, kind, prec, n, ell)
    if tol < ELEMENTWISE_MAX:
        assert rel_max(got, want) <= tol


@pytest.mark.parametrize("kind", ["heat", "wave_bd2", "wave_bd4"])
@pytest.mark.parametrize("transpose", [False, True])
def test_dst_single_mode_is_divided_by_its_symbol(kind, transpose):
    """X = Re(s_j (x) e^{2 pi i k t/ell}) for the mode with the smallest
    |symbol|, the largest, and one in between: FP32 output within
    2^-24 (8 log2(2(n+1)) + 16) of the mode divided by its symbol, relative
    to that output's size."""
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n, ell = 255, 256
    S = oracle_system(kind, n, ell)
    lam = precond.sine_fourier_symbols(S, transpose)
    half = np.abs(lam[: ell // 2 + 1])
    a = AllAtOnce(n, ell, 1.0 / ell, equation=kind, precision="fp32", restart=1, space="dst")
    t = np.arange(ell)
    xs = syn.grid(n)
    tol = (8 * math.log2(2 * (n + 1)) + 16) * U32
    picks = [np.unravel_index(np.argmin(half), half.shape),
             np.unravel_index(np.argmax(half), half.shape), (ell // 8, n // 3)]
    for k, j0 in picks:
        s = np.sin((j0 + 1) * np.pi * xs)
        ph = np.exp(2j * np.pi * k * t / ell)
        X = (ph[:, None] * s[None, :]).real
        want = ((ph / lam[k, j0])[:, None] * s[None, :]).real
        got = to_host(a.precond_apply(to_dev(torch, X), transpose=transpose))
        assert rel_max(got, want) <= tol, (k, j0, rel_max(got, want))


@pytest.mark.parametrize("transpose", [False, True])
def test_dst_neumann_and_refined(transpose):
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n, ell = 63, 128
    taus = syn.time_steps(ell, 0.9, syn.rng(5))
    S = oracle_system("heat", n, ell, taus=taus)
    X = rand_block(n, ell, 8)
    a = AllAtOnce(n, ell, 1.0 / ell, precision="fp64", restart=1, space="dst")
    a.set_steps(taus)
    for terms in (1, 2, 3):
        want = precond.neumann_inverse(S, X, terms, transpose=transpose)
        got = to_host(a.neumann_apply(to_dev(torch, X), terms, transpose=transpose))
        assert rel_max(got, want) <= 1e-10, terms
    a.set_steps(None)
    S0 = oracle_system("heat", n, ell)
    want = precond.circulant_inverse(S0, X, transpose=transpose)
    a.set_precision("fp32_refined")
    got = to_host(a.precond_apply(to_dev(torch, X), transpose=transpose))
    t = fp32_tol(n, ell)
    assert rel_max(got, want) <= 32 * t * t + 4 * kappa(S0) * U64
    a.set_precision("fp32")
    z0 = to_host(a.precond_apply(to_dev(torch, X), transpose=transpose))
    d = np.linalg.norm(z0 - got) / np.linalg.norm(got)
    assert backward_error(S0, X, got, transpose) <= refined_bw_tol(n, ell, d)


@pytest.mark.parametrize("kind", ["heat", "wave_bd2"])
@pytest.mark.parametrize("prec", ["fp64", "fp32_refined", "fp32"])
def test_dst_solve_matches_time_stepping(kind, prec):
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
    a = AllAtOnce(n, ell, 1.0 / ell, equation=kind, precision=prec, restart=40, space="dst")
    x, info = a.solve(to_dev(torch, B), restart=40, rtol=1e-10)
    assert info["relres_true"] <= 1e-10
    assert rel_max(to_host(x), want) <= 1e-8


def test_dst_full_size_heat():
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n, ell = 4095, 4096
    S = oracle_system("heat", n, ell)
    X = rand_block(n, ell, 12)
    a = AllAtOnce(n, ell, 1.0 / ell, precision="fp32", restart=30, space="dst")
    for tr in (False, True):
        Y = to_host(a.precond_apply(to_dev(torch, X), transpose=tr))
        assert rel_max(Y, precond.circulant_inverse_spectral(S, X, transpose=tr)) <= fp32_tol(n, ell)
    b = a.build_rhs(to_dev(torch, syn.heat_initial(n, modes=8)))
    for prec in ("fp32_refined", "fp32"):
        a.set_precision(prec)
        x, info = a.solve(b, rtol=1e-10)
        assert info["relres_true"] <= 1e-10
        assert info["iters"] <= (3 if prec == "fp32_refined" else 6)


def test_dst_unsupported_shapes_and_switching_back():
    torch = need_gpu()
    from paper_1810_00615_gb300 import AAOError, AllAtOnce
    for n in (14, 100, 8191, 7):
        a = AllAtOnce(n, 16, 1.0 / 16, restart=1)
        with pytest.raises(AAOError):
            a.set_space_solver("dst")
    n, ell = 31, 32
    X = rand_block(n, ell, 2)
    a = AllAtOnce(n, ell, 1.0 / ell, precision="fp64", restart=1, space="dst")
    y_dst = to_host(a.precond_apply(to_dev(torch, X)))
    a.set_space_solver("tridiag")
    y_tri = to_host(a.precond_apply(to_dev(torch, X)))
    assert rel_max(y_dst, y_tri) <= 1e-12
    # kappa changes after the switch reach the DST tables
    a.set_space_solver("dst")
    a.set_kappa(0.3)
    want = precond.circulant_inverse(oracle_system("heat", n, ell, kappa=0.3), X)
    assert rel_max(to_host(a.precond_apply(to_dev(torch, X))), want) <= 1e-10
