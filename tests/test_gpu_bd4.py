"""The BD4 wave system C_BD4 and its preconditioner R_BD4 (Section 2) on the
GPU against the oracle: solves by FGMRES with R_BD4 reproduce time stepping
(forward substitution through the BD2 start-up rows), the adjoint solve
reproduces backward substitution, and the iteration counts follow Section 4
(Table 3): with the non-smooth bump BD4 needs several times the BD2
iterations, with the smooth sin(2 pi x) about two.

R_BD4 is far worse conditioned than R_BD2 (its symbol (1 - w)^2 (2 - w) m +
tau^2 k nearly vanishes where the angle of w is about tau sqrt(k/m): the
imaginary part of the M factor cancels to third order), so these solves need
long restarts and many iterations even in FP64."""
import numpy as np
import pytest

import synthetic as syn
from oracle import fem, system
from tests._helpers import need_gpu, oracle_system, rel_max, to_dev, to_host

pytestmark = pytest.mark.gpu


def _bump_rhs(S, n):
    return system.rhs_bd4(S, syn.wave_nonsmooth(n))


@pytest.mark.parametrize("prec", ["fp64", "fp32_refined", "fp32"])
def test_bd4_solve_matches_time_stepping(prec):
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n, ell = 63, 64
    S = oracle_system("wave_bd4", n, ell)
    u0, v0 = syn.wave_initial(n, modes=16)
    B = system.rhs_bd4(S, u0, v0)
    want = system.forward_substitution(S, B)
    a = AllAtOnce(n, ell, 1.0 / ell, equation="wave_bd4", precision=prec, restart=40)
    # the right-hand side built on the GPU is the oracle's
    b = a.build_rhs(to_dev(torch, u0), to_dev(torch, v0))
    assert rel_max(to_host(b), B) <= 1e-13
    x, info = a.solve(b, restart=40, rtol=1e-10, maxit=2000)
    assert info["relres_true"] <= 1e-10
    assert rel_max(to_host(x), want) <= 1e-7
    assert info["iters"] <= 200


@pytest.mark.parametrize("n,ell", [(255, 256), (511, 512)])
def test_bd4_bump_tolerance_1e5(n, ell):
    """The paper's Table 3 setting (non-smooth bump, tolerance 1e-5) at
    larger sizes, FP64 R_BD4, GMRES(60)."""
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    S = oracle_system("wave_bd4", n, ell)
    B = _bump_rhs(S, n)
    want = system.forward_substitution(S, B)
    a = AllAtOnce(n, ell, 1.0 / ell, equation="wave_bd4", precision="fp64", restart=60)
    x, info = a.solve(to_dev(torch, B), restart=60, rtol=1e-5, maxit=3000)
    assert info["relres_true"] <= 1e-5
    # the solution error is bounded by cond(C_BD4) times the residual; 1e-5
    # residuals measured here gave errors up to 5e-4
    assert rel_max(to_host(x), want) <= 5e-3


def test_bd4_adjoint_matches_backward_substitution():
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n, ell = 63, 64
    S = oracle_system("wave_bd4", n, ell)
    G = syn.block_vector(n, ell, syn.rng(41))
    want = system.backward_substitution(S, G)
    a = AllAtOnce(n, ell, 1.0 / ell, equation="wave_bd4", precision="fp64", restart=40)
    lam, info = a.adjoint_solve(to_dev(torch, G), restart=40, rtol=1e-10, maxit=2000)
    assert info["relres_true"] <= 1e-10
    assert rel_max(to_host(lam), want) <= 1e-7


@pytest.mark.parametrize("n,ell", [(32, 32), (64, 64), (96, 96), (32, 96)])
def test_table3_bd4_versus_bd2_counts(n, ell):
    """Section 4: with the non-smooth bump BD4 takes many more iterations
    than BD2 (the oracle: about three times as many; at least twice is
    held), and with sin(2 pi x) both take about two (at most three here).
    The printed BD4 counts (60 to 200) are reproduced by no GMRES variant
    of the oracle, so only this comparison is checked."""
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    counts = {}
    for kind in ("wave_bd2", "wave_bd4"):
        S = oracle_system(kind, n, ell)
        rhs = system.rhs_bd2 if kind == "wave_bd2" else system.rhs_bd4
        a = AllAtOnce(n, ell, 1.0 / ell, equation=kind, precision="fp64", restart=50)
        for name, u0 in (("bump", fem.l2_projection(
                lambda x: np.where((x > 3 / 8) & (x < 5 / 8), np.cos(4 * np.pi * (x - 0.5)) ** 2, 0.0), n)),
                ("smooth", fem.l2_projection(lambda x: np.sin(2 * np.pi * x), n))):
            B = rhs(S, u0)
            x, info = a.solve(to_dev(torch, B), restart=50, rtol=1e-5, maxit=1000)
            assert info["relres_true"] <= 1e-5
            counts[kind, name] = info["iters"]
    assert counts["wave_bd4", "smooth"] <= 3
    assert counts["wave_bd2", "smooth"] <= 3
    assert counts["wave_bd4", "bump"] >= 2 * counts["wave_bd2", "bump"], counts


def test_bd4_rejects_variable_steps():
    torch = need_gpu()
    from paper_1810_00615_gb300 import AAOError, AllAtOnce
    a = AllAtOnce(15, 16, 1.0 / 16, equation="wave_bd4", restart=1)
    with pytest.raises(AAOError):
        a.set_steps(syn.time_steps(16, 0.5, syn.rng(1)))


@pytest.mark.parametrize("ell", [1, 2, 3, 5])
def test_bd4_tiny_ell(ell):
    """ell below the four-step stencil: the system is the BD2 start-up rows
    (and the first four-step row), the circulant wraps over fewer blocks."""
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    from oracle import precond
    n = 17
    S = oracle_system("wave_bd4", n, ell)
    X = syn.block_vector(n, ell, syn.rng(ell))
    a = AllAtOnce(n, ell, 1.0 / ell, equation="wave_bd4", precision="fp64", restart=10)
    for tr in (False, True):
        f = system.matvec_T if tr else system.matvec
        assert rel_max(to_host(a.matvec(to_dev(torch, X), transpose=tr)), f(S, X)) <= 1e-13
        want = precond.circulant_inverse(S, X, transpose=tr)
        assert rel_max(to_host(a.precond_apply(to_dev(torch, X), transpose=tr)), want) <= 1e-10
    B = system.rhs_bd4(S, syn.wave_nonsmooth(n))
    x, info = a.solve(to_dev(torch, B), restart=10, rtol=1e-12, maxit=200)
    assert rel_max(to_host(x), system.forward_substitution(S, B)) <= 1e-9


@pytest.mark.parametrize("prec", ["fp64", "fp32_refined", "fp32"])
def test_bd4_long_cycles_stay_finite(prec):
    """n = 1023, ell = 1024, GMRES(100): R_BD4's condition number (~1e11)
    makes the Hessenberg subdiagonals large, and over a long cycle the stored
    Arnoldi vectors' norms would leave the FP64 squared-norm range and the
    FP32 range without the solver's renormalisation.  FP64 and refined FP32
    reach 1e-5 (measured: 99 and 181 iterations); plain FP32, whose
    elimination error is kappa_k 2^-24 >> 1 on the near-singular frequency
    blocks, is only required to stay finite and make progress."""
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n, ell = 1023, 1024
    S = oracle_system("wave_bd4", n, ell)
    B = _bump_rhs(S, n)
    a = AllAtOnce(n, ell, 1.0 / ell, equation="wave_bd4", precision=prec, restart=100)
    if prec == "fp32":
        x, info = a.solve(to_dev(torch, B), restart=100, rtol=1e-5, maxit=300)
        assert np.isfinite(info["relres_true"]) and info["relres_true"] < 0.1
        assert np.all(np.isfinite(to_host(x)))
        return
    want = system.forward_substitution(S, B)
    x, info = a.solve(to_dev(torch, B), restart=100, rtol=1e-5, maxit=1000)
    assert info["relres_true"] <= 1e-5
    assert rel_max(to_host(x), want) <= 5e-2
