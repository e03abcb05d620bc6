"""Mixed-radix time FFTs (ell = 2^a 3^b 5^c, not a power of two): parity of
the preconditioner applies with the oracle's dense-DFT circulant inverse
(Section 3, any ell), in both precisions, both orientations, the refined
mode and a Neumann term; tolerances as in test_gpu_precond."""
import numpy as np
import pytest

import synthetic as syn
from oracle import precond, system
from tests._helpers import (U32, U64, backward_error, bw_tol, fp32_tol, kappa, need_gpu,
                            oracle_system, rand_block, refined_bw_tol, rel_max, to_dev, to_host)

pytestmark = pytest.mark.gpu

ELEMENTWISE_MAX = 1e-2   # element-wise tolerances at or above this pin nothing


def tol_for(S, kind, prec, n, ell):
    t32 = fp32_tol(n, ell)
    if kind == "wave_bd2":
        t32 = max(t32, kappa(S) * U32)
    if prec == "fp64":
        return max(1e-10, 4 * kappa(S) * U64)
    if prec == "fp32_refined":
        return 32 * t32 * t32 + 4 * kappa(S) * U64
    return t32


LENGTHS = [3, 5, 6, 10, 12, 15, 24, 30, 45, 48, 90, 96, 160, 360, 768, 1440]


@pytest.mark.parametrize("ell", LENGTHS)
@pytest.mark.parametrize("kind", ["heat", "wave_bd2"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_refined"])
@pytest.mark.parametrize("transpose", [False, True])
def test_mixed_radix_precond_matches_oracle(ell, kind, prec, transpose):
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n = 37 if ell <= 360 else 63
    S = oracle_system(kind, n, ell)
    X = rand_block(n, ell, 300 + ell)
    want = precond.circulant_inverse(S, X, transpose=transpose)
    a = AllAtOnce(n, ell, 1.0 / ell, equation=kind, precision=prec, restart=1)
    got = to_host(a.precond_apply(to_dev(torch, X), transpose=transpose))
    tol = tol_for(S, kind, prec, n, ell)
    if tol < ELEMENTWISE_MAX:
        assert rel_max(got, want) <= tol
    eta = backward_error(S, X, got, transpose)
    if prec == "fp32_refined":
        a.set_precision("fp32")
        z0 = to_host(a.precond_apply(to_dev(torch, X), transpose=transpose))
        d = np.linalg.norm(z0 - got) / np.linalg.norm(got)
        assert eta <= refined_bw_tol(n, ell, d)
    else:
        assert eta <= bw_tol(n, ell, U64 if prec == "fp64" else U32)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mixed_radix_neumann(prec):
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n, ell = 47, 96
    taus = syn.time_steps(ell, 0.7, syn.rng(9))
    S = oracle_system("heat", n, ell, taus=taus)
    X = rand_block(n, ell, 10)
    a = AllAtOnce(n, ell, 1.0 / ell, precision=prec, restart=1)
    a.set_steps(taus)
    for terms in (1, 2, 3):
        want = precond.neumann_inverse(S, X, terms)
        got = to_host(a.neumann_apply(to_dev(torch, X), terms))
        tol = 1e-10 if prec == "fp64" else 3 * fp32_tol(n, ell)
        assert rel_max(got, want) <= tol, terms


@pytest.mark.parametrize("ell", [768, 1440])
def test_mixed_radix_solve_matches_time_stepping(ell):
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n = 511
    S = oracle_system("heat", n, ell)
    B = system.rhs_heat(S, syn.heat_initial(n, modes=8))
    want = system.forward_substitution(S, B)
    for prec in ("fp32", "fp32_refined", "fp64"):
        a = AllAtOnce(n, ell, 1.0 / ell, precision=prec, restart=30)
        x, info = a.solve(to_dev(torch, B), rtol=1e-10)
        assert info["relres_true"] <= 1e-10
        assert rel_max(to_host(x), want) <= 1e-8


def test_unsupported_lengths_are_rejected():
    need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce, _capi
    for ell in (7, 14, 4100, 8192):
        with pytest.raises(_capi.AAOError):
            AllAtOnce(15, ell, 1.0 / ell, restart=1)
