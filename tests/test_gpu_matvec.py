"""Parity of the FP64 all-at-once matvec and right-hand side (Section 2) with
the oracle.  Both sides are FP64 sums of a handful of products; the GPU
evaluates the same operator in a different order (differences of
neighbours), so the agreement is a few ulps of the largest term: the
tolerance 1e-13 relative to max|y| allows ~500 ulps."""
import numpy as np
import pytest

import synthetic as syn
from oracle import system
from tests._helpers import need_gpu, oracle_system, rand_block, rel_max, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,ell", [(1, 1), (2, 3), (5, 7), (33, 16), (255, 64), (1000, 9)])
@pytest.mark.parametrize("kind", ["heat", "wave_bd2", "heat_literal", "steps", "wave_bd4"])
@pytest.mark.parametrize("transpose", [False, True])
def test_matvec_matches_oracle(n, ell, kind, transpose):
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    m = ell
    for p in (2, 3, 5):
        while m % p == 0:
            m //= p
    if m != 1:
        pytest.skip("contexts need ell = 2^a 3^b 5^c")
    taus = syn.time_steps(ell, 0.6, syn.rng(ell)) if kind == "steps" else None
    S = oracle_system("heat" if kind == "steps" else kind, n, ell, kappa=1.0, taus=taus)
    X = rand_block(n, ell, 3 + n)
    want = system.matvec_T(S, X) if transpose else system.matvec(S, X)
    a = AllAtOnce(n, ell, 1.0 / ell, equation="heat" if kind == "steps" else kind, restart=1)
    if taus is not None:
        a.set_steps(taus)
    got = to_host(a.matvec(to_dev(torch, X), transpose=transpose))
    assert rel_max(got, want) <= 1e-13


@pytest.mark.parametrize("ell", [1, 2, 8, 64])
def test_matvec_kappa(ell):
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n = 40
    S = oracle_system("heat", n, ell, kappa=2.5)
    X = rand_block(n, ell, 4)
    a = AllAtOnce(n, ell, 1.0 / ell, kappa=2.5, restart=1)
    assert rel_max(to_host(a.matvec(to_dev(torch, X))), system.matvec(S, X)) <= 1e-13


def test_matvec_full_size():
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n, ell = 4095, 4096
    S = oracle_system("heat", n, ell)
    X = rand_block(n, ell, 5)
    a = AllAtOnce(n, ell, 1.0 / ell, restart=1)
    got = to_host(a.matvec(to_dev(torch, X)))
    assert rel_max(got, system.matvec(S, X)) <= 1e-13
    got = to_host(a.matvec(to_dev(torch, X), transpose=True))
    assert rel_max(got, system.matvec_T(S, X)) <= 1e-13


@pytest.mark.parametrize("kind", ["heat", "wave_bd2", "heat_literal", "wave_bd4"])
@pytest.mark.parametrize("with_v0", [False, True])
@pytest.mark.parametrize("ell", [1, 2, 4, 16])
def test_rhs_matches_oracle(kind, with_v0, ell):
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    if with_v0 and not kind.startswith("wave"):
        pytest.skip("initial velocity is a wave input")
    n = 63
    S = oracle_system(kind, n, ell)
    u0, v0 = syn.wave_initial(n, modes=16)
    a = AllAtOnce(n, ell, 1.0 / ell, equation=kind, restart=1)
    if kind == "wave_bd2":
        want = system.rhs_bd2(S, u0, v0 if with_v0 else None)
    elif kind == "wave_bd4":
        want = system.rhs_bd4(S, u0, v0 if with_v0 else None)
    else:
        want = system.rhs_heat(S, u0)
    got = to_host(a.build_rhs(to_dev(torch, u0), to_dev(torch, v0) if with_v0 else None))
    assert rel_max(got, want) <= 1e-13


@pytest.mark.parametrize("kind", ["heat", "wave_bd2", "wave_bd4", "heat_literal", "steps"])
@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("n,ell", [(1, 1), (33, 16), (255, 64), (70, 3)])
def test_residual_and_fused_norm(kind, transpose, n, ell):
    """aao_residual: r = A x - b and ||r||^2 from the same pass, against the
    oracle's A x - b and numpy's norm of it."""
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    taus = syn.time_steps(ell, 0.6, syn.rng(ell)) if kind == "steps" else None
    S = oracle_system("heat" if kind == "steps" else kind, n, ell, kappa=1.0, taus=taus)
    a = AllAtOnce(n, ell, 1.0 / ell, equation="heat" if kind == "steps" else kind, restart=1)
    if taus is not None:
        a.set_steps(taus)
    X = rand_block(n, ell, 5 + n)
    B = rand_block(n, ell, 6 + n)
    want = (system.matvec_T(S, X) if transpose else system.matvec(S, X)) - B
    r, nrm2 = a.residual(to_dev(torch, X), to_dev(torch, B), transpose=transpose)
    assert rel_max(to_host(r), want) <= 1e-13
    ref = float(np.sum(want * want))
    assert abs(nrm2 - ref) <= 1e-12 * ref


@pytest.mark.parametrize("kind", ["heat", "wave_bd2", "wave_bd4", "steps"])
@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("with_v0", [False, True])
def test_matvec_dots(kind, transpose, with_v0):
    """aao_matvec_dots: w = A x - v with [v0 . w,] v . w, w . w from the same
    pass, against the oracle's A x - v and numpy's dots of it."""
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    n, ell = 130, 64
    taus = syn.time_steps(ell, 0.6, syn.rng(ell)) if kind == "steps" else None
    S = oracle_system("heat" if kind == "steps" else kind, n, ell, kappa=1.0, taus=taus)
    a = AllAtOnce(n, ell, 1.0 / ell, equation="heat" if kind == "steps" else kind, restart=1)
    if taus is not None:
        a.set_steps(taus)
    X, V, V0 = rand_block(n, ell, 21), rand_block(n, ell, 22), rand_block(n, ell, 23)
    want = (system.matvec_T(S, X) if transpose else system.matvec(S, X)) - V
    w, d = a.matvec_dots(to_dev(torch, X), to_dev(torch, V),
                         to_dev(torch, V0) if with_v0 else None, transpose=transpose)
    assert rel_max(to_host(w), want) <= 1e-13
    ref = ([float(np.sum(V0 * want))] if with_v0 else []) + [float(np.sum(V * want)),
                                                              float(np.sum(want * want))]
    scale = float(np.sqrt(np.sum(want * want)) * max(np.sqrt(np.sum(V * V)), np.sqrt(np.sum(V0 * V0))))
    for got, r in zip(d, ref):
        assert abs(got - r) <= 1e-12 * max(scale, abs(r))
