"""The multithreaded CPU baseline (oracle/cbaseline.c) against the plain
oracle on small heat systems: its matvec is the oracle's block matvec, its
FFT + Thomas circulant solve is the oracle's dense-DFT + banded-LU one (and
inverts the oracle's circulant product), and its GMRES reproduces time
stepping.  Also the child-process entry that bench.py times."""
import shutil

import numpy as np
import pytest

import synthetic as syn
from oracle import precond, system

pytestmark = pytest.mark.skipif(shutil.which("gcc") is None and shutil.which("cc") is None,
                                reason="needs a C compiler")

SHAPES = [(63, 64), (37, 32), (1, 8), (5, 1), (100, 16), (17, 2)]


@pytest.fixture(scope="module")
def cb():
    from oracle import cbaseline
    cbaseline.build()
    return cbaseline


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("n,ell", SHAPES)
@pytest.mark.parametrize("kappa", [1.0, 0.37])
def test_matvec_is_the_oracle_block_matvec(cb, n, ell, kappa):
    S = system.heat(n, ell, 1.0 / ell, kappa=kappa)
    X = syn.block_vector(n, ell, syn.rng(n + ell))
    assert _rel(cb.heat_matvec(n, ell, 1.0 / ell, X, kappa=kappa), system.matvec(S, X)) <= 1e-14


@pytest.mark.parametrize("n,ell", SHAPES)
def test_circulant_solve_is_the_oracle_one(cb, n, ell):
    S = system.heat(n, ell, 1.0 / ell)
    X = syn.block_vector(n, ell, syn.rng(2 * n + ell))
    Y = cb.heat_precond(n, ell, 1.0 / ell, X)
    assert _rel(Y, precond.circulant_inverse(S, X)) <= 1e-12
    # and it inverts the circulant block product P
    assert _rel(precond.circulant_matvec(S, Y), X) <= 1e-12


@pytest.mark.parametrize("n,ell", [(63, 64), (100, 16), (31, 128)])
def test_gmres_reproduces_time_stepping(cb, n, ell):
    S = system.heat(n, ell, 1.0 / ell)
    B = system.rhs_heat(S, syn.heat_initial(n, modes=8))
    U = system.forward_substitution(S, B)
    X, it, rel, ok = cb.heat_fgmres(n, ell, 1.0 / ell, B, restart=30, rtol=1e-10)
    assert ok and rel <= 1e-10
    assert _rel(X, U) <= 1e-8
    # with the exact circulant, P^{-1} A has eigenvalues 1 and 1/(1 - rho_j^ell):
    # two iterations
    assert it <= 2
    # a nonzero initial guess reaches the same solution
    X2, _, rel2, ok2 = cb.heat_fgmres(n, ell, 1.0 / ell, B, X0=0.5 * U, restart=30, rtol=1e-10)
    assert ok2 and rel2 <= 1e-10 and _rel(X2, U) <= 1e-8


def test_rejects_bad_arguments(cb):
    X = np.zeros((12, 5))
    with pytest.raises(RuntimeError):
        cb.heat_precond(5, 12, 1.0 / 12, X)          # ell not a power of two
    with pytest.raises(RuntimeError):
        cb.heat_fgmres(5, 8, 1.0 / 8, np.ones((8, 5)), restart=0)


def test_bench_child_process_entry(monkeypatch):
    import bench
    monkeypatch.setattr(bench, "N_SPACE", 63)
    monkeypatch.setattr(bench, "ELL", 64)
    got = bench._cpu_references()
    assert "error" not in got, got
    fs, fg = got["forward_substitution"], got["cpu_fgmres"]
    assert fs["value"] > 0 and fs["cores"] == 1
    assert fg["converged"] and fg["iters"] == 2 and fg["relres_true"] <= 1e-10
    assert fg["rel_err_vs_time_stepping"] <= 1e-8 and fg["cores"] >= 1
