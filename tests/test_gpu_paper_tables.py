"""The paper's own Table 1 and Table 2 problems (ell = 768 and 1440 run the
mixed-radix time FFTs, ell = 1024 the radix-16 ones): heat equation,
u0 = x(1 - x), GMRES tolerance 1e-5 as in the captions.  The paper preconditions on the left; this solver is
right-preconditioned flexible GMRES stopping on the true residual (which
needs fewer iterations at 1e-5: measured 1 for Table 1's 2, and 1-3 fewer
in Table 2), and Table 2's time grids come from the paper's own random
draws, so the counts are held to at most the printed ones plus one, with the
trend the paper reports: more Neumann terms never cost iterations."""
import json
import os

import numpy as np
import pytest

import synthetic as syn
from tests._helpers import need_gpu

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_iteration_counts.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def _rhs(torch, n, ell):
    B = np.zeros((ell, n))
    B[0] = syn.parabola_load(n)
    return torch.from_numpy(B).cuda()


@pytest.mark.parametrize("prec", ["fp64", "fp32_refined"])
def test_table1_uniform_steps_two_iterations(prec):
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    for n, ell, want in _golden()["heat_uniform_x1mx"]["cases"]:
        a = AllAtOnce(n, ell, 1.0 / ell, precision=prec, restart=30)
        _, info = a.solve(_rhs(torch, n, ell), rtol=1e-5)
        assert info["relres_true"] <= 1e-5
        assert abs(info["iters"] - want) <= 1, (n, info["iters"])


@pytest.mark.parametrize("table", ["neumann_table2_abc", "neumann_table2_def"])
def test_table2_neumann_counts(table):
    torch = need_gpu()
    from paper_1810_00615_gb300 import AllAtOnce
    for n, ell, delta, want in _golden()[table]["cases"]:
        a = AllAtOnce(n, ell, 1.0 / ell, precision="fp64", restart=30)
        a.set_steps(syn.time_steps(ell, delta, syn.rng(7)))
        b = _rhs(torch, n, ell)
        got = []
        for terms in (1, 2, 3):
            _, info = a.solve(b, rtol=1e-5, precond=terms)
            assert info["relres_true"] <= 1e-5
            got.append(info["iters"])
        # the paper's trend: more Neumann terms never cost iterations, and on
        # the rougher grids they save some
        assert got[0] >= got[1] >= got[2], (n, delta, got)
        if delta >= 0.5:
            assert got[2] < got[0], (n, delta, got)
        # right preconditioning with a true-residual stop needs at most the
        # left-preconditioned counts the paper prints (plus one)
        for g, w in zip(got, want):
            assert 1 <= g <= w + 1, (n, delta, got, want)
