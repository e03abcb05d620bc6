"""Parity of the matvec of an FP32 vector (aao_matvec_f32, the product the
mixed solver forms with its FP32 preconditioned basis) with the oracle's
A x (Section 2) on the same FP32 values.

The heat and BD2 forms are evaluated in 64-bit fixed point per warp tile and
rounded once to FP64, so besides the max-relative parity used for the FP64
matvec, every element is held to a few FP64 roundings of sum_j |A_ij| |x_j|
against an extended-precision product of the oracle's matrices."""
import numpy as np
import pytest

import synthetic as syn
from oracle import system
from tests._helpers import need_gpu, oracle_system, rand_block, rel_max, to_host

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53


def _f32_dev(torch, X):
    return torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()


def _abs_system(S):
    """|A| as a block system of entrywise absolute values."""
    T = system.BlockSystem.__new__(system.BlockSystem)
    T.__dict__.update(S.__dict__)
    T.diag = [abs(D) for D in S.diag]
    T.lower = [abs(L) for L in S.lower]
    return T


def _context(kind, n, ell):
    from paper_1810_00615_gb300 import AllAtOnce
    taus = syn.time_steps(ell, 0.6, syn.rng(ell)) if kind == "steps" else None
    S = oracle_system("heat" if kind == "steps" else kind, n, ell, kappa=1.0, taus=taus)
    a = AllAtOnce(n, ell, 1.0 / ell, equation="heat" if kind == "steps" else kind, restart=1,
                  precision="fp32")
    if taus is not None:
        a.set_steps(taus)
    return S, a


def _exact(S, X, transpose):
    """A x with the oracle's FP64 matrix entries, summed in long double."""
    Xl = X.astype(np.longdouble)

    def apply(Mat, v):
        Mat = Mat.tocsr()
        out = np.zeros(Mat.shape[0], dtype=np.longdouble)
        for r in range(Mat.shape[0]):
            lo, hi = Mat.indptr[r], Mat.indptr[r + 1]
            out[r] = np.sum(Mat.data[lo:hi].astype(np.longdouble) * v[Mat.indices[lo:hi]])
        return out

    Y = np.zeros_like(Xl)
    for t in range(S.ell):
        y = apply(S.diag[t].T if transpose else S.diag[t], Xl[t])
        for j, Aj in enumerate(S.lower, start=1):
            s = t + j if transpose else t - j
            if 0 <= s < S.ell:
                y = y + apply(Aj.T if transpose else Aj, Xl[s])
        Y[t] = y
    return Y


@pytest.mark.parametrize("n,ell", [(1, 1), (2, 2), (5, 8), (33, 16), (65, 64), (255, 128),
                                   (1000, 32)])
@pytest.mark.parametrize("kind", ["heat", "wave_bd2", "heat_literal", "steps"])
@pytest.mark.parametrize("transpose", [False, True])
def test_matvec_f32_matches_oracle(n, ell, kind, transpose):
    torch = need_gpu()
    S, a = _context(kind, n, ell)
    X = rand_block(n, ell, 11 + n).astype(np.float32).astype(np.float64)
    want = system.matvec_T(S, X) if transpose else system.matvec(S, X)
    got = to_host(a.matvec_f32(_f32_dev(torch, X), transpose=transpose))
    assert rel_max(got, want) <= 1e-13
    # the FP64 entry point on the same values agrees as closely
    fp64 = to_host(a.matvec(torch.from_numpy(X).cuda(), transpose=transpose))
    assert rel_max(got, fp64) <= 1e-13


@pytest.mark.parametrize("kind", ["heat", "wave_bd2", "steps"])
@pytest.mark.parametrize("transpose", [False, True])
def test_matvec_f32_elementwise_rounding_bound(kind, transpose):
    """A near-cancelling input (the FP32-rounded time-stepping solution) and a
    random one: |y - A x| <= 8 eps (|A| |x|) in every element."""
    torch = need_gpu()
    n, ell = 70, 64
    S, a = _context(kind, n, ell)
    if kind == "wave_bd2":
        u0, v0 = syn.wave_initial(n, modes=16)
        B = system.rhs_bd2(S, u0, v0)
    else:
        B = system.rhs_heat(S, syn.heat_initial(n, modes=8))
    U = system.forward_substitution(S, B)
    for X in (U, rand_block(n, ell, 77)):
        X = X.astype(np.float32).astype(np.float64)
        got = to_host(a.matvec_f32(_f32_dev(torch, X), transpose=transpose)).astype(np.longdouble)
        exact = _exact(S, X, transpose)
        absS = _abs_system(S)
        mag = (system.matvec_T if transpose else system.matvec)(absS, np.abs(X))
        err = np.abs(got - exact).astype(np.float64)
        assert np.all(err <= 8 * EPS * mag + 1e-300)


def test_matvec_f32_wide_dynamic_range_in_a_tile():
    """Values spanning 2^0 .. 2^-70 inside one 32 x 32 tile: the small ones are
    truncated at 2^-57 of the tile maximum, far below an FP64 rounding of it."""
    torch = need_gpu()
    n, ell = 64, 32
    S, a = _context("heat", n, ell)
    r = syn.rng(5)
    X = r.standard_normal((ell, n)) * np.exp2(-r.integers(0, 71, size=(ell, n)))
    X = X.astype(np.float32).astype(np.float64)
    got = to_host(a.matvec_f32(_f32_dev(torch, X))).astype(np.longdouble)
    exact = _exact(S, X, False)
    scale = np.max(np.abs(system.matvec(_abs_system(S), np.abs(X))))
    assert float(np.max(np.abs(got - exact))) <= 8 * EPS * scale


def test_matvec_f32_zero_and_nonfinite():
    torch = need_gpu()
    n, ell = 100, 64
    S, a = _context("heat", n, ell)
    X = np.zeros((ell, n))
    assert np.all(to_host(a.matvec_f32(_f32_dev(torch, X))) == 0.0)
    for bad in (np.nan, np.inf):
        X = rand_block(n, ell, 8)
        X[40, 50] = bad                 # tile: columns 32..63, steps 32..63
        got = to_host(a.matvec_f32(_f32_dev(torch, X)))
        assert np.isnan(got[40, 50])
        assert np.all(np.isfinite(got[:32]))          # earlier steps untouched
        assert np.all(np.isfinite(got[:, :32]))       # other column tiles untouched


def test_matvec_f32_full_size():
    torch = need_gpu()
    n, ell = 4095, 4096
    S, a = _context("heat", n, ell)
    X = rand_block(n, ell, 5).astype(np.float32).astype(np.float64)
    Xd = _f32_dev(torch, X)
    for tr in (False, True):
        got = to_host(a.matvec_f32(Xd, transpose=tr))
        want = system.matvec_T(S, X) if tr else system.matvec(S, X)
        assert rel_max(got, want) <= 1e-13
