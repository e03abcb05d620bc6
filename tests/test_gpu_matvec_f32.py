"""Parity of the fixed-point matvec with the oracle's A x (Section 2): for an
FP32 vector (aao_matvec_f32, the product the mixed solver forms with its FP32
preconditioned basis) and for an FP64 one (aao_matvec, heat and BD2 forms).

Both evaluate the stencil sums in 64-bit fixed point per warp tile and round
them once to FP64, so besides the max-relative parity, every element is held
to a few FP64 roundings of sum_j |A_ij| |x_j| against an extended-precision
product of the oracle's matrices."""
import numpy as np
import pytest

import synthetic as syn
from oracle import system
from tests._helpers import need_gpu, oracle_system, rand_block, rel_max, to_host

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53


def _f32_dev(torch, X):
    return torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()


def _apply(torch, a, X, dtype, transpose=False):
    """The GPU product of X (already representable in dtype) in FP64."""
    if dtype == "f32":
        return to_host(a.matvec_f32(_f32_dev(torch, X), transpose=transpose))
    return to_host(a.matvec(torch.from_numpy(np.ascontiguousarray(X)).cuda(), transpose=transpose))


def _rounded(X, dtype):
    return X.astype(np.float32).astype(np.float64) if dtype == "f32" else X


def _abs_system(S):
    """|A| as a block system of entrywise absolute values."""
    T = system.BlockSystem.__new__(system.BlockSystem)
    T.__dict__.update(S.__dict__)
    T.diag = [abs(D) for D in S.diag]
    T.lower = [abs(L) for L in S.lower]
    T.startup = {k: abs(B) for k, B in S.startup.items()}
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


def _tile_max(X, lags=2):
    """For each output (t, i): max |x| over the fixed-point tile that forms it
    (its 32 columns with one halo column each side, its 32 steps with the
    lag steps on either side: two, three for BD4)."""
    ell, n = X.shape
    A = np.abs(X)
    T = np.zeros_like(A)
    for t0 in range(0, ell, 32):
        for i0 in range(0, n, 32):
            blk = A[max(0, t0 - lags):min(ell, t0 + 32 + lags), max(0, i0 - 1):min(n, i0 + 33)]
            T[t0:t0 + 32, i0:i0 + 32] = blk.max()
    return T


def _bound(S, X, transpose):
    """8 FP64 roundings of (|A| |x|)_i plus the documented truncation: inputs
    far below their tile maximum enter with an absolute error under 2^-57 of
    it (2^-55 for BD4, whose fixed point keeps two guard bits; here twice
    that for margin), times the row sums of |A|."""
    absS = _abs_system(S)
    f = system.matvec_T if transpose else system.matvec
    mag = f(absS, np.abs(X))
    rows = f(absS, np.ones_like(X))
    bd4 = S.kind == "bd4"
    trunc = 2.0 ** (-54 if bd4 else -56)
    return 8 * EPS * mag + trunc * rows * _tile_max(X, 3 if bd4 else 2)


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
        for j in range(1, len(S.lower) + 1):
            s = t + j if transpose else t - j
            if 0 <= s < S.ell:
                Aj = system.lag_block(S, s if transpose else t, j)
                y = y + apply(Aj.T if transpose else Aj, Xl[s])
        Y[t] = y
    return Y


@pytest.mark.parametrize("n,ell", [(1, 1), (2, 2), (5, 8), (33, 16), (65, 64), (255, 128),
                                   (1000, 32)])
@pytest.mark.parametrize("kind", ["heat", "wave_bd2", "heat_literal", "steps", "wave_bd4"])
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
    # the fused shifted-Arnoldi form y = A x - v, for FP32 and FP64 x
    V = rand_block(n, ell, 29 + n)
    fused = to_host(a.matvec_f32(_f32_dev(torch, X), transpose=transpose,
                                 sub=torch.from_numpy(V).cuda()))
    assert rel_max(fused, want - V) <= 1e-13
    fused64 = to_host(a.matvec(torch.from_numpy(X).cuda(), transpose=transpose,
                               sub=torch.from_numpy(V).cuda()))
    assert rel_max(fused64, want - V) <= 1e-13


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("kind", ["heat", "wave_bd2", "steps", "wave_bd4"])
@pytest.mark.parametrize("transpose", [False, True])
def test_matvec_elementwise_rounding_bound(kind, transpose, dtype):
    """A near-cancelling input (the rounded time-stepping solution) and a
    random one: every element within the documented bound (_bound)."""
    torch = need_gpu()
    n, ell = 70, 64
    S, a = _context(kind, n, ell)
    if kind == "wave_bd2":
        u0, v0 = syn.wave_initial(n, modes=16)
        B = system.rhs_bd2(S, u0, v0)
    elif kind == "wave_bd4":
        u0, v0 = syn.wave_initial(n, modes=16)
        B = system.rhs_bd4(S, u0, v0)
    else:
        B = system.rhs_heat(S, syn.heat_initial(n, modes=8))
    U = system.forward_substitution(S, B)
    for X in (U, rand_block(n, ell, 77)):
        X = _rounded(X, dtype)
        got = _apply(torch, a, X, dtype, transpose).astype(np.longdouble)
        exact = _exact(S, X, transpose)
        err = np.abs(got - exact).astype(np.float64)
        assert np.all(err <= _bound(S, X, transpose) + 1e-300)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_matvec_wide_dynamic_range_in_a_tile(dtype):
    """Values spanning 2^0 .. 2^-70 inside one 32 x 32 tile: the small ones are
    truncated at 2^-57 of the tile maximum, far below an FP64 rounding of it."""
    torch = need_gpu()
    n, ell = 64, 32
    S, a = _context("heat", n, ell)
    r = syn.rng(5)
    X = _rounded(r.standard_normal((ell, n)) * np.exp2(-r.integers(0, 71, size=(ell, n))), dtype)
    got = _apply(torch, a, X, dtype).astype(np.longdouble)
    exact = _exact(S, X, False)
    scale = np.max(np.abs(system.matvec(_abs_system(S), np.abs(X))))
    assert float(np.max(np.abs(got - exact))) <= 8 * EPS * scale


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_matvec_zero_and_nonfinite(dtype):
    torch = need_gpu()
    n, ell = 100, 64
    S, a = _context("heat", n, ell)
    assert np.all(_apply(torch, a, np.zeros((ell, n)), dtype) == 0.0)
    for bad in (np.nan, np.inf):
        X = _rounded(rand_block(n, ell, 8), dtype)
        X[40, 50] = bad                 # tile: columns 32..63, steps 32..63
        got = _apply(torch, a, X, dtype)
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


def _exact_circulant(S, Z, X, transpose, absolute=False):
    """P z - x with the oracle's FP64 blocks, summed in long double (P the
    block circulant: constant-step A0, lags wrapped around in time); with
    absolute, |P| |z| (the size of the terms) instead."""
    from oracle import system as osys
    Zl = np.abs(Z).astype(np.longdouble) if absolute else Z.astype(np.longdouble)
    A0 = osys.constant_A0(S).tocsr()

    def apply(Mat, v):
        out = np.zeros(Mat.shape[0], dtype=np.longdouble)
        for r in range(Mat.shape[0]):
            lo, hi = Mat.indptr[r], Mat.indptr[r + 1]
            d = Mat.data[lo:hi].astype(np.longdouble)
            out[r] = np.sum((np.abs(d) if absolute else d) * v[Mat.indices[lo:hi]])
        return out

    Y = np.zeros_like(Zl)
    for t in range(S.ell):
        y = apply(A0, Zl[t])
        for j, Aj in enumerate(S.lower, start=1):
            src = (t + j) % S.ell if transpose else (t - j) % S.ell
            y = y + apply(Aj.tocsr(), Zl[src])
        Y[t] = y if absolute else y - X[t].astype(np.longdouble)
    return Y


@pytest.mark.parametrize("kind", ["heat", "wave_bd2", "wave_bd4", "heat_literal"])
@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("n,ell", [(1, 1), (5, 3), (70, 64), (33, 2)])
def test_circulant_residual_f32(kind, transpose, n, ell):
    """aao_circulant_residual_f32: r = P z - x for an FP32 z.  With z the FP32
    rounding of P^{-1} x, P z and x cancel to ~1e-7 of their size; the
    fixed-point evaluation keeps r to a few FP64 roundings of the terms
    (the literal form's FP64 stencil to a few hundred)."""
    torch = need_gpu()
    from oracle import precond
    from paper_1810_00615_gb300 import AllAtOnce
    S = oracle_system(kind, n, ell)
    a = AllAtOnce(n, ell, 1.0 / ell, equation=kind, restart=1, precision="fp32")
    X = rand_block(n, ell, 90 + n)
    Z = precond.circulant_inverse(S, X, transpose=transpose).astype(np.float32)
    got = to_host(a.circulant_residual_f32(_f32_dev(torch, Z), torch.from_numpy(X).cuda(),
                                           transpose=transpose)).astype(np.longdouble)
    exact = _exact_circulant(S, Z.astype(np.float64), X, transpose)
    terms = _exact_circulant(S, Z.astype(np.float64), X, transpose, absolute=True)
    scale = float(np.max(terms)) + float(np.max(np.abs(X)))
    tol = (16 if kind == "heat_literal" else 4) * EPS * scale
    assert float(np.max(np.abs(got - exact))) <= tol
    # the residual is the FP32 rounding error of z, far below the terms
    assert float(np.max(np.abs(exact))) <= 1e-3 * scale
