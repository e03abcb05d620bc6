"""Shared helpers for the GPU parity tests (inputs come from `synthetic`,
expected values from `oracle`; nothing here computes the method)."""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import precond, system

EQ = {"heat": 0, "wave_bd2": 1, "heat_literal": 2, "wave_bd4": 3}
U32 = 2.0 ** -24   # unit roundoff, FP32
U64 = 2.0 ** -53   # unit roundoff, FP64


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def oracle_system(kind, n, ell, tau=None, kappa=1.0, taus=None):
    tau = 1.0 / ell if tau is None else tau
    if taus is not None:
        return system.heat_steps(n, taus, kappa, tau)
    if kind == "heat":
        return system.heat(n, ell, tau, kappa)
    if kind == "heat_literal":
        return system.heat(n, ell, tau, literal=True)
    if kind == "wave_bd4":
        return system.bd4(n, ell, tau)
    return system.bd2(n, ell, tau)


def rel_max(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))


def to_dev(torch, X):
    return torch.from_numpy(np.ascontiguousarray(X, dtype=np.float64)).cuda()


def to_host(t):
    return t.detach().cpu().numpy()


def rand_block(n, ell, seed):
    return syn.block_vector(n, ell, syn.rng(seed))


# ------------------------------------------------------------ tolerances
def fp32_tol(n, ell):
    """Element-wise (max-norm relative) FP32 bound for the heat circulant,
    whose frequency blocks are shifted Laplacians with a non-negative row
    excess: input rounding, the FFT both ways (log2 ell roundings each), the
    chunk Thomas (16 steps) and the separator levels (log2 n)."""
    return 4 * (2 * math.log2(max(ell, 2)) + 16 + 2 * math.log2(max(n, 2)) + 8) * U32


def kappa(S, transpose=False):
    """2-norm condition number of the block circulant: it is normal (its
    blocks are polynomials in one symmetric tridiagonal Toeplitz matrix and
    the cyclic shift), so kappa = max|lam| / min|lam| over its sine (x)
    Fourier symbols (Section 3)."""
    lam = np.abs(precond.sine_fourier_symbols(S, transpose))
    return float(lam.max() / lam.min())


def circulant_norm(S):
    """||P||_2 = max |lam| over the sine (x) Fourier symbols (P normal)."""
    return float(np.abs(precond.sine_fourier_symbols(S)).max())


def backward_error(S, X, Y, transpose=False):
    """Normwise backward error of Y as a solution of P Y = X (or P^T Y = X):
    eta = ||P Y - X|| / (||P|| ||Y|| + ||X||), with P applied from its
    definition by the oracle (Section 2).  Unlike the forward error it does
    not grow with the condition number: a backward-stable apply gives eta of
    a few unit roundoffs however close to singular P is."""
    R = precond.circulant_matvec(S, Y, transpose=transpose) - X
    return float(np.linalg.norm(R) /
                 (circulant_norm(S) * np.linalg.norm(Y) + np.linalg.norm(X)))


def bw_tol(n, ell, u):
    """Backward-error bound of one apply in unit roundoff u: the time FFT
    forward and back (a few roundings per radix pass: log2 ell each way),
    the per-frequency elimination (a few roundings per unknown and per
    separator level: log2(n+1) in all) and the rounding of input and output,
    with a factor 2 of margin: 2 (log2 ell + log2(n+1) + 4) u."""
    return 2 * (math.log2(max(ell, 2)) + math.log2(n + 1) + 4) * u


def refined_bw_tol(n, ell, rel_correction):
    """Backward-error bound of the refined FP32 apply z = z0 - d,
    d = P32^{-1} r, r = P z0 - x formed in compensated FP32.  Its residual is
    P z - x = -dr + dP d: dr is the rounding of r (2^-24 of r plus a few
    2^-41 of the terms |P||z0| + |x|, and || |P| || <= 4 ||P|| here), dP the
    backward error of the FP32 apply of the correction.  Hence
    eta <= bw_tol32 ||d|| / ||z|| + 2^-24 bw_tol32 + 2^-36, where
    rel_correction = ||d|| / ||z|| is measured from the same inputs (d is
    the plain FP32 apply minus the refined one).  A refinement that adds the
    correction with the wrong sign, or forms r from the wrong operator,
    leaves eta at the FP32 level and fails."""
    t = bw_tol(n, ell, U32)
    return t * rel_correction + U32 * t + 2.0 ** -36
