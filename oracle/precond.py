"""Block-circulant preconditioners and the Neumann series (Sections 2 and 3).

P (heat), R_BD2 and R_BD4 (wave) are block circulant: P = I (x) A0 +
Sigma (x) A1 (+ Sigma^2 (x) A2 for BD2, + Sigma^3 (x) A3 for BD4), the
Kronecker form of Section 3, with Sigma the ell x ell cyclic
down-shift, (Sigma x)_t = x_{t-1 mod ell} (the paper writes Sigma in
R^{n x n}; its size is ell).  Sigma = U Lambda U^* with U the unitary DFT of
size ell, U_{tk} = exp(+2 pi i t k / ell)/sqrt(ell), and Lambda_kk = w_k =
exp(-2 pi i k/ell) (the printed U has lost the factor 2 and has n for ell).
So the inverse of the diagonalised form in Section 3 reads P^{-1} = (U (x) I)[I (x) A0 + Lambda (x) A1]^{-1}(U^* (x) I).

``circulant_inverse`` applies that formula in the order the paper gives it,
with the dense U (Section 3, "method 1": each block row of (U (x) I) is a
combination of all ell blocks), and a tridiagonal solve per frequency (the
Thomas-algorithm step of Section 3, here LAPACK's banded LU).
"""
from __future__ import annotations

import numpy as np

from .system import BlockSystem, constant_A0, neumann_E, solve_tridiag


def circulant_matvec(S: BlockSystem, X: np.ndarray, transpose: bool = False) -> np.ndarray:
    """Y = P X (or P^T X) from the definition of the block circulant
    (Section 2): (P x)_t = A0 x_t + sum_j A_j x_{(t - j) mod ell}; the
    transpose takes x_{(t + j) mod ell} (all blocks are symmetric)."""
    A0 = constant_A0(S)
    Y = np.empty_like(X, dtype=np.float64)
    for t in range(S.ell):
        y = A0 @ X[t]
        for j, Aj in enumerate(S.lower, start=1):
            src = (t + j) % S.ell if transpose else (t - j) % S.ell
            y = y + Aj @ X[src]
        Y[t] = y
    return Y


def sine_fourier_symbols(S: BlockSystem, transpose: bool = False) -> np.ndarray:
    """lam[k, j-1]: eigenvalue of the circulant on s_j (x) f_k.

    Every block is a constant-coefficient symmetric tridiagonal (Toeplitz)
    matrix tridiag(e, d, e), whose eigenvectors are the sine vectors
    s_j(i) = sin(j pi i h) with eigenvalues d + 2 e cos(j pi h) (textbook);
    the Fourier vectors f_k diagonalise Sigma with eigenvalue w_k (Section
    3).  Block k of the diagonalised circulant is A0 + w_k A1 (+ w_k^2 A2)."""
    n, ell = S.n, S.ell
    th = np.arange(1, n + 1) * np.pi / (n + 1)

    def eig(B):
        d = B.diagonal(0)[0]
        e = B.diagonal(1)[0] if n > 1 else 0.0
        return d + 2.0 * e * np.cos(th)
    w = shift_eigenvalues(ell)
    if transpose:
        w = np.conj(w)
    lam = np.zeros((ell, n), dtype=np.complex128) + eig(constant_A0(S))[None, :]
    for j, Aj in enumerate(S.lower, start=1):
        lam = lam + (w[:, None] ** j) * eig(Aj)[None, :]
    return lam


def circulant_inverse_spectral(S: BlockSystem, X: np.ndarray,
                               transpose: bool = False) -> np.ndarray:
    """P^{-1} X through the sine (x) Fourier eigenbasis: an orthonormal DST-I
    along space, the DFT along time, division by the symbols, and the
    inverses.  Exact in exact arithmetic like circulant_inverse, but
    O(n ell log) instead of O(n ell^2), so it reaches the benchmark sizes."""
    import scipy.fft as sfft
    lam = sine_fourier_symbols(S, transpose)
    Z = sfft.dst(X.astype(np.float64), type=1, axis=1, norm="ortho")
    Z = np.fft.fft(Z, axis=0) / lam
    Z = np.fft.ifft(Z, axis=0).real
    return sfft.dst(Z, type=1, axis=1, norm="ortho")


def fourier_matrix(ell: int) -> np.ndarray:
    """Unitary U with U_{tk} = exp(2 pi i t k/ell)/sqrt(ell) (Section 3)."""
    t = np.arange(ell)
    return np.exp(2j * np.pi * np.outer(t, t) / ell) / np.sqrt(ell)


def shift_eigenvalues(ell: int) -> np.ndarray:
    """Diagonal of Lambda: Sigma = U Lambda U^*, w_k = exp(-2 pi i k/ell)."""
    return np.exp(-2j * np.pi * np.arange(ell) / ell)


def frequency_block(S: BlockSystem, w: complex):
    """I (x) A0 + sum_j Lambda^j (x) A_j restricted to frequency w."""
    B = constant_A0(S).astype(np.complex128)
    for j, Aj in enumerate(S.lower, start=1):
        B = B + (w ** j) * Aj
    return B


def circulant_inverse(S: BlockSystem, X: np.ndarray,
                      transpose: bool = False) -> np.ndarray:
    """Y = P^{-1} X (or P^{-T} X) by the diagonalised inverse of Section 3.

    P^T = I (x) A0^T + Sigma^T (x) A1^T; the blocks are symmetric and
    Sigma^T = U conj(Lambda) U^*, so the transpose uses conj(w_k).
    """
    ell = S.ell
    U = fourier_matrix(ell)
    w = shift_eigenvalues(ell)
    if transpose:
        w = np.conj(w)
    Z = U.conj().T @ X.astype(np.complex128)       # (U^* (x) I) x
    for k in range(ell):
        Z[k] = solve_tridiag(frequency_block(S, w[k]), Z[k])
    Y = U @ Z                                      # (U (x) I) y
    return Y.real.copy()


def dense_inverse_apply(C: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Solve C y = x with a dense LU (tiny sizes; C from system.dense_*)."""
    ell, n = X.shape
    return np.linalg.solve(C, X.reshape(-1)).reshape(ell, n)


def neumann_inverse(S: BlockSystem, X: np.ndarray, terms: int,
                    transpose: bool = False) -> np.ndarray:
    """Q_i^{-1} X with i = ``terms``, the Neumann approximation of Section 2:

        Q_i^{-1} = sum_{m=0}^{i-1} (-1)^m P^{-1} ([sigma (x) K] P^{-1})^m.

    E = sigma (x) kappa K is block diagonal and symmetric, so the transpose
    is sum_m (-1)^m (P^{-T} E)^m P^{-T}, i.e. the same sum with P^{-T}
    applied last.  terms = 1 gives P^{-1}.
    """
    if terms < 1:
        raise ValueError("terms >= 1")
    if not transpose:
        total = np.zeros_like(X, dtype=np.float64)
        W = X.astype(np.float64)
        for m in range(terms):
            PW = circulant_inverse(S, W)             # P^{-1} (E P^{-1})^m x
            total += (-1.0) ** m * PW
            W = neumann_E(S, PW)
        return total
    total = np.zeros_like(X, dtype=np.float64)
    for m in range(terms):
        V = circulant_inverse(S, X, transpose=True)   # P^{-T} x
        for _ in range(m):
            V = circulant_inverse(S, neumann_E(S, V), transpose=True)
        total += (-1.0) ** m * V
    return total
