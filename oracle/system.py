"""All-at-once block systems of Section 2 (heat, variable-step heat, BD2 and
BD4 wave).

A block vector is an array of shape (ell, n); row t holds u_{t+1}.

Time-stepping blocks:

* Heat, implicit Euler with constant step tau (Section 2, monolithic heat
  system): A0 = M + tau*kappa*K, A1 = -M.  The paper prints A0 = K + tau M,
  which is not implicit Euler applied to M u' = -K u (the time step must
  multiply the stiffness term) and contradicts its own splitting
  Q = P + sigma (x) K; this oracle reads A0 = M + tau*kappa*K and keeps the
  printed form behind ``literal=True`` (A0 = K + tau M).
* Heat with steps tau_1..tau_ell (system B of Section 2): A0^t = M +
  tau_t*kappa*K on the block diagonal, A1 = -M below it.
* Wave, BD2 (Section 2, C_BD2): A0 = M + tau^2 K, A1 = -2M, A2 = M.
* Wave, BD4 (Section 2, C_BD4): the four-step formula gives A0 = 2M +
  tau^2 K, A1 = -5M, A2 = 4M, A3 = -M; its first two rows are BD2 steps
  (diagonal B = M + tau^2 K, and C = -2M below the second one), so the
  matrix is Toeplitz only from the third block row on.

The monolithic matrix is block lower-triangular (block-diagonal part per
step for B and for the BD4 start-up rows):
(A U)_t = A0^t u_t + sum_{j>=1} A_j^t u_{t-j}, with A_j^t = A_j except where
``startup`` names another block for row t.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.sparse as sp
import scipy.linalg as sla

from .fem import p1_matrices


def solve_tridiag(A, r: np.ndarray) -> np.ndarray:
    """Solve A y = r for a tridiagonal (sparse or dense) A with LAPACK's
    banded LU (partial pivoting); A and r may be complex."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    ab = np.zeros((3, n), dtype=np.result_type(A.dtype, r.dtype))
    ab[1] = A.diagonal(0)
    if n > 1:
        ab[0, 1:] = A.diagonal(1)
        ab[2, :-1] = A.diagonal(-1)
    return sla.solve_banded((1, 1), ab, r)


@dataclass
class BlockSystem:
    """Block lower-triangular system: diagonal blocks ``diag[t]`` (one per
    step) and constant sub-diagonal blocks ``lower[j-1]`` = A_j, j >= 1."""
    n: int
    ell: int
    diag: List[sp.csr_matrix]
    lower: List[sp.csr_matrix]
    M: sp.csr_matrix
    K: sp.csr_matrix
    kind: str
    tau: float                       # the constant step of the circulant
    taus: Optional[np.ndarray] = None  # per-step tau_t (system B), else None
    kappa: float = 1.0
    extra: dict = field(default_factory=dict)
    startup: dict = field(default_factory=dict)  # (t, j) -> block at row t, lag j


def lag_block(S: BlockSystem, t: int, j: int):
    """The block multiplying u_{t-j} in block row t (j >= 1)."""
    return S.startup.get((t, j), S.lower[j - 1])


def heat(n: int, ell: int, tau: float, kappa: float = 1.0,
         literal: bool = False) -> BlockSystem:
    """Monolithic heat system (Section 2, implicit Euler, constant tau)."""
    M, K = p1_matrices(n)
    if literal:
        A0 = (K + tau * M).tocsr()
    else:
        A0 = (M + tau * kappa * K).tocsr()
    A1 = (-M).tocsr()
    return BlockSystem(n, ell, [A0] * ell, [A1], M, K,
                       "heat_literal" if literal else "heat", tau, None, kappa)


def heat_steps(n: int, taus: np.ndarray, kappa: float = 1.0,
               tau: Optional[float] = None) -> BlockSystem:
    """System B of Section 2: A0^t = M + tau_t kappa K, A1 = -M.

    ``tau`` is the constant step of the circulant P that approximates it;
    the paper sets tau = 1/ell (T = 1)."""
    taus = np.asarray(taus, dtype=np.float64)
    ell = taus.size
    M, K = p1_matrices(n)
    diag = [(M + t * kappa * K).tocsr() for t in taus]
    if tau is None:
        tau = 1.0 / ell
    return BlockSystem(n, ell, diag, [(-M).tocsr()], M, K, "heat", tau,
                       taus.copy(), kappa)


def bd2(n: int, ell: int, tau: float) -> BlockSystem:
    """C_BD2 of Section 2: A0 = M + tau^2 K, A1 = -2M, A2 = M."""
    M, K = p1_matrices(n)
    A0 = (M + tau * tau * K).tocsr()
    return BlockSystem(n, ell, [A0] * ell, [(-2.0 * M).tocsr(), M.copy()],
                       M, K, "bd2", tau)


def bd4(n: int, ell: int, tau: float) -> BlockSystem:
    """C_BD4 of Section 2.  Rows t >= 2 (0-based) apply the four-step formula
    (2M + tau^2 K) u_t - 5M u_{t-1} + 4M u_{t-2} - M u_{t-3}; rows 0 and 1
    are BD2 steps, B u_1 and C u_1 + B u_2 with B = M + tau^2 K, C = -2M."""
    M, K = p1_matrices(n)
    B = (M + tau * tau * K).tocsr()
    A0 = (2.0 * M + tau * tau * K).tocsr()
    diag = [B if t < 2 else A0 for t in range(ell)]
    lower = [(-5.0 * M).tocsr(), (4.0 * M).tocsr(), (-M).tocsr()]
    startup = {(1, 1): (-2.0 * M).tocsr()}
    return BlockSystem(n, ell, diag, lower, M, K, "bd4", tau, startup=startup)


def matvec(S: BlockSystem, X: np.ndarray) -> np.ndarray:
    """Y = A X with (A X)_t = A0^t x_t + sum_j A_j^t x_{t-j} (x_{<0} = 0)."""
    Y = np.empty_like(X, dtype=np.result_type(X, np.float64))
    for t in range(S.ell):
        y = S.diag[t] @ X[t]
        for j in range(1, len(S.lower) + 1):
            if t - j >= 0:
                y = y + lag_block(S, t, j) @ X[t - j]
        Y[t] = y
    return Y


def matvec_T(S: BlockSystem, X: np.ndarray) -> np.ndarray:
    """Y = A^T X: (A^T X)_t = (A0^t)^T x_t + sum_j (A_j^{t+j})^T x_{t+j}."""
    Y = np.empty_like(X, dtype=np.result_type(X, np.float64))
    for t in range(S.ell):
        y = S.diag[t].T @ X[t]
        for j in range(1, len(S.lower) + 1):
            if t + j < S.ell:
                y = y + lag_block(S, t + j, j).T @ X[t + j]
        Y[t] = y
    return Y


def forward_substitution(S: BlockSystem, B: np.ndarray) -> np.ndarray:
    """Exact A^{-1} B: u_t = (A0^t)^{-1}(b_t - sum_j A_j u_{t-j}), in t order.

    This is time stepping itself; it is what the preconditioned GMRES
    solve must reproduce."""
    U = np.zeros_like(B, dtype=np.float64)
    for t in range(S.ell):
        r = B[t].copy()
        for j in range(1, len(S.lower) + 1):
            if t - j >= 0:
                r = r - lag_block(S, t, j) @ U[t - j]
        U[t] = solve_tridiag(S.diag[t], r)
    return U


def heat_modal_solution(n: int, taus, u0: np.ndarray, kappa: float = 1.0) -> np.ndarray:
    """Exact A^{-1} [M u0; 0; ...; 0] of the heat systems (Section 2, constant
    or variable steps taus = tau_1..tau_ell) by the sine-mode closed form.

    M and K are diagonalised by the orthonormal DST-I vectors s_j with
    eigenvalues m_j = h (1 - (2/3) sin^2(th_j/2)) and k_j = (4/h)
    sin^2(th_j/2), th_j = j pi/(n+1) (textbook; the same eigenpairs pin
    fem.p1_matrices), so implicit Euler acts on each mode by itself:
    (m_j + tau_t kappa k_j) u_{t,j} = m_j u_{t-1,j}, i.e.
    u_{t,j} = prod_{s<=t} rho_j(tau_s) u0_j, rho_j = m_j/(m_j + tau kappa k_j).
    The modes come from orthonormal DST-I transforms, whose error is a few
    ulps whatever the step blocks' condition.  It is the reference where
    banded time stepping (forward_substitution) loses accuracy to that
    condition: a backward-stable solve of A0 = M + tau kappa K perturbs a
    smooth solution by about eps (4 tau kappa / h^2) per step, ~4e-9 at
    n = 65535, tau = 1/512, and the smooth modes carry it for many steps."""
    import scipy.fft as sfft
    taus = np.asarray(taus, dtype=np.float64)
    h = 1.0 / (n + 1)
    s2 = np.sin(np.arange(1, n + 1) * np.pi / (2.0 * (n + 1))) ** 2
    m = h * (1.0 - (2.0 / 3.0) * s2)
    k = (4.0 / h) * s2
    c = sfft.dst(np.asarray(u0, dtype=np.float64), type=1, norm="ortho")
    U = np.empty((taus.size, n), dtype=np.float64)
    fac = np.ones(n)
    for t, tau in enumerate(taus):
        fac = fac * (m / (m + tau * kappa * k))
        U[t] = fac * c
    return sfft.idst(U, type=1, norm="ortho", axis=1)


def backward_substitution(S: BlockSystem, G: np.ndarray) -> np.ndarray:
    """Exact A^{-T} G (block upper-triangular), t from ell-1 down to 0."""
    L = np.zeros_like(G, dtype=np.float64)
    for t in range(S.ell - 1, -1, -1):
        r = G[t].copy()
        for j in range(1, len(S.lower) + 1):
            if t + j < S.ell:
                r = r - lag_block(S, t + j, j).T @ L[t + j]
        L[t] = solve_tridiag(S.diag[t].T, r)
    return L


def rhs_heat(S: BlockSystem, u0: np.ndarray) -> np.ndarray:
    """b = [M u0; 0; ...; 0] (Section 2, monolithic heat system)."""
    B = np.zeros((S.ell, S.n))
    B[0] = S.M @ u0
    return B


def rhs_bd2(S: BlockSystem, u0: np.ndarray,
            v0: Optional[np.ndarray] = None) -> np.ndarray:
    """b_BD2 = [(M + tau^2 K) u0; -M u0; 0; ...] (Section 2).

    With an initial velocity v0 (not in the paper, whose wave problem starts
    at rest) the first row becomes A0 (u0 + tau v0), i.e. u_1 = u0 + tau v0,
    a first-order start; the second row stays -M u0."""
    B = np.zeros((S.ell, S.n))
    A0 = S.diag[0]
    first = u0 if v0 is None else u0 + S.tau * v0
    B[0] = A0 @ first
    if S.ell > 1:
        B[1] = -(S.M @ u0)
    return B


def rhs_bd4(S: BlockSystem, u0: np.ndarray,
            v0: Optional[np.ndarray] = None) -> np.ndarray:
    """b_BD4 = [B u0; -M u0; M u0; 0; ...] (Section 2): the BD2 start-up rows
    as in rhs_bd2 (B = M + tau^2 K, the first row B (u0 + tau v0) with an
    initial velocity), and the third row carries the -M u_0 term of the
    first four-step equation to the right-hand side."""
    B = np.zeros((S.ell, S.n))
    first = u0 if v0 is None else u0 + S.tau * v0
    B[0] = S.diag[0] @ first
    if S.ell > 1:
        B[1] = -(S.M @ u0)
    if S.ell > 2:
        B[2] = S.M @ u0
    return B


# ---------------------------------------------------------------- dense forms
def dense_monolithic(S: BlockSystem) -> np.ndarray:
    """Dense n*ell x n*ell matrix of A (tiny sizes only)."""
    n, ell = S.n, S.ell
    A = np.zeros((n * ell, n * ell))
    for t in range(ell):
        A[t * n:(t + 1) * n, t * n:(t + 1) * n] = S.diag[t].toarray()
        for j in range(1, len(S.lower) + 1):
            if t - j >= 0:
                A[t * n:(t + 1) * n, (t - j) * n:(t - j + 1) * n] = lag_block(S, t, j).toarray()
    return A


def dense_circulant(S: BlockSystem, per_step: bool = False) -> np.ndarray:
    """Dense block circulant built entry by entry (tiny sizes only).

    per_step=False: P (heat, Section 2), R_BD2 or R_BD4 (wave): every
    diagonal block is the constant-step A0 (M + tau kappa K for heat,
    M + tau^2 K for BD2, 2M + tau^2 K for BD4), and block A_j sits at block
    column (t - j) mod ell in every row.  R_BD4 is the circulant of the
    Toeplitz part of C_BD4; the start-up rows do not enter it.
    per_step=True: Q of Section 2, the diagonal blocks A0^t of system B.
    """
    n, ell = S.n, S.ell
    if per_step:
        diag = [d.toarray() for d in S.diag]
    else:
        diag = [constant_A0(S).toarray()] * ell
    C = np.zeros((n * ell, n * ell))
    for t in range(ell):
        C[t * n:(t + 1) * n, t * n:(t + 1) * n] = diag[t]
        for j, Aj in enumerate(S.lower, start=1):
            c = (t - j) % ell
            C[t * n:(t + 1) * n, c * n:(c + 1) * n] += Aj.toarray()
    return C


def constant_A0(S: BlockSystem) -> sp.csr_matrix:
    """The constant-step diagonal block used by the circulant."""
    if S.kind == "heat":
        return (S.M + S.tau * S.kappa * S.K).tocsr()
    if S.kind == "heat_literal":
        return (S.K + S.tau * S.M).tocsr()
    if S.kind == "bd2":
        return (S.M + S.tau * S.tau * S.K).tocsr()
    if S.kind == "bd4":
        return (2.0 * S.M + S.tau * S.tau * S.K).tocsr()
    raise ValueError(S.kind)


def neumann_E(S: BlockSystem, X: np.ndarray) -> np.ndarray:
    """E X with E = sigma (x) kappa K, sigma_t = tau_t - tau (Section 2,
    Q = P + sigma (x) K; t = 1..ell, the paper's index range [0, ell] read
    as the ell steps)."""
    if S.taus is None:
        return np.zeros_like(X)
    sig = S.taus - S.tau
    Y = np.empty_like(X)
    for t in range(S.ell):
        Y[t] = sig[t] * S.kappa * (S.K @ X[t])
    return Y
