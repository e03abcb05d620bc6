"""Adjoint gradients of a data-misfit loss through the heat all-at-once solve.

Not in the paper: the loss L(u0, kappa) = 1/2 ||U - U_obs||^2 with
A(kappa) U = b(u0), b = [M u0; 0; ...] (Section 2, monolithic heat system,
A0 = M + tau_t kappa K, A1 = -M).  By the adjoint method, with
A^T lam = U - U_obs (block upper-triangular, solved by backward
substitution),

    dL/du0    = M^T lam_1 = M lam_1                (b depends on u0 via M u0)
    dL/dkappa = -lam^T (dA/dkappa) U = -sum_t tau_t lam_t^T K u_t.
"""
from __future__ import annotations

import numpy as np

from .system import (BlockSystem, backward_substitution, forward_substitution,
                     heat, heat_steps, rhs_heat)


def _system(n, ell, tau, kappa, taus=None) -> BlockSystem:
    if taus is None:
        return heat(n, ell, tau, kappa)
    return heat_steps(n, taus, kappa, tau)


def loss(n, ell, tau, kappa, u0, U_obs, taus=None) -> float:
    """L = 1/2 ||U - U_obs||^2 with U the exact all-at-once solution."""
    S = _system(n, ell, tau, kappa, taus)
    U = forward_substitution(S, rhs_heat(S, u0))
    D = U - U_obs
    return 0.5 * float(np.sum(D * D))


def gradients(n, ell, tau, kappa, u0, U_obs, taus=None):
    """Return (L, dL/du0, dL/dkappa, U, lam)."""
    S = _system(n, ell, tau, kappa, taus)
    U = forward_substitution(S, rhs_heat(S, u0))
    G = U - U_obs
    lam = backward_substitution(S, G)
    g_u0 = S.M.T @ lam[0]
    steps = np.full(ell, tau) if taus is None else np.asarray(taus)
    g_kappa = -sum(steps[t] * float(lam[t] @ (S.K @ U[t])) for t in range(ell))
    L = 0.5 * float(np.sum(G * G))
    return L, g_u0, g_kappa, U, lam
