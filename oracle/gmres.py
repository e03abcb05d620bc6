"""Restarted GMRES (Saad & Schultz), the Krylov method the paper uses.

The paper states neither the restart length, the orthogonalisation, nor
what its tolerance 1e-5 measures.  This oracle offers both forms:

* ``side="left"``: GMRES on P^{-1} A U = P^{-1} b, the form of the paper's
  table captions; convergence is tested on the preconditioned residual.
* ``side="right"``: flexible GMRES (Saad 1993) on A Z y with Z = [P^{-1} v_j]
  stored, so that the preconditioner may vary; convergence is tested on
  the true residual ||b - A x|| / ||b||, re-computed at every restart.

Orthogonalisation is modified Gram-Schmidt; the Hessenberg least-squares
problem is reduced by Givens rotations.  ``iters`` counts Arnoldi steps,
i.e. products with A.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np


@dataclass
class Info:
    iters: int = 0
    restarts: int = 0
    relres_true: float = np.inf
    relres_est: float = np.inf
    converged: bool = False
    history: List[float] = field(default_factory=list)


def _givens(a: float, b: float):
    if b == 0.0:
        return 1.0, 0.0
    r = np.hypot(a, b)
    return a / r, b / r


def gmres(apply_A: Callable[[np.ndarray], np.ndarray], b: np.ndarray,
          x0: Optional[np.ndarray] = None,
          apply_P: Optional[Callable[[np.ndarray], np.ndarray]] = None,
          restart: int = 30, rtol: float = 1e-10, maxit: int = 1000,
          side: str = "right"):
    """Solve A x = b; returns (x, Info).  Vectors may be any shape."""
    shape = b.shape
    bf = b.reshape(-1).astype(np.float64)
    A = lambda v: apply_A(v.reshape(shape)).reshape(-1)
    P = (lambda v: v) if apply_P is None else \
        (lambda v: apply_P(v.reshape(shape)).reshape(-1))
    x = np.zeros_like(bf) if x0 is None else x0.reshape(-1).astype(np.float64)
    info = Info()
    bnorm = np.linalg.norm(bf)
    if bnorm == 0.0:
        info.relres_true = 0.0
        info.converged = True
        return np.zeros(shape), info
    if side == "left":
        target = np.linalg.norm(P(bf))
    else:
        target = bnorm
    while True:
        r = bf - A(x)
        info.relres_true = np.linalg.norm(r) / bnorm
        if side == "left":
            r = P(r)
        beta = np.linalg.norm(r)
        if side == "right" and info.relres_true <= rtol:
            info.converged = True
            break
        if side == "left" and beta <= rtol * target:
            info.converged = True
            break
        if info.iters >= maxit or beta == 0.0:
            break
        m = restart
        V = np.zeros((m + 1, bf.size))
        Z = np.zeros((m, bf.size)) if side == "right" else None
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            if side == "right":
                Z[j] = P(V[j])
                w = A(Z[j])
            else:
                w = P(A(V[j]))
            for i in range(j + 1):               # modified Gram-Schmidt
                H[i, j] = np.dot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            breakdown = H[j + 1, j] == 0.0
            if not breakdown:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                   # apply previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            info.iters += 1
            j_done = j + 1
            est = abs(g[j + 1]) / target
            info.relres_est = est
            info.history.append(est)
            if est <= rtol or breakdown or info.iters >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        if side == "right":
            x = x + Z[:j_done].T @ y
        else:
            x = x + V[:j_done].T @ y
        info.restarts += 1
        if info.iters >= maxit:
            r = bf - A(x)
            info.relres_true = np.linalg.norm(r) / bnorm
            if side == "right":
                info.converged = info.relres_true <= rtol
            else:
                info.converged = np.linalg.norm(P(r)) <= rtol * target
            break
    return x.reshape(shape), info
