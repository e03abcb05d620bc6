"""P1 finite elements on [0, 1] (Section 2, eq. for M du/dt = -K u).

The paper names M and K but never prints their entries.  Reading: standard
continuous piecewise-linear Galerkin elements on a uniform grid with n
interior nodes, h = 1/(n+1), homogeneous Dirichlet conditions, so that
M = (h/6) tridiag(1, 4, 1) and K = (1/h) tridiag(-1, 2, -1).  Here they are
assembled element by element, which is the definition, not the stencil.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def p1_matrices(n: int):
    """Assemble (M, K) element by element; returns scipy CSR matrices.

    Element e spans nodes e and e+1 (global nodes 0..n+1, the two ends are
    Dirichlet and dropped).  Local mass (h/6)[[2,1],[1,2]], local stiffness
    (1/h)[[1,-1],[-1,1]].
    """
    h = 1.0 / (n + 1)
    mloc = (h / 6.0) * np.array([[2.0, 1.0], [1.0, 2.0]])
    kloc = (1.0 / h) * np.array([[1.0, -1.0], [-1.0, 1.0]])
    rows, cols, mv, kv = [], [], [], []
    for e in range(n + 1):
        nodes = (e - 1, e)  # interior index of global nodes e, e+1
        for a in range(2):
            for b in range(2):
                ia, ib = nodes[a], nodes[b]
                if 0 <= ia < n and 0 <= ib < n:
                    rows.append(ia)
                    cols.append(ib)
                    mv.append(mloc[a, b])
                    kv.append(kloc[a, b])
    M = sp.coo_matrix((mv, (rows, cols)), shape=(n, n)).tocsr()
    K = sp.coo_matrix((kv, (rows, cols)), shape=(n, n)).tocsr()
    return M, K


def l2_projection(f, n: int, qorder: int = 12) -> np.ndarray:
    """P1 L2 projection of a function f on [0,1]: solve M u = (f, phi_i).

    The load vector uses Gauss-Legendre quadrature of order ``qorder`` on
    each element.  Section 2 takes u_0 as a projection of the initial data.
    """
    h = 1.0 / (n + 1)
    xg, wg = np.polynomial.legendre.leggauss(qorder)
    load = np.zeros(n)
    for e in range(n + 1):
        x0 = e * h
        xq = x0 + 0.5 * h * (xg + 1.0)
        wq = 0.5 * h * wg
        fq = f(xq)
        phi_left = (x0 + h - xq) / h   # hat of global node e (interior e-1)
        phi_right = (xq - x0) / h      # hat of global node e+1 (interior e)
        if e - 1 >= 0:
            load[e - 1] += np.sum(wq * fq * phi_left)
        if e < n:
            load[e] += np.sum(wq * fq * phi_right)
    M, _ = p1_matrices(n)
    return spla.spsolve(M.tocsc(), load)
