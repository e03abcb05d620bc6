"""Seeded synthetic inputs shared by the CUDA path's callers and the oracle.

This module draws random numbers and samples closed-form initial data.  It
holds none of the all-at-once method's arithmetic: no mass or stiffness
matrix, no time-stepping block, no preconditioner.  Both the tests and
``bench.py`` take their inputs from here, and the oracle checks the one
closed form used here (the L2 projection of a sine mode) against its own
quadrature route.

Recipe (numpy PCG64, seed 1810615 unless a caller passes another seed):

* Initial data ``s(x) = sum_j c_j sin(j pi x)`` on [0, 1] with ``c_j ~
  N(0, 1) / j**2`` (8 modes for the heat workloads, 16 for the wave
  workload), drawn in mode order.
* The nodal vector ``u0`` handed to the solver is the L2 projection of
  ``s`` onto continuous piecewise-linear functions on the uniform grid with
  ``n`` interior nodes, ``h = 1/(n+1)`` (Section 2: u_0 is a projection of
  the initial data).  For a single sine mode the projection is the mode
  itself scaled by ``gamma_j = [h * 2(1 - cos t)/t**2] / m_j`` with
  ``t = j pi h`` and ``m_j = (h/6)(4 + 2 cos t)``; the sine vector is an
  eigenvector of the P1 mass matrix, so the projection stays in that mode.
* Non-uniform time grids follow Section 4: ``t_0 = 0``, ``t_ell = 1`` and
  ``t_j = (j + delta (R_j - 0.5)) / ell`` with ``R_j`` uniform on [0, 1).
* The non-smooth wave initial condition of Section 4 (Tables 3 and 4):
  ``u0(x) = cos^2(4 pi (x - 1/2))`` on (3/8, 5/8), zero elsewhere, sampled
  at the interior nodes (the paper does not say how it is discretised).
* Random block vectors (parity inputs) are standard normal, shape
  ``(ell, n)``, row ``t`` holding time block ``t+1``.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 1810615


def rng(seed: int = DEFAULT_SEED) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def sine_coefficients(modes: int, gen: np.random.Generator) -> np.ndarray:
    """c_j ~ N(0,1)/j^2 for j = 1..modes."""
    j = np.arange(1, modes + 1, dtype=np.float64)
    return gen.standard_normal(modes) / j**2


def grid(n: int) -> np.ndarray:
    """Interior nodes x_i = i h, i = 1..n, h = 1/(n+1)."""
    h = 1.0 / (n + 1)
    return h * np.arange(1, n + 1, dtype=np.float64)


def sine_nodal(coeffs: np.ndarray, n: int) -> np.ndarray:
    """Nodal samples of s(x) = sum_j c_j sin(j pi x) at the interior nodes."""
    x = grid(n)
    out = np.zeros(n)
    for j, c in enumerate(coeffs, start=1):
        out += c * np.sin(j * np.pi * x)
    return out


def sine_l2_projection(coeffs: np.ndarray, n: int) -> np.ndarray:
    """Nodal vector of the P1 L2 projection of sum_j c_j sin(j pi x)."""
    h = 1.0 / (n + 1)
    x = grid(n)
    out = np.zeros(n)
    for j, c in enumerate(coeffs, start=1):
        t = j * np.pi * h
        load = h * 2.0 * (1.0 - np.cos(t)) / t**2
        mass = (h / 6.0) * (4.0 + 2.0 * np.cos(t))
        out += c * (load / mass) * np.sin(j * np.pi * x)
    return out


def time_grid(ell: int, delta: float, gen: np.random.Generator) -> np.ndarray:
    """Perturbed grid t_0..t_ell of Section 4 (1/ell spacing reading)."""
    t = np.empty(ell + 1)
    t[0] = 0.0
    t[ell] = 1.0
    r = gen.random(ell - 1) if ell > 1 else np.zeros(0)
    j = np.arange(1, ell, dtype=np.float64)
    t[1:ell] = (j + delta * (r - 0.5)) / ell
    return t


def time_steps(ell: int, delta: float, gen: np.random.Generator) -> np.ndarray:
    """Steps tau_j = t_j - t_{j-1}, j = 1..ell."""
    return np.diff(time_grid(ell, delta, gen))


def block_vector(n: int, ell: int, gen: np.random.Generator) -> np.ndarray:
    """Standard-normal block vector, shape (ell, n)."""
    return gen.standard_normal((ell, n))


def parabola_load(n: int) -> np.ndarray:
    """Load vector (u0, phi_i) of the paper's Table 1/2 initial condition
    u0(x) = x(1 - x) against the P1 hats on the uniform grid, in closed form:
    h x_i (1 - x_i) - h^3 / 6.  It is M times the L2 projection of u0, i.e.
    the first block of the heat right-hand side."""
    h = 1.0 / (n + 1)
    x = grid(n)
    return h * x * (1.0 - x) - h ** 3 / 6.0


def heat_initial(n: int, modes: int = 8, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Projected u0 for the heat workloads (seeded sine modes)."""
    g = rng(seed)
    return sine_l2_projection(sine_coefficients(modes, g), n)


def wave_initial(n: int, modes: int = 16, seed: int = DEFAULT_SEED):
    """Projected (u0, v0) for the wave workload: displacement then velocity."""
    g = rng(seed)
    a = sine_coefficients(modes, g)
    b = sine_coefficients(modes, g)
    return sine_l2_projection(a, n), sine_l2_projection(b, n)


def wave_nonsmooth(n: int) -> np.ndarray:
    """Nodal samples of the non-smooth wave initial condition of Section 4:
    cos^2(4 pi (x - 1/2)) for 3/8 < x < 5/8, zero elsewhere."""
    x = grid(n)
    return np.where((x > 0.375) & (x < 0.625), np.cos(4.0 * np.pi * (x - 0.5)) ** 2, 0.0)
