"""CPU oracle for the all-at-once MPW-preconditioned solve (test infrastructure).

This package is test infrastructure.  Only ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline and reference legs of ``bench.py`` may import it.  The
CUDA library never calls it, and it shares no code with the CUDA path: it is
plain, slow FP64 numpy/scipy written from the paper (Goddard & Wathen, "A
note on parallel preconditioning for all-at-once evolutionary PDEs").

Contents (each function cites the passage it follows):

* ``fem``      P1 mass/stiffness matrices and the L2 projection (Section 2).
* ``system``   time-stepping blocks for the heat equation (uniform and
               variable steps) and the BD2 and BD4 wave schemes (BD4 with
               its BD2 start-up rows); the monolithic
               operators, their transposes, exact solves by forward and
               backward substitution, right-hand sides, and dense assembly
               of every block matrix for tiny sizes (Section 2).
* ``precond``  the block-circulant preconditioners P, Q, R_BD2, R_BD4 applied
               through the Fourier diagonalisation with a dense DFT (Section
               3, method 1) and per-frequency tridiagonal solves; the
               Neumann-series approximation Q_i^{-1} (Section 2).
* ``gmres``    restarted GMRES with modified Gram-Schmidt, left- and right-
               (flexible) preconditioned.
* ``adjoint``  the loss 1/2||U - U_obs||^2 and its gradients with respect to
               u0 and the diffusion coefficient by the adjoint system.
* ``cbaseline`` a multithreaded C baseline of the heat solve (radix-2 FFT
               along time, Thomas per frequency, GMRES; OpenMP) that the
               benchmark times on the host cores beside the GPU solve.  It
               is not an oracle: ``tests/test_oracle_cbaseline.py`` checks it
               against the functions above.  It is imported on demand, not
               here.

Readings of the paper where it is silent or garbled (all stated again where
they are used):

* A0 = M + tau*kappa*K, A1 = -M for implicit Euler (the paper prints
  K + tau M, which is not implicit Euler for M u' = -K u and does not give
  Q - P = sigma (x) K; the literal form stays available as ``literal=True``).
* M and K are the uniform P1 matrices on [0,1] with n interior nodes.
* Sigma is the ell x ell cyclic down-shift, and U is the unitary DFT of
  size ell, so block k of the diagonalised circulant is A0 + w_k A1 (+ w_k^2
  A2) with w_k = exp(-2 pi i k / ell).
* sigma_t = tau_t - tau for t = 1..ell with tau = T/ell.

Parity pins: every function is checked in ``tests/test_oracle_pins.py``
against closed forms, brute-force dense algebra or invariants; none is
without such a pin.
"""
from . import fem, system, precond, gmres, adjoint  # noqa: F401
