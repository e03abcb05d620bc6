"""Shared helpers for the GPU parity tests (inputs come from `synthetic`,
expected values from `oracle`; nothing here computes the method)."""
import numpy as np
import pytest

import synthetic as syn
from oracle import system

EQ = {"heat": 0, "wave_bd2": 1, "heat_literal": 2, "wave_bd4": 3}


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
