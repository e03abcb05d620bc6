"""Multithreaded CPU baseline of the all-at-once heat solve (`cbaseline.c`).

Test and measurement infrastructure, like the rest of this package: the
benchmark times it beside the GPU solve as the fast CPU comparison (the
plain oracle, dense DFT and banded LU per frequency, is the slow exact one).
It computes the same right-preconditioned GMRES on the Section 2
implicit-Euler system with the block-circulant P of Section 2, applied by
radix-2 FFTs along time and Thomas solves per frequency (Section 3), in FP64
with OpenMP.  Heat equation, uniform steps, ell a power of two.

The shared library is compiled with gcc on first use (or by the
repository's build step) next to the source.
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import shutil
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cbaseline.c")
LIB = os.path.join(HERE, "libcbaseline.so")
_lock = threading.Lock()
_lib = None


def compile_cmd(out: str = LIB):
    cc = os.environ.get("CC") or shutil.which("gcc") or "cc"
    return [cc, "-O3", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", SRC, "-o", out, "-lm"]


def build(force: bool = False) -> str:
    """Compile libcbaseline.so if it is missing or older than its source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = f"{LIB}.{os.getpid()}.{platform.machine()}.tmp"
    r = subprocess.run(compile_cmd(tmp), capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"gcc failed for cbaseline.c:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def lib() -> C.CDLL:
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        try:
            h = C.CDLL(LIB)
        except OSError:          # built for another machine: rebuild here
            build(force=True)
            h = C.CDLL(LIB)
        d, i64, p = C.c_double, C.c_int64, C.c_void_p
        for name in ("cb_heat_precond", "cb_heat_matvec"):
            f = getattr(h, name)
            f.restype = C.c_int
            f.argtypes = [i64, i64, d, d, p, p]
        h.cb_heat_fgmres.restype = C.c_int
        h.cb_heat_fgmres.argtypes = [i64, i64, d, d, p, p, C.c_int, d, C.c_int,
                                     C.POINTER(C.c_int), C.POINTER(d)]
        h.cb_threads.restype = C.c_int
        h.cb_threads.argtypes = []
        _lib = h
        return _lib


def _vec(a, n, ell):
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if a.size != n * ell:
        raise ValueError("need n * ell values")
    return a


def _check(st, where):
    if st < 0:
        raise RuntimeError(f"{where} failed with status {st}")


def threads() -> int:
    return int(lib().cb_threads())


def heat_precond(n, ell, tau, X, kappa=1.0):
    """P^{-1} X for the heat system (X: [ell, n])."""
    x = _vec(X, n, ell)
    y = np.empty_like(x)
    _check(lib().cb_heat_precond(n, ell, tau, kappa, x.ctypes.data, y.ctypes.data),
           "cb_heat_precond")
    return y.reshape(ell, n)


def heat_matvec(n, ell, tau, X, kappa=1.0):
    """A X for the heat system (X: [ell, n])."""
    x = _vec(X, n, ell)
    y = np.empty_like(x)
    _check(lib().cb_heat_matvec(n, ell, tau, kappa, x.ctypes.data, y.ctypes.data),
           "cb_heat_matvec")
    return y.reshape(ell, n)


def heat_fgmres(n, ell, tau, B, kappa=1.0, restart=30, rtol=1e-10, maxit=300, X0=None):
    """Solve A X = B from X0 (default 0).  Returns (X, iterations, true
    relative residual, converged)."""
    b = _vec(B, n, ell)
    x = np.zeros_like(b) if X0 is None else _vec(X0, n, ell).copy()
    it, rel = C.c_int(0), C.c_double(0.0)
    st = lib().cb_heat_fgmres(n, ell, tau, kappa, b.ctypes.data, x.ctypes.data, int(restart),
                              float(rtol), int(maxit), C.byref(it), C.byref(rel))
    _check(st, "cb_heat_fgmres")
    return x.reshape(ell, n), it.value, rel.value, st == 0


def _bench_main(argv=None) -> int:
    """Time the host-core references for one heat workload and print one
    JSON object: the oracle's forward substitution (exact time stepping; one
    core, the sequential method the all-at-once solve competes with) and
    this multithreaded FGMRES (one untimed solve, then the median of
    `reps`).  Run as a separate process so that its OpenMP runtime never
    shares a process with the caller's."""
    import argparse
    import json
    import statistics
    import sys
    import time

    sys.path.insert(0, os.path.dirname(HERE))
    import synthetic as syn
    from oracle import system

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, required=True)
    ap.add_argument("--ell", type=int, required=True)
    ap.add_argument("--modes", type=int, default=8)
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)
    S = system.heat(a.n, a.ell, 1.0 / a.ell)
    B = system.rhs_heat(S, syn.heat_initial(a.n, modes=a.modes))
    out = {}
    t0 = time.perf_counter()
    U = system.forward_substitution(S, B)
    out["forward_substitution"] = {
        "value": time.perf_counter() - t0, "unit": "s", "cores": 1,
        "kind": "oracle time stepping: one banded LU solve per step, in step order"}
    x, it, rel, ok = heat_fgmres(a.n, a.ell, 1.0 / a.ell, B, restart=a.restart, rtol=a.rtol)
    ts = []
    for _ in range(max(1, a.reps)):
        t0 = time.perf_counter()
        x, it, rel, ok = heat_fgmres(a.n, a.ell, 1.0 / a.ell, B, restart=a.restart, rtol=a.rtol)
        ts.append(time.perf_counter() - t0)
    err = float(np.max(np.abs(x - U)) / np.max(np.abs(U)))
    out["cpu_fgmres"] = {
        "value": statistics.median(ts), "unit": "s", "cores": threads(),
        "kind": f"right-preconditioned GMRES({a.restart}), P by radix-2 FFT + Thomas, FP64, "
                "OpenMP (oracle/cbaseline.c)",
        "iters": it, "relres_true": rel, "converged": bool(ok), "rel_err_vs_time_stepping": err,
        "sample": f"median of {len(ts)} full solves after one untimed"}
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(_bench_main())
