"""Run one kernel family of the solver repeatedly on synthetic inputs, for
profilers (ncu) and quick timing.

    python -m paper_1810_00615_gb300.profile_case --op precond --n 4095 --ell 4096 \\
        --prec fp32 --reps 3

--space tridiag | dst selects the frequency-block solver.
--op precond | neumann | matvec | matvec_sub | matvec_f32 | matvec_dots | solve
(matvec_sub, matvec_f32: the fused product w = A z - v of an FP64 or FP32 z,
as the solver forms it in its Arnoldi step; matvec_dots: the same with the
Arnoldi dots v0 . w, v . w, w . w fused).  --transpose applies the transposed
operators (the adjoint solve's).  Prints one line with the mean CUDA-
event time per call.  Inputs are seeded standard-normal block vectors (or the
8-mode heat initial data for `solve`).
"""
from __future__ import annotations

import argparse
import os
import sys

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", default="precond", choices=["precond", "neumann", "matvec", "matvec_sub", "matvec_f32",
                             "matvec_dots", "solve"])
    ap.add_argument("--n", type=int, default=4095)
    ap.add_argument("--ell", type=int, default=4096)
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp32_refined", "fp64"])
    ap.add_argument("--equation", default="heat")
    ap.add_argument("--terms", type=int, default=2)
    ap.add_argument("--space", default="tridiag", choices=["tridiag", "dst"])
    ap.add_argument("--transpose", action="store_true")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    a = ap.parse_args(argv)

    import synthetic as syn
    from paper_1810_00615_gb300 import AllAtOnce

    s = AllAtOnce(a.n, a.ell, 1.0 / a.ell, equation=a.equation, precision=a.prec,
                  restart=30 if a.op == "solve" else 1, space=a.space)
    if a.op == "neumann":
        s.set_steps(syn.time_steps(a.ell, 0.5, syn.rng(3)))
    g = torch.Generator(device="cuda").manual_seed(1)
    x = torch.randn(a.ell, a.n, dtype=torch.float64, device="cuda", generator=g)
    y = torch.empty_like(x)
    x32 = x.float() if a.op == "matvec_f32" else None
    x2 = torch.randn_like(x) if a.op in ("matvec_sub", "matvec_dots") else None
    x3 = torch.randn_like(x) if a.op == "matvec_dots" else None
    tr = bool(a.transpose)
    if a.op == "solve":
        b = s.build_rhs(torch.from_numpy(syn.heat_initial(a.n)).cuda())

    def once():
        if a.op == "precond":
            s.precond_apply(x, out=y, transpose=tr)
        elif a.op == "neumann":
            s.neumann_apply(x, a.terms, out=y, transpose=tr)
        elif a.op == "matvec":
            s.matvec(x, out=y, transpose=tr)
        elif a.op == "matvec_sub":
            s.matvec(x, out=y, sub=x2, transpose=tr)
        elif a.op == "matvec_f32":
            s.matvec_f32(x32, out=y, sub=x, transpose=tr)
        elif a.op == "matvec_dots":
            s.matvec_dots(x, x2, x3, out=y, transpose=tr)
        else:
            s.solve(b, restart=30, rtol=1e-10)

    for _ in range(a.warmup):
        once()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        once()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    print(f"op={a.op} n={a.n} ell={a.ell} prec={a.prec} space={a.space} transpose={int(tr)} "
          f"equation={a.equation} ms_per_call={ms:.4f} "
          f"launches={s.kernel_launches()}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
