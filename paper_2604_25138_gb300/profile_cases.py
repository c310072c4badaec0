"""Small, self-contained invocations of single stages of the path, for
profiling one kernel at a time with Nsight Compute.

    python -m paper_2604_25138_gb300.profile_cases operator --n 16384 --precision bf16x3 --reps 5
    python -m paper_2604_25138_gb300.profile_cases fit --n 16384
    python -m paper_2604_25138_gb300.profile_cases solve --n 16384
    python -m paper_2604_25138_gb300.profile_cases residual --n 16384 --d 64 --reps 3

`operator` builds the operator of the benchmark instance (clustered layout,
d = 32, lambda = 1e-4) and applies it `reps` times; `fit` builds it and fits
the CCCP preconditioner only (printing how many kernels ran before the fit, for
a launch window over the fit); `solve` also fits the CCCP
preconditioner (N_r from the default schedule) and runs the mixed PCG solve;
`map` evaluates the radio map on a grid of m points; `residual` applies the
float64-accurate product (the true residual of mixed solves) `reps` times.  All inputs are the seeded
synthetic ones of `synth.py`; nothing here is timed for reporting.
"""
import argparse

import numpy as np
import torch

from . import laker as L
from . import synth

PRECISIONS = {"fp64": L.FP64, "fp32": L.FP32, "bf16x3": L.BF16X3}
VARIANTS = {"auto": L.AUTO, "materialised": L.MATERIALISED, "matrix-free": L.MATRIX_FREE}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["operator", "fit", "solve", "map", "residual"])
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--d", type=int, default=32)
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default="bf16x3")
    ap.add_argument("--variant", choices=sorted(VARIANTS), default="auto")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--seed", type=int, default=2000)
    a = ap.parse_args(argv)

    inst = synth.make_instance(a.n, a.d, 1e-4, n_tx=8, seed=a.seed, layout="clustered", grid=a.grid)
    dev = lambda x: torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    ctx = L.Context(0)
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, PRECISIONS[a.precision], VARIANTS[a.variant])
    if a.case in ("operator", "residual"):
        x = dev(synth.random_vector(a.n, a.seed))
        w = torch.empty_like(x)
        for _ in range(a.reps):
            L.laker_op_matvec(ctx, op, x, w, fp64=(a.case == "residual"))
        torch.cuda.synchronize()
        print(f"{a.case} n={a.n} d={a.d} {a.precision}: {a.reps} products, |w| = {float(w.norm()):.6e}")
        return
    Z = dev(synth.directions(a.n, synth.default_num_directions(a.n), a.seed))
    torch.cuda.synchronize()
    print(f"launches before fit {ctx.launches()}", flush=True)
    P = L.laker_fit_preconditioner(ctx, op, Z)
    torch.cuda.synchronize()
    if a.case == "fit":
        print(f"fit n={a.n} {a.precision}: {P.info}, launches after fit {ctx.launches()}")
        return
    print(f"launches before solve {ctx.launches()}", flush=True)
    if a.case == "solve":
        alpha, info = L.laker_pcg_solve(ctx, op, P, dev(inst.y), 1e-6, max_iter=20000, refine_every=20)
        print(f"solve n={a.n} {a.precision}: {info}")
        return
    alpha, info = L.laker_pcg_solve(ctx, op, P, dev(inst.y), 1e-6, max_iter=20000, refine_every=20)
    out = L.laker_eval_map(ctx, op, dev(inst.Qg), alpha)
    torch.cuda.synchronize()
    print(f"map n={a.n} m={out.numel()}: mean {float(out.mean()):.6e}")


if __name__ == "__main__":
    main()
