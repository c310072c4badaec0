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
float64-accurate product (the true residual of mixed solves) `reps` times;
`batched` builds `--count` float32 operators (n uniform in [1024, 4096],
d = 32, lambda log-uniform in [1e-5, 1e-2], 1-8 Tx), fits their CCCP
preconditioners and runs one persistent batched solve to 1e-6, printing the
per-instance products and stop times.  All inputs are the seeded synthetic
ones of `synth.py`; nothing here is timed for reporting.
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
    ap.add_argument("case", choices=["operator", "fit", "solve", "map", "residual", "batched"])
    ap.add_argument("--count", type=int, default=24)
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--d", type=int, default=32)
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default="bf16x3")
    ap.add_argument("--variant", choices=sorted(VARIANTS), default="auto")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--seed", type=int, default=2000)
    a = ap.parse_args(argv)

    dev = lambda x: torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    ctx = L.Context(0)
    if a.case == "batched":
        rng = np.random.default_rng(a.seed)
        items, keep = [], []
        for k in range(a.count):
            n = int(rng.integers(1024, 4097))
            lam = float(10 ** rng.uniform(-5, -2))
            bi = synth.make_instance(n, 32, lam, n_tx=int(rng.integers(1, 9)), seed=a.seed + k, grid=2)
            op = L.laker_build_kernel(ctx, dev(bi.Q), bi.scale, bi.lam, L.FP32, L.MATERIALISED)
            P = L.laker_fit_preconditioner(ctx, op, dev(synth.directions(n, synth.default_num_directions(n), bi.seed)))
            keep.append((op, P))
            items.append((op, P, dev(bi.y), None))
        torch.cuda.synchronize()
        _, infos, done = L.laker_pcg_solve_batched(ctx, items, 1e-6, max_iter=20000, refine_every=20)
        print("batched %d: products %s" % (a.count, [f["iterations"] for f in infos]))
        print("stop ms %s" % [round(x, 2) for x in done])
        return
    inst = synth.make_instance(a.n, a.d, 1e-4, n_tx=8, seed=a.seed, layout="clustered", grid=a.grid)
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
