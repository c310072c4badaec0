"""Data, training and evaluation around the learned set network.

Every numerical step runs in liblaker (operator build, CCCP fit, feature
assembly, the network's forward / backward / Adam kernels, PCG); this module
only moves tensors between those calls and keeps the bookkeeping:

* ``fit_example`` fits the CCCP preconditioner of one instance (cold start)
  and returns the network's inputs (point and direction features) and targets
  (log c, log D_k);
* ``train`` runs Adam over mini-batches of such examples;
* ``compare`` solves held-out instances with the cold CCCP fit, the warm
  started fit, the network's prediction used directly, Jacobi and no
  preconditioner, and applies the fallback rule (CCCP is used whenever the
  prediction needs more than 1.2 times CCCP's PCG iterations).
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from . import laker as L
from . import synth


@dataclasses.dataclass
class Example:
    X: torch.Tensor        # n x (d + 3) float32 point features (device)
    F: torch.Tensor        # n_r x 2 float32 direction features (device)
    logc: float
    logD: torch.Tensor     # n_r float32 (device)
    cccp_iterations: int


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def instance_inputs(ctx, inst, side: float = 1000.0):
    """Point features of an instance: [location / L, q, y]."""
    return L.laker_setnet_point_features(ctx, _dev(inst.X / side), _dev(inst.Q), _dev(inst.y))


def fit_example(ctx, inst, precision=L.FP32, n_r=None, seed=0) -> Example:
    n_r = n_r or synth.default_num_directions(inst.n)
    op = L.laker_build_kernel(ctx, _dev(inst.Q), inst.scale, inst.lam, precision)
    P = L.laker_fit_preconditioner(ctx, op, _dev(synth.directions(inst.n, n_r, seed)))
    c, D, _ = L.laker_precond_export(ctx, P)
    F = L.laker_precond_direction_features(ctx, P)
    X = instance_inputs(ctx, inst)
    ex = Example(X=X, F=F, logc=float(np.log(c)),
                 logD=(torch.log(torch.clamp(D, min=1e-30)) + float(np.log(n_r / inst.n))).to(torch.float32),
                 cccp_iterations=P.info["iterations"])
    P.close()
    op.close()
    return ex


def batch_tensors(examples):
    X = torch.cat([e.X for e in examples]).contiguous()
    F = torch.cat([e.F for e in examples]).contiguous()
    tc = torch.tensor([e.logc for e in examples], dtype=torch.float32, device="cuda")
    tD = torch.cat([e.logD for e in examples]).contiguous()
    return X, [e.X.shape[0] for e in examples], F, [e.F.shape[0] for e in examples], tc, tD


def train(ctx, net, examples, steps: int, batch: int = 8, lr: float = 1e-3, seed: int = 0):
    rng = np.random.default_rng(seed)
    losses = []
    for _ in range(steps):
        idx = rng.choice(len(examples), size=min(batch, len(examples)), replace=False)
        X, npts, F, ndir, tc, tD = batch_tensors([examples[i] for i in idx])
        losses.append(L.laker_setnet_train_step(ctx, net, X, npts, F, ndir, tc, tD, lr))
    return losses


def compare(ctx, net, inst, tol: float = 1e-6, precision=L.FP32, n_r=None, seed=0, refine_every: int = 20):
    """PCG iterations, times and the Lanczos estimate of kappa(P A) for one
    instance under the cold CCCP fit, the warm-started fit, the prediction used
    directly, Jacobi and none."""
    n_r = n_r or synth.default_num_directions(inst.n)
    op = L.laker_build_kernel(ctx, _dev(inst.Q), inst.scale, inst.lam, precision)
    Z = _dev(synth.directions(inst.n, n_r, seed))
    y = _dev(inst.y)
    X = instance_inputs(ctx, inst)
    out = {}

    def run(name, make):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        P = make()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        _, info = L.laker_pcg_solve(ctx, op, P, y, tol, max_iter=50000, refine_every=refine_every,
                                    allow_maxiter=True)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        # kappa(P A) from the Lanczos tridiagonal of an untimed traced solve
        # (at most 2000 products: a lower estimate for the slow preconditioners)
        _, _, tr = L.laker_pcg_solve_trace(ctx, op, P, y, tol, max_iter=2000, refine_every=refine_every,
                                           allow_maxiter=True)
        lo, hi = L.laker_lanczos_extremes(tr)
        out[name] = dict(fit_s=t1 - t0, solve_s=t2 - t1, iterations=info["iterations"],
                         converged=info["converged"], rel_res_true=info["rel_res_true"],
                         cccp_iterations=(P.info.get("iterations") if P is not None else 0),
                         kappa_PA=(hi / lo) if lo > 0 else float("inf"))
        if P is not None:
            P.close()

    run("cccp", lambda: L.laker_fit_preconditioner(ctx, op, Z))
    run("warm", lambda: L.laker_fit_preconditioner_learned(ctx, op, Z, net, X, mode=0))
    run("learned", lambda: L.laker_fit_preconditioner_learned(ctx, op, Z, net, X, mode=1))
    run("jacobi", lambda: L.laker_precond_jacobi(ctx, op))
    run("none", lambda: None)
    out["fallback"] = out["learned"]["iterations"] > 1.2 * out["cccp"]["iterations"]
    op.close()
    return out
