"""The guard of the mixed forms' residual replacement (the PCG stage of
Algorithm 1 with an inexact operator between float64-accurate residuals).

On the 16384-point clustered instance (d = 32, lambda = 1e-4) the split-bf16
operator differs from the float64 one by more than lambda along the bottom of
the spectrum.  With a replacement only every 200 products, CG resolves those
directions with the inexact operator and the unguarded iteration broke down
(p^T A~ p <= 0).  The guard rolls back to the lowest-residual iterate, restarts
the direction and halves the interval; the solve must then still reach the
true relative residual 1e-6.  At the default interval of 20 the guard must
stay idle."""
import numpy as np
import pytest

from paper_2604_25138_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2604_25138_gb300 import build, laker
    build.build()
    return laker


@pytest.fixture(scope="module")
def ctx(L):
    return L.Context(0)


@pytest.fixture(scope="module")
def problem(L, ctx):
    from tests.gpu_util import dev
    n = 16384
    inst = synth.make_instance(n, 32, 1e-4, n_tx=8, seed=2000, layout="clustered", grid=2)
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.BF16X3)
    P = L.laker_fit_preconditioner(ctx, op, dev(synth.directions(n, synth.default_num_directions(n), 2000)))
    yield inst, op, P, dev(inst.y)
    P.close()
    op.close()


def _true_rel_res(L, ctx, op, y, alpha):
    import torch
    w = torch.empty_like(alpha)
    with ctx:
        ctx.check(L.library().laker_op_matvec_fp64(ctx.handle, op.handle, L._ptr(alpha, "alpha", op.n),
                                                     L._ptr(w, "w", op.n)))
    torch.cuda.synchronize()
    return float((y - w).norm() / y.norm())


def test_default_interval_leaves_the_guard_idle(L, ctx, problem):
    inst, op, P, y = problem
    alpha, info = L.laker_pcg_solve(ctx, op, P, y, 1e-6, max_iter=40000, refine_every=20)
    assert info["converged"] == 1 and info["restarts"] == 0
    assert info["rel_res_true"] <= 1e-6
    assert _true_rel_res(L, ctx, op, y, alpha) <= 1e-6 * (1 + 1e-6)


def test_long_interval_recovers_through_the_guard(L, ctx, problem):
    inst, op, P, y = problem
    alpha, info = L.laker_pcg_solve(ctx, op, P, y, 1e-6, max_iter=40000, refine_every=200)
    assert info["converged"] == 1, info
    assert info["restarts"] >= 1, info
    assert _true_rel_res(L, ctx, op, y, alpha) <= 1e-6 * (1 + 1e-6)


def test_unreachable_tolerance_returns_the_lowest_energy_iterate(L, ctx, problem):
    """A tolerance below the operator's accuracy floor ends in stagnation (or
    max_iter) with the iterate of the lowest true residual seen, which is
    finite and well below the zero start's."""
    inst, op, P, y = problem
    alpha, info = L.laker_pcg_solve(ctx, op, P, y, 1e-14, max_iter=6000, refine_every=20, allow_maxiter=True)
    assert info["converged"] == 0
    r = _true_rel_res(L, ctx, op, y, alpha)
    assert np.isfinite(r) and r < 1e-3, (r, info)
