"""Concurrent single-instance solves (laker_pcg_solve_concurrent): many
independent PCG solves of Algorithm 1, one per instance, on several streams.

Each instance runs exactly the single-instance solver's arithmetic (fixed-order
reductions, the same launch shapes), so its alpha must equal laker_pcg_solve's
bit for bit whatever the stream it ran on and whatever ran beside it; float64
instances must also reproduce the oracle's PCG (1e-9 at tol 1e-10), and mixed
ones meet the true relative residual 1e-6 under the oracle's dense operator."""
import numpy as np
import pytest
import torch

from oracle import laker_oracle as O
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


def test_fp64_instances_match_single_solves_and_the_oracle(L, ctx):
    from tests.gpu_util import dev, host
    spec = [(300, 16, 1e-1, "cccp"), (513, 16, 1e-2, "jacobi"), (64, 8, 1.0, "none"), (1000, 16, 1e-1, "cccp"),
            (777, 32, 1e-2, "cccp"), (129, 16, 1e-1, "jacobi"), (450, 16, 1e-2, "cccp")]
    items, keep, refs = [], [], []
    for k, (n, d, lam, kind) in enumerate(spec):
        inst = synth.make_instance(n, d, lam, n_tx=1 + k % 8, seed=1700 + k, grid=2)
        A = O.system_matrix(inst.Q, inst.scale, inst.lam)
        op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.FP64)
        if kind == "cccp":
            Z = synth.directions(n, min(n, 64), 1800 + k)
            P = L.laker_fit_preconditioner(ctx, op, dev(Z))
            Pd = O.inverse_sqrt(O.cccp_fit(O.random_directions(A, Z), 0.1, O.shrinkage_rho(n, Z.shape[1], 0.1),
                                           1e-8).Sigma)
        elif kind == "jacobi":
            P, Pd = L.laker_precond_jacobi(ctx, op), O.jacobi_preconditioner(A)
        else:
            P, Pd = None, None
        y = dev(inst.y)
        keep.append((op, P))
        items.append((op, P, y, None))
        refs.append((A, inst.y, Pd))
    alphas, infos, done = L.laker_pcg_solve_concurrent(ctx, items, 1e-10, max_iter=20000, streams=4)
    for (op, P, y, _), a, f, (A, yy, Pd) in zip(items, alphas, infos, refs):
        single, fs = L.laker_pcg_solve(ctx, op, P, y, 1e-10, max_iter=20000)
        torch.cuda.synchronize()
        assert torch.equal(a, single)
        assert f["iterations"] == fs["iterations"] and f["converged"] == 1
        ref = O.pcg(A, yy, Pd, 1e-10).alpha
        np.testing.assert_allclose(host(a), ref, rtol=0, atol=1e-9 * np.abs(ref).max())
    assert len(done) == len(items) and min(done) > 0.0


def test_mixed_instances_of_every_kind_in_one_call(L, ctx):
    """FP32 materialised, FP32 matrix-free and split-bf16 operators side by
    side: each alpha equals its single solve, and the true residual (oracle's
    dense operator) meets 1e-6."""
    from tests.gpu_util import dev, host
    kinds = [(L.FP32, L.MATERIALISED), (L.BF16X3, L.MATRIX_FREE), (L.FP32, L.MATRIX_FREE)] * 3
    items, keep, refs = [], [], []
    rng = np.random.default_rng(5)
    for k, (prec, var) in enumerate(kinds):
        n = int(rng.integers(600, 2400))
        lam = float(10 ** rng.uniform(-4, -2))
        inst = synth.make_instance(n, 32, lam, n_tx=1 + k % 8, seed=1900 + k, grid=2)
        op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, prec, var)
        P = L.laker_fit_preconditioner(ctx, op, dev(synth.directions(n, synth.default_num_directions(n), 1900 + k)))
        keep.append((op, P))
        items.append((op, P, dev(inst.y), None))
        refs.append(inst)
    alphas, infos, _ = L.laker_pcg_solve_concurrent(ctx, items, 1e-6, max_iter=40000, refine_every=20, streams=6)
    for (op, P, y, _), a, f, inst in zip(items, alphas, infos, refs):
        single, fs = L.laker_pcg_solve(ctx, op, P, y, 1e-6, max_iter=40000, refine_every=20)
        torch.cuda.synchronize()
        assert torch.equal(a, single) and f["iterations"] == fs["iterations"]
        A = O.system_matrix(inst.Q, inst.scale, inst.lam)
        assert f["converged"] == 1
        assert O.relative_residual(A, host(a), inst.y) <= 1e-6 * 1.01


def test_errors_and_partial_failure(L, ctx):
    from tests.gpu_util import dev
    inst = synth.make_instance(700, 16, 1e-3, seed=2100, grid=2)
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.BF16X3)
    y = dev(inst.y)
    with pytest.raises(L.LakerError) as e:
        L.laker_pcg_solve_concurrent(ctx, [(op, None, y, None), (op, None, y, None)], 1e-6, refine_every=20)
    assert e.value.status == L.ERR_ARG
    # one instance capped at 5 products: MAXITER overall, the others converge
    ops = [L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.FP64) for _ in range(3)]
    items = [(o, None, y, None) for o in ops]
    alphas, infos, _ = L.laker_pcg_solve_concurrent(ctx, items, 1e-8, max_iter=5, streams=3, allow_maxiter=True)
    assert all(f["converged"] == 0 and f["iterations"] == 5 for f in infos)
    with pytest.raises(L.LakerError) as e:
        L.laker_pcg_solve_concurrent(ctx, items, 1e-8, max_iter=20000, streams=0)
    assert e.value.status == L.ERR_ARG
