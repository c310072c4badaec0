"""Streaming update (the paper's future work, Sec. VI: measurements that
arrive sequentially): operator append, warm-started PCG and warm-started CCCP
on the GPU against the oracle.

* laker_op_append must give, bit for bit, the products of a fresh build on
  the concatenated embeddings (it copies the old entries and evaluates the
  rest with the same kernels), for every precision, on ragged and aligned
  splits.
* Warm-started PCG (float64 operator): the iterates after k products equal
  the oracle's warm-started PCG from the same start (to 1e-9, before CG's
  rounding divergence sets in); a start that meets the tolerance stops at 0.
* Warm-started CCCP (float64 operator): the oracle runs its own chain (cold
  fit on the old points, its (c, D) in coefficient form, warm fit on the
  grown set) and
  the GPU its own; both reach the same Sigma_* (to 1e-8) and the GPU's warm
  fit needs fewer iterations than its cold fit.
* A mixed streaming sequence reaches the true residual 1e-6 (checked with the
  oracle's dense operator) at each step."""
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


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("prec,var,d", [("FP64", "MATERIALISED", 16), ("FP32", "MATERIALISED", 16),
                                        ("FP32", "MATERIALISED", 80), ("FP32", "MATRIX_FREE", 32),
                                        ("BF16X3", "MATRIX_FREE", 64), ("BF16X3", "MATRIX_FREE", 20)])
@pytest.mark.parametrize("n0,m", [(300, 77), (256, 1), (384, 300), (1, 129)])
def test_append_equals_fresh_build(L, ctx, prec, var, d, n0, m):
    inst = synth.make_instance(n0 + m, d, 1e-3, seed=17, grid=2)
    Q = _dev(inst.Q)
    P, V = getattr(L, prec), getattr(L, var)
    op0 = L.laker_build_kernel(ctx, Q[:n0].contiguous(), inst.scale, inst.lam, P, V)
    op1 = L.laker_op_append(ctx, op0, Q[n0:].contiguous())
    ref = L.laker_build_kernel(ctx, Q, inst.scale, inst.lam, P, V)
    assert op1.n == n0 + m
    x = _dev(synth.random_vector(n0 + m, 5))
    for fp64 in (False, True):
        a = L.laker_op_matvec(ctx, op1, x, fp64=fp64)
        b = L.laker_op_matvec(ctx, ref, x, fp64=fp64)
        torch.cuda.synchronize()
        assert torch.equal(a, b), (fp64, float((a - b).abs().max()))
    # the old operator is untouched
    x0 = x[:n0].contiguous()
    w0 = L.laker_op_matvec(ctx, op0, x0, fp64=True)
    A0 = O.system_matrix(inst.Q[:n0], inst.scale, inst.lam)
    torch.cuda.synchronize()
    np.testing.assert_allclose(w0.cpu().numpy(), A0 @ x0.cpu().numpy(), rtol=1e-10,
                               atol=1e-10 * np.abs(A0).sum(axis=1).max() * float(x0.abs().max()))
    for o in (op0, op1, ref):
        o.close()


def test_warm_pcg_iterates_match_the_oracle(L, ctx):
    n = 700
    inst = synth.make_instance(n, 16, 1e-3, seed=23, grid=2)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    op = L.laker_build_kernel(ctx, _dev(inst.Q), inst.scale, inst.lam, L.FP64)
    Pj = L.laker_precond_jacobi(ctx, op)
    Pd = O.jacobi_preconditioner(A)
    a0 = 0.3 * synth.random_vector(n, 8)
    y = _dev(inst.y)
    for k in (1, 4, 12):
        ag, info = L.laker_pcg_solve_warm(ctx, op, Pj, y, _dev(a0), 0.0, max_iter=k, allow_maxiter=True)
        ao = O.pcg(A, inst.y, Pd, 0.0, max_iter=k, alpha0=a0).alpha
        assert info["iterations"] == k
        np.testing.assert_allclose(ag.cpu().numpy(), ao, rtol=0, atol=1e-9 * np.abs(ao).max())
    # the whole solve: converged, true residual, and the warm start from the
    # answer stops before any product
    a, info = L.laker_pcg_solve_warm(ctx, op, Pj, y, _dev(a0), 1e-8, max_iter=20000)
    assert info["converged"] == 1
    assert O.relative_residual(A, a.cpu().numpy(), inst.y) <= 1e-8 * (1 + 1e-6)
    a2, info2 = L.laker_pcg_solve_warm(ctx, op, Pj, y, a, 1e-7, max_iter=20000)
    assert info2["iterations"] == 0 and torch.equal(a2, a)
    Pj.close()
    op.close()


def test_warm_cccp_matches_the_oracle_chain(L, ctx):
    n0, m = 480, 64
    n = n0 + m
    n_r = synth.default_num_directions(n0)
    inst = synth.make_instance(n, 16, 1e-3, seed=29, grid=2)
    Z = synth.directions(n, n_r, 29)
    gamma, eps = 0.1, 1e-8
    # GPU chain
    op0 = L.laker_build_kernel(ctx, _dev(inst.Q[:n0]), inst.scale, inst.lam, L.FP64)
    P0 = L.laker_fit_preconditioner(ctx, op0, _dev(Z[:n0]))
    op1 = L.laker_op_append(ctx, op0, _dev(inst.Q[n0:]))
    P1 = L.laker_fit_preconditioner_warm(ctx, op1, _dev(Z), P0)
    P1c = L.laker_fit_preconditioner(ctx, op1, _dev(Z))
    c1, D1, U1 = L.laker_precond_export(ctx, P1)
    U1 = U1.cpu().numpy()
    S_gpu = c1 * np.eye(n) + (U1 * D1.cpu().numpy()) @ U1.T
    # oracle chain, from the oracle's own cold fit on the old points
    A0 = O.system_matrix(inst.Q[:n0], inst.scale, inst.lam)
    Ub0 = O.random_directions(A0, Z[:n0])
    rho0 = O.shrinkage_rho(n0, n_r, gamma)
    fit0 = O.cccp_fit(Ub0, gamma, rho0, eps, tol=1e-10)
    c0, D0 = O.cccp_step_coefficients(fit0.Sigma, Ub0, gamma, rho0, eps)
    A1 = O.system_matrix(inst.Q, inst.scale, inst.lam)
    Ub1 = O.random_directions(A1, Z)
    rho1 = O.shrinkage_rho(n, n_r, gamma)
    fit1 = O.cccp_fit(Ub1, gamma, rho1, eps, tol=1e-10, Sigma0=O.warm_sigma0(Ub1, c0, D0))
    cold1 = O.cccp_fit(Ub1, gamma, rho1, eps, tol=1e-10)
    assert fit1.converged and P1.info["converged"] == 1
    np.testing.assert_allclose(S_gpu, fit1.Sigma, rtol=0, atol=1e-8 * np.abs(fit1.Sigma).max())
    assert abs(P1.info["iterations"] - fit1.iterations) <= 1, (P1.info["iterations"], fit1.iterations)
    assert P1.info["iterations"] < P1c.info["iterations"], (P1.info, P1c.info)
    assert fit1.iterations < cold1.iterations
    for o in (P0, P1, P1c, op0, op1):
        o.close()


def test_mixed_streaming_sequence(L, ctx):
    """n0 = 3000 points, then three batches of 256: append, warm fit, warm
    solve to the true residual 1e-6 each time (mixed split-bf16 operator)."""
    n0, m, steps = 3000, 256, 3
    n = n0 + steps * m
    inst = synth.make_instance(n, 32, 1e-4, n_tx=4, seed=31, grid=2)
    n_r = synth.default_num_directions(n0)
    Z = synth.directions(n, n_r, 31)
    op = L.laker_build_kernel(ctx, _dev(inst.Q[:n0]), inst.scale, inst.lam, L.BF16X3)
    P = L.laker_fit_preconditioner(ctx, op, _dev(Z[:n0]))
    alpha, info = L.laker_pcg_solve(ctx, op, P, _dev(inst.y[:n0]), 1e-6, max_iter=20000, refine_every=20)
    for s in range(steps):
        k = n0 + (s + 1) * m
        op1 = L.laker_op_append(ctx, op, _dev(inst.Q[k - m:k]))
        P1 = L.laker_fit_preconditioner_warm(ctx, op1, _dev(Z[:k]), P)
        a0 = torch.cat([alpha, torch.zeros(m, dtype=torch.float64, device="cuda")])
        alpha, info = L.laker_pcg_solve_warm(ctx, op1, P1, _dev(inst.y[:k]), a0, 1e-6, max_iter=20000,
                                             refine_every=20)
        A = O.system_matrix(inst.Q[:k], inst.scale, inst.lam)
        assert info["converged"] == 1
        assert O.relative_residual(A, alpha.cpu().numpy(), inst.y[:k]) <= 1e-6 * 1.01
        for o in (P, op):
            o.close()
        op, P = op1, P1
    P.close()
    op.close()
