"""GPU parity of the boundary's added calls against the oracle:

* the device-drawn random directions (Philox4x32-10 words bit for bit, the
  Gaussian directions to rounding) and the seeded CCCP fit;
* gradient descent on R(alpha), the paper's first-order baseline (Sec. V-A);
* PCG stopped on the objective gap (Eq. iterations, TAR.TOL = 1e-3) and the
  prediction discrepancy (Eq. prediction-discrepancy);
* the set network's checkpoint (save, load, resumed training);
* a bounded device wait run out on purpose through a tiny wait budget.
"""
import os
import tempfile

import numpy as np
import pytest

from oracle import laker_oracle as O
from oracle import philox as X
from paper_2604_25138_gb300 import synth
from tests.pcg_envelope import gap_envelope, within_envelope

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
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("key,c0,count", [(0, 0, 1), (0xFFFFFFFFFFFFFFFF, (1 << 32) - 3, 7), (20260, 12345, 1000)])
def test_philox_words_bit_exact(L, ctx, key, c0, count):
    got = L.laker_philox4x32_10(ctx, key, c0, count).cpu().numpy().astype(np.uint64)
    want = X.philox_blocks(key, c0, count).astype(np.uint64)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("seed,n,n_r", [(7, 1, 1), (2026, 333, 17), (1 << 40, 4097, 64)])
def test_random_directions_match_oracle(L, ctx, seed, n, n_r):
    Z = L.laker_random_directions(ctx, seed, n, n_r).cpu().numpy()
    Zo = X.gaussian_directions(seed, n, n_r)
    # same uniforms bit for bit; log / sin / cos of two libraries differ by ulps
    assert np.max(np.abs(Z - Zo)) <= 1e-13 * max(1.0, np.max(np.abs(Zo)))


def test_seeded_fit_equals_fit_with_oracle_directions(L, ctx):
    n, n_r, seed = 300, 40, 99
    inst = synth.make_instance(n, 8, 1e-2, seed=5, grid=2)
    op = L.laker_build_kernel(ctx, _dev(inst.Q), inst.scale, inst.lam, L.FP64)
    Ps = L.laker_fit_preconditioner_seeded(ctx, op, seed, n_r)
    Pz = L.laker_fit_preconditioner(ctx, op, _dev(X.gaussian_directions(seed, n, n_r)))
    cs, Ds, Us = L.laker_precond_export(ctx, Ps)
    cz, Dz, Uz = L.laker_precond_export(ctx, Pz)
    assert abs(cs - cz) <= 1e-12 * cz
    assert float((Us - Uz).abs().max()) <= 1e-11
    assert Ps.info["iterations"] == Pz.info["iterations"]
    # and against the dense oracle fit on the oracle's own directions
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    ref = O.cccp_fit(O.random_directions(A, X.gaussian_directions(seed, n, n_r)), 0.1,
                     O.shrinkage_rho(n, n_r, 0.1), 1e-8)
    U = Us.cpu().numpy()
    Sigma = cs * np.eye(n) + (U * Ds.cpu().numpy()) @ U.T
    assert np.linalg.norm(Sigma - ref.Sigma) <= 1e-9 * np.linalg.norm(ref.Sigma)


@pytest.mark.parametrize("n,lam,steps", [(200, 1e-2, 50), (777, 1e-3, 40)])
def test_gradient_descent_matches_oracle(L, ctx, n, lam, steps):
    """Same step size, same number of steps: the GPU iterates equal the oracle's
    (float64 operator; GD is a contraction, so rounding does not grow)."""
    inst = synth.make_instance(n, 16, lam, seed=11 + n, grid=2)
    G = O.kernel_matrix(inst.Q, inst.scale)
    op = L.laker_build_kernel(ctx, _dev(inst.Q), inst.scale, inst.lam, L.FP64)
    mu_ref = float(np.linalg.eigvalsh(G)[-1])
    mu = L.laker_op_lambda_max(ctx, op, 50)
    assert abs(mu - mu_ref) <= 1e-9 * mu_ref
    alpha, info, eta, trace = L.laker_gd_solve(ctx, op, _dev(inst.y), eta=0.0, tol=0.0, max_iter=steps,
                                              trace_cap=steps)
    assert abs(eta - 1.0 / (2 * mu_ref * (mu_ref + lam))) <= 1e-8 * eta
    ref = O.gradient_descent(G, inst.y, inst.lam, eta, steps)
    assert info["iterations"] == steps and not info["converged"]
    a = alpha.cpu().numpy()
    assert np.linalg.norm(a - ref.alpha) <= 1e-11 * np.linalg.norm(ref.alpha)
    np.testing.assert_allclose(trace[:, 1], ref.R, rtol=1e-10)
    np.testing.assert_allclose(np.sqrt(trace[:, 0]), ref.rel_res, rtol=1e-8)
    # the paper's observation: GD stalls far from the solution on these systems
    A = G + lam * np.eye(n)
    assert O.relative_residual(A, a, inst.y) > 1e-3


@pytest.mark.parametrize("n,lam,prec", [(400, 1e-1, "cccp"), (1024, 1e-2, "cccp"), (500, 1e-2, "jacobi")])
def test_gap_stop_matches_oracle(L, ctx, n, lam, prec):
    """The solve stops at the first product whose objective gap to the
    reference R is <= 1e-3: the returned alpha meets the gap, the iterate one
    product earlier does not (checked by the oracle), and the index lies in
    the oracle's own rounding envelope of it, widened by its width (the gap
    oscillates near the threshold, so rounding decides the index)."""
    inst = synth.make_instance(n, 16, lam, seed=41, grid=4)
    G = O.kernel_matrix(inst.Q, inst.scale)
    A = G + inst.lam * np.eye(n)
    op = L.laker_build_kernel(ctx, _dev(inst.Q), inst.scale, inst.lam, L.FP64)
    if prec == "cccp":
        Z = synth.directions(n, 64, 41)
        P = L.laker_fit_preconditioner(ctx, op, _dev(Z))
        Pd = O.inverse_sqrt(O.cccp_fit(O.random_directions(A, Z), 0.1, O.shrinkage_rho(n, 64, 0.1), 1e-8).Sigma)
    else:
        P = L.laker_precond_jacobi(ctx, op)
        Pd = O.jacobi_preconditioner(A)
    R_ref = O.objective_R(G, O.solve_direct(A, inst.y), inst.y, inst.lam)
    alpha, info = L.laker_pcg_solve_gap(ctx, op, P, _dev(inst.y), R_ref, gap=1e-3)
    v = synth.random_vector(n, 4)
    pv_err = np.linalg.norm(L.laker_precond_apply(ctx, P, _dev(v)).cpu().numpy() - Pd @ v) / np.linalg.norm(Pd @ v)
    assert pv_err < 1e-7
    env = gap_envelope(A, G, inst.y, Pd, inst.lam, R_ref, 1e-3, 2000, p_rel=max(pv_err, 1e-15))
    assert env is not None
    assert info["converged"] == 1 and within_envelope(info["iterations"], env), (info, env)
    k = info["iterations"]
    if k > 1:   # the stop is the first crossing of the GPU's own iterates
        a_p, _ = L.laker_pcg_solve(ctx, op, P, _dev(inst.y), 0.0, max_iter=k - 1, allow_maxiter=True)
        assert O.objective_gap(G, a_p.cpu().numpy(), O.solve_direct(A, inst.y), inst.y, inst.lam) > 1e-3 * (1 - 1e-9)
    assert O.objective_gap(G, alpha.cpu().numpy(), O.solve_direct(A, inst.y), inst.y, inst.lam) <= 1e-3 * (1 + 1e-6)


def test_prediction_discrepancy_matches_oracle(L, ctx):
    n = 900
    inst = synth.make_instance(n, 16, 1e-3, seed=12, grid=2)
    G = O.kernel_matrix(inst.Q, inst.scale)
    A = G + inst.lam * np.eye(n)
    a_star = O.solve_direct(A, inst.y)
    a = O.pcg(A, inst.y, None, 0.0, max_iter=30).alpha
    for prec in ("FP64", "FP32"):
        op = L.laker_build_kernel(ctx, _dev(inst.Q), inst.scale, inst.lam, getattr(L, prec))
        pd = L.laker_prediction_discrepancy(ctx, op, _dev(a), _dev(a_star))
        want = O.prediction_discrepancy(G, a, a_star)
        assert abs(pd - want) <= 1e-9 * want, (prec, pd, want)


def test_setnet_checkpoint_roundtrip_and_resume(L, ctx):
    """Save after three Adam steps, load into a new network, take one more step
    on both: identical loss and identical parameters."""
    import torch
    d = 8
    insts = [synth.make_instance(n, d, 1e-3, seed=60 + n, grid=2) for n in (150, 230)]
    Xs = [L.laker_setnet_point_features(ctx, _dev(i.X), _dev(i.Q), _dev(i.y)) for i in insts]
    X_all = torch.cat(Xs)
    F = torch.randn(10, 2, dtype=torch.float32, device="cuda")
    tc = torch.tensor([0.3, -0.2], dtype=torch.float32, device="cuda")
    tD = torch.randn(10, dtype=torch.float32, device="cuda")
    net = L.SetNet(ctx, d + 3, 32, 16, seed=3)
    args = (X_all, [150, 230], F, [4, 6], tc, tD, 1e-3)
    for _ in range(3):
        L.laker_setnet_train_step(ctx, net, *args)
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "net.ckpt")
        net.save(path)
        net2 = L.SetNet.load(ctx, path, d + 3, 32, 16)
        with open(path, "rb") as f:
            assert f.read(8) == b"LAKERSN1"
        bad = os.path.join(tmp, "bad.ckpt")
        with open(bad, "wb") as f:
            f.write(b"not a checkpoint")
        with pytest.raises(L.LakerError) as e:
            L.SetNet.load(ctx, bad, d + 3, 32, 16)
        assert e.value.status == L.ERR_ARG
    assert np.array_equal(net.get_params(), net2.get_params())
    l1 = L.laker_setnet_train_step(ctx, net, *args)
    l2 = L.laker_setnet_train_step(ctx, net2, *args)
    assert l1 == l2
    assert np.array_equal(net.get_params(), net2.get_params())


def test_bounded_wait_runs_out_and_context_survives(L, ctx):
    """A wait budget of 64 cycles makes the batched solver's grid-barrier waits
    run out (nothing can complete a barrier that fast): the call returns
    LAKER_ERR_TIMEOUT through the kernel's status word, every block leaves,
    and with the default budget restored the same batch solves."""
    items = []
    for k, n in enumerate((300, 517)):
        inst = synth.make_instance(n, 16, 1e-2, seed=80 + k, grid=2)
        op = L.laker_build_kernel(ctx, _dev(inst.Q), inst.scale, inst.lam, L.FP64)
        items.append((op, None, _dev(inst.y), None))
    L.laker_set_wait_budget(ctx, 64)
    try:
        with pytest.raises(L.LakerError) as e:
            L.laker_pcg_solve_batched(ctx, items, 1e-8, max_iter=5000)
        assert e.value.status == L.ERR_TIMEOUT
    finally:
        L.laker_set_wait_budget(ctx, 0)
    alphas, infos, _ = L.laker_pcg_solve_batched(ctx, items, 1e-8, max_iter=5000)
    assert all(i["converged"] == 1 for i in infos)
