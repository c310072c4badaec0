"""The PCG trace and the paper's numerical-layer metrics (Sec. V-A) on the GPU
against the float64 oracle: per-product objective R(alpha_k) (Eq.
simu-R-definition) and recursive residual, iterations to the objective gap
TAR.TOL = 1e-3 (Eq. iterations), and the condition-number estimate
kappa(P A) from the Lanczos tridiagonal of the PCG coefficients against the
oracle's dense eigenvalues."""
import numpy as np
import pytest

from oracle import laker_oracle as O
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


def _oracle_iterates(A, y, P, kmax):
    """alpha after each of the first kmax products of the oracle's PCG."""
    return [O.pcg(A, y, P, 0.0, max_iter=k).alpha for k in range(1, kmax + 1)]


@pytest.mark.parametrize("n,lam", [(400, 1e-1), (1024, 1e-2)])
def test_trace_matches_oracle_and_metrics(L, ctx, n, lam):
    from tests.gpu_util import dev, host
    inst = synth.make_instance(n, 16, lam, seed=41, grid=4)
    G = O.kernel_matrix(inst.Q, inst.scale)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    Z = synth.directions(n, 64, 41)
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.FP64)
    P = L.laker_fit_preconditioner(ctx, op, dev(Z))
    Pd = O.inverse_sqrt(O.cccp_fit(O.random_directions(A, Z), 0.1, O.shrinkage_rho(n, 64, 0.1), 1e-8).Sigma)
    alpha, info, trace = L.laker_pcg_solve_trace(ctx, op, P, dev(inst.y), 1e-12, max_iter=2000)
    k = info["iterations"]
    assert trace.shape == (k, 4) and np.all(np.isfinite(trace))
    # the first ten products, in two parts.  (1) The GPU's iterate after k
    # products equals the oracle's to 1e-9 (the float64 alpha parity).  (2)
    # The trace's R and residual equal the oracle's evaluation of them on the
    # GPU's own iterate to 1e-10: they differ only in how R is formed (from the
    # recursive residual, |r|^2 + lambda (r.alpha + y.alpha), against dense
    # products).  Comparing the trace with the oracle's R at the oracle's own
    # iterate would mix in R's sensitivity to alpha, |grad R| |alpha| / |R|,
    # which reaches 2.7e4 by the ninth product at n = 1024.
    its = _oracle_iterates(A, inst.y, Pd, 10)
    ny2 = float(inst.y @ inst.y)
    for j, a in enumerate(its):
        ag, _ = L.laker_pcg_solve(ctx, op, P, dev(inst.y), 0.0, max_iter=j + 1, allow_maxiter=True)
        ag = host(ag)
        assert np.linalg.norm(ag - a) <= 1e-9 * np.linalg.norm(a), j
        R = O.objective_R(G, ag, inst.y, inst.lam)
        rr = float(np.sum((inst.y - A @ ag) ** 2)) / ny2
        assert abs(trace[j, 2] - R) <= 1e-10 * abs(R), (j, trace[j, 2], R)
        assert abs(trace[j, 1] - rr) <= 1e-10 * rr + 1e-28, (j, trace[j, 1], rr)
    # iterations to the objective gap 1e-3 against the reference solution
    a_ref = O.solve_direct(A, inst.y)
    R_ref = O.objective_R(G, a_ref, inst.y, inst.lam)
    k_gpu = L.laker_trace_gap_iterations(trace, R_ref, 1e-3)
    env = gap_envelope(A, G, inst.y, Pd, inst.lam, R_ref, 1e-3, k, p_rel=1e-9)
    assert env is not None and within_envelope(k_gpu, env), (k_gpu, env)
    # kappa(P A) from the Lanczos tridiagonal of the converged solve
    lo, hi = L.laker_lanczos_extremes(trace)
    kappa = O.condition_number(A, Pd)
    assert hi / lo <= kappa * (1 + 1e-6), (hi / lo, kappa)
    assert hi / lo >= 0.95 * kappa, (hi / lo, kappa)


def test_trace_of_a_mixed_solve(L, ctx):
    """Mixed (split-bf16) solve: iterations to the objective gap TAR.TOL =
    1e-3 from the trace (which follows the recursive residual between
    replacements).  The index is an exact first crossing of the GPU's own
    iterates, evaluated by the oracle (to 1 % of TAR.TOL: the recursive
    residual of the float32-class operator drifts from the true one by ~1e-6
    relative), and it lies within the oracle's float64 envelope widened by
    its width and by 15 %: the mixed preconditioner is Sigma_*^-1/2 to a few %
    along every direction (readings 11-12), which moves CG's progress by
    about that much.  The Lanczos extremes are positive and ordered."""
    from tests.gpu_util import bf16_round, dev, host
    n = 2048
    inst = synth.make_instance(n, 32, 1e-4, seed=43, layout="clustered", grid=4)
    G = O.kernel_matrix(inst.Q, inst.scale)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    Z = bf16_round(synth.directions(n, 181, 43))
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.BF16X3)
    P = L.laker_fit_preconditioner(ctx, op, dev(Z))
    alpha, info, trace = L.laker_pcg_solve_trace(ctx, op, P, dev(inst.y), 1e-6, max_iter=20000, refine_every=20)
    assert info["converged"] == 1 and np.all(np.isfinite(trace))
    a_star = O.solve_direct(A, inst.y)
    R_ref = O.objective_R(G, a_star, inst.y, inst.lam)
    k = L.laker_trace_gap_iterations(trace, R_ref, 1e-3)
    assert k >= 1
    a_k, _ = L.laker_pcg_solve(ctx, op, P, dev(inst.y), 0.0, max_iter=k, allow_maxiter=True, refine_every=20)
    assert O.objective_gap(G, host(a_k), a_star, inst.y, inst.lam) <= 1e-3 * 1.01
    if k > 1:
        a_p, _ = L.laker_pcg_solve(ctx, op, P, dev(inst.y), 0.0, max_iter=k - 1, allow_maxiter=True, refine_every=20)
        assert O.objective_gap(G, host(a_p), a_star, inst.y, inst.lam) > 1e-3 * 0.99
    Pd = O.inverse_sqrt(O.cccp_fit(O.random_directions(A, Z), 0.1, O.shrinkage_rho(n, 181, 0.1), 1e-8).Sigma)
    env = gap_envelope(A, G, inst.y, Pd, inst.lam, R_ref, 1e-3, 20000, p_rel=1e-3)
    w = max(1, env[1] - env[0])
    assert env[0] - w - 0.15 * env[0] <= k <= env[1] + w + 0.15 * env[1], (k, env)
    lo, hi = L.laker_lanczos_extremes(trace)
    assert 0 < lo < hi
