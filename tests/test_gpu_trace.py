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
    # the first ten products against the oracle's iterates (float64 parity:
    # the iterates agree to ~1e-9 there, R to 1.6e-9 at the tenth at n = 1024)
    its = _oracle_iterates(A, inst.y, Pd, 10)
    ny2 = float(inst.y @ inst.y)
    for j, a in enumerate(its):
        R = O.objective_R(G, a, inst.y, inst.lam)
        rr = float(np.sum((inst.y - A @ a) ** 2)) / ny2
        assert abs(trace[j, 2] - R) <= 1e-7 * abs(R), (j, trace[j, 2], R)
        assert abs(trace[j, 1] - rr) <= 1e-7 * rr + 1e-28, (j, trace[j, 1], rr)
    # iterations to the objective gap 1e-3 against the reference solution
    a_ref = O.solve_direct(A, inst.y)
    R_ref = O.objective_R(G, a_ref, inst.y, inst.lam)
    k_gpu = L.laker_trace_gap_iterations(trace, R_ref, 1e-3)
    k_ora = next(j + 1 for j, a in enumerate(_oracle_iterates(A, inst.y, Pd, k))
                 if abs(O.objective_R(G, a, inst.y, inst.lam) - R_ref) <= 1e-3 * abs(R_ref))
    assert abs(k_gpu - k_ora) <= 1, (k_gpu, k_ora)
    # kappa(P A) from the Lanczos tridiagonal of the converged solve
    lo, hi = L.laker_lanczos_extremes(trace)
    kappa = O.condition_number(A, Pd)
    assert hi / lo <= kappa * (1 + 1e-6), (hi / lo, kappa)
    assert hi / lo >= 0.95 * kappa, (hi / lo, kappa)


def test_trace_of_a_mixed_solve(L, ctx):
    """Mixed (split-bf16) solve: the trace is finite, its objective comes within
    1e-2 of the reference objective (it follows the recursive residual between
    replacements) and the Lanczos extremes are positive and ordered."""
    from tests.gpu_util import dev
    n = 2048
    inst = synth.make_instance(n, 32, 1e-4, seed=43, layout="clustered", grid=4)
    G = O.kernel_matrix(inst.Q, inst.scale)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.BF16X3)
    P = L.laker_fit_preconditioner(ctx, op, dev(synth.directions(n, 181, 43)))
    alpha, info, trace = L.laker_pcg_solve_trace(ctx, op, P, dev(inst.y), 1e-6, max_iter=20000, refine_every=20)
    assert info["converged"] == 1 and np.all(np.isfinite(trace))
    R_ref = O.objective_R(G, O.solve_direct(A, inst.y), inst.y, inst.lam)
    assert L.laker_trace_gap_iterations(trace, R_ref, 1e-2) >= 1
    lo, hi = L.laker_lanczos_extremes(trace)
    assert 0 < lo < hi
