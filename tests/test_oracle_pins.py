"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test checks the oracle against the paper's printed Example 1, exact
rational arithmetic, a closed form, a textbook property or one of the paper's
theorems -- never against a re-typed copy of the oracle's own formula.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import laker_oracle as O
from paper_2604_25138_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _example1():
    with open(os.path.join(GOLDEN, "example1.json")) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# Example 1 (Sec. IV-E): the paper's worked numbers
# --------------------------------------------------------------------------

def test_example1_kernel_matches_printed_values():
    ex = _example1()
    E = np.array(ex["embeddings"])
    G = O.kernel_matrix(E, ex["scale"])
    # embeddings are printed to 3 decimals, G too: G_22 evaluates to 1.134
    # against the printed 1.133, so 2e-3 absolute is the honest bound.
    np.testing.assert_allclose(G, np.array(ex["G"]), atol=2e-3, rtol=0)
    A = O.system_matrix(E, ex["scale"], ex["lambda"])
    np.testing.assert_allclose(A, np.array(ex["lambda_I_plus_G"]), atol=2e-3, rtol=0)


def test_example1_alpha_and_prediction():
    ex = _example1()
    E = np.array(ex["embeddings"])
    y = np.array(ex["y_dbm"])
    A = O.system_matrix(E, ex["scale"], ex["lambda"])
    a_direct = O.solve_direct(A, y)
    a_print = np.array(ex["alpha"])
    rel = np.linalg.norm(a_direct - a_print) / np.linalg.norm(a_print)
    assert rel < 2e-3, rel
    res = O.pcg(A, y, None, tol=1e-14)
    assert res.converged and res.iterations <= 4
    np.testing.assert_allclose(res.alpha, a_direct, rtol=1e-10, atol=1e-10)
    eq = np.array([ex["query_embedding"]])
    row = O.kernel_matrix(eq, ex["scale"], E)[0]
    np.testing.assert_allclose(row, np.array(ex["query_kernel_row"]), atol=1e-3, rtol=0)
    pred = O.radio_map(eq, E, a_direct, ex["scale"])[0]
    assert abs(pred - ex["query_prediction_dbm"]) < 0.05, pred


# --------------------------------------------------------------------------
# Kernel: closed forms independent of np.exp
# --------------------------------------------------------------------------

def test_kernel_equals_hadamard_power_series():
    """exp of a matrix elementwise = sum_m (S)^{o m} / m! (Hadamard powers)."""
    rng = np.random.default_rng(3)
    E = rng.normal(size=(13, 5)) * 0.4
    s = 0.7
    S = s * (E @ E.T)
    acc = np.zeros_like(S)
    term = np.ones_like(S)
    for m in range(0, 40):
        acc += term
        term = term * S / (m + 1)
    np.testing.assert_allclose(O.kernel_matrix(E, s), acc, rtol=1e-14, atol=0)


def test_kernel_zero_embedding_is_all_ones():
    G = O.kernel_matrix(np.zeros((7, 3)), 1.0)
    assert np.array_equal(G, np.ones((7, 7)))


def test_system_is_spd_and_calibrated_n512():
    inst = synth.make_instance(512, 16, 1e-3, seed=11, grid=4)
    G = O.kernel_matrix(inst.Q, inst.scale)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    assert np.array_equal(A, A.T)
    assert (G > 0).all()
    w = np.linalg.eigvalsh(A)
    # Schur product theorem: G = exp(S) elementwise is PSD, so
    # lambda_min(A) >= lambda.
    assert w[0] >= inst.lam * (1 - 1e-9)
    # Sec. III-B: kappa ~ 1 + n/(Q lambda) for one cluster of unit entries;
    # with entries of mean m the top eigenvalue is ~ n m.
    approx = 1 + 512 * G.mean() / inst.lam
    kappa = w[-1] / w[0]
    assert 0.3 * approx < kappa < 3.0 * approx


# --------------------------------------------------------------------------
# Solve: exact rational brute force and limits
# --------------------------------------------------------------------------

def _exact_solve(A, y):
    n = len(y)
    M = [[Fraction(float(A[i, j])) for j in range(n)] + [Fraction(float(y[i]))] for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    return np.array([float(M[i][n] / M[i][i]) for i in range(n)])


@pytest.mark.parametrize("n,lam", [(1, 0.5), (2, 1e-2), (5, 1e-3), (8, 1e-1), (8, 1e-4)])
def test_solve_matches_exact_rational_arithmetic(n, lam):
    rng = np.random.default_rng(100 + n)
    E = rng.normal(size=(n, 3)) * 0.5
    y = rng.normal(size=n)
    A = O.system_matrix(E, 1.0, lam)
    exact = _exact_solve(A, y)
    scale = np.linalg.norm(exact)
    assert np.linalg.norm(O.solve_direct(A, y) - exact) / scale < 1e-10
    for P in (None, O.jacobi_preconditioner(A)):
        res = O.pcg(A, y, P, tol=1e-14, max_iter=200)
        assert np.linalg.norm(res.alpha - exact) / scale < 1e-8


def test_large_lambda_limit():
    """alpha -> y / lambda as lambda grows, with |lambda alpha - y| = O(|G|/lambda)."""
    inst = synth.make_instance(64, 8, 1.0, seed=5, grid=2)
    G = O.kernel_matrix(inst.Q, inst.scale)
    gnorm = np.linalg.norm(G, 2)
    errs = []
    for lam in (1e4, 1e6):
        A = G + lam * np.eye(64)
        a = O.solve_direct(A, inst.y)
        e = np.linalg.norm(lam * a - inst.y) / np.linalg.norm(inst.y)
        assert e <= 1.01 * gnorm / lam
        errs.append(e)
    assert errs[1] < errs[0] / 50


# --------------------------------------------------------------------------
# PCG: textbook properties
# --------------------------------------------------------------------------

def _spd_with_spectrum(eigs, seed):
    rng = np.random.default_rng(seed)
    V, _ = np.linalg.qr(rng.normal(size=(len(eigs), len(eigs))))
    return (V * np.asarray(eigs)) @ V.T, V


def test_cg_terminates_in_number_of_distinct_eigenvalues():
    eigs = [1.0] * 10 + [7.0] * 10 + [40.0] * 10
    A, _ = _spd_with_spectrum(eigs, 1)
    y = np.random.default_rng(2).normal(size=30)
    res = O.pcg(A, y, None, tol=1e-11)
    assert res.converged and res.iterations == 3
    np.testing.assert_allclose(A @ res.alpha, y, atol=1e-9)


def test_pcg_with_exact_inverse_takes_one_iteration():
    A, _ = _spd_with_spectrum(np.linspace(0.01, 50.0, 20), 4)
    y = np.random.default_rng(5).normal(size=20)
    res = O.pcg(A, y, np.linalg.inv(A), tol=1e-10)
    assert res.iterations == 1


def test_pcg_two_distinct_preconditioned_eigenvalues():
    """If P A has two distinct eigenvalues, PCG stops after two products."""
    A, V = _spd_with_spectrum(np.linspace(1.0, 1000.0, 24), 6)
    target = np.array([1.0] * 12 + [3.0] * 12)
    # P = V diag(target / eig(A)) V^T so that P A = V diag(target) V^T
    P = (V * (target / np.linspace(1.0, 1000.0, 24))) @ V.T
    y = np.random.default_rng(7).normal(size=24)
    res = O.pcg(A, y, P, tol=1e-10)
    assert res.iterations == 2


def test_pcg_matches_direct_within_condition_bound():
    inst = synth.make_instance(256, 16, 1e-3, seed=9, grid=2)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    a_star = O.solve_direct(A, inst.y)
    kappa = O.condition_number(A)
    for P in (None, O.jacobi_preconditioner(A)):
        res = O.pcg(A, inst.y, P, tol=1e-12)
        assert res.converged
        err = np.linalg.norm(res.alpha - a_star) / np.linalg.norm(a_star)
        assert err <= kappa * 1e-12 * 10


# --------------------------------------------------------------------------
# CCCP: Theorem 1, Tyler's fixed point, stationarity of the MLE objective
# --------------------------------------------------------------------------

def _ubar(n, n_r, seed):
    inst = synth.make_instance(n, 6, 1e-2, seed=seed, grid=2)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    return O.random_directions(A, synth.directions(n, n_r, seed)), A


def test_random_directions_are_unit_columns_along_A_z():
    U, A = _ubar(20, 7, 1)
    Z = synth.directions(20, 7, 1)
    np.testing.assert_allclose(np.linalg.norm(U, axis=0), 1.0, rtol=1e-14)
    for k in range(7):
        # u_k is parallel to A z_k with a positive factor
        v = A @ Z[:, k]
        cos = v @ U[:, k] / np.linalg.norm(v)
        assert abs(cos - 1.0) < 1e-13


def test_cccp_theorem1_invariants():
    n, n_r = 24, 10
    U, _ = _ubar(n, n_r, 2)
    gamma, rho, eps = 0.1, 0.05, 1e-8
    S = np.eye(n)
    for _ in range(15):
        F = O.cccp_map_F(S, U, gamma, eps)
        St = (1 - rho) * F + rho * np.eye(n)
        assert np.linalg.eigvalsh(St)[0] >= rho * (1 - 1e-12)   # Sigma~ >= rho I
        S_next = O.cccp_fit(U, gamma, rho, eps, max_iter=1, Sigma0=S).Sigma
        np.testing.assert_allclose(S_next, St / (np.trace(St) / n), rtol=1e-12, atol=1e-14)
        assert abs(np.trace(S_next) - n) < 1e-10 * n             # tr = n
        assert np.abs(S_next - S_next.T).max() < 1e-12           # symmetric
        assert np.linalg.eigvalsh(S_next)[0] > 0
        S = S_next
    res = O.cccp_fit(U, gamma, rho, eps, max_iter=500, tol=1e-12)
    assert res.converged
    # fixed point of T (Theorem 1)
    again = O.cccp_fit(U, gamma, rho, eps, max_iter=1, Sigma0=res.Sigma).Sigma
    assert np.linalg.norm(again - res.Sigma) / np.linalg.norm(res.Sigma) < 1e-10


def _sym_dirs(S, k, seed):
    """Random symmetric directions scaled to S (S^1/2 H S^1/2), so a finite
    step is small relative to every eigenvalue of S."""
    n = S.shape[0]
    w, V = np.linalg.eigh(S)
    Sh = (V * np.sqrt(w)) @ V.T
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(k):
        H = rng.normal(size=(n, n))
        out.append(Sh @ ((H + H.T) / 2) @ Sh)
    return out


def test_cccp_gamma0_reaches_tyler_fixed_point_and_is_stationary():
    """gamma = rho = eps = 0: the normalised iteration is Tyler's estimator;
    its limit satisfies Eq. tyler-fixed-point with tr = n and is a stationary
    point of the scale-invariant ACG likelihood (Sec. IV-A)."""
    n, n_r = 8, 40
    U, _ = _ubar(n, n_r, 3)
    res = O.cccp_fit(U, 0.0, 0.0, 0.0, max_iter=5000, tol=1e-14)
    S = res.Sigma
    Sinv = np.linalg.inv(S)
    rhs = np.zeros((n, n))
    for k in range(n_r):
        u = U[:, k]
        rhs += np.outer(u, u) / (u @ Sinv @ u)
    rhs *= n / n_r
    np.testing.assert_allclose(S, rhs, rtol=1e-9, atol=1e-11)
    assert abs(np.trace(S) - n) < 1e-9
    f0 = O.mle_objective(S, U, 0.0)
    h = 1e-5
    for H in _sym_dirs(S, 4, 8):
        g = (O.mle_objective(S + h * H, U, 0.0) - O.mle_objective(S - h * H, U, 0.0)) / (2 * h)
        assert abs(g) < 1e-6 * max(1.0, abs(f0))


def test_unnormalised_cccp_is_monotone_and_stationary():
    """gamma > 0, rho = eps = 0, no normalisation: CCCP (Sec. IV-C) is a
    majorise-minimise scheme for Eq. prob:kernel-mle; the objective never
    increases and the limit has zero directional derivatives."""
    n, n_r = 8, 40
    U, _ = _ubar(n, n_r, 4)
    gamma = 0.3
    S = np.eye(n)
    prev = O.mle_objective(S, U, gamma)
    for _ in range(60):
        S = O.cccp_fit(U, gamma, 0.0, 0.0, max_iter=1, normalize=False, Sigma0=S).Sigma
        cur = O.mle_objective(S, U, gamma)
        assert cur <= prev + 1e-12 * abs(prev)
        prev = cur
    res = O.cccp_fit(U, gamma, 0.0, 0.0, max_iter=20000, tol=1e-14, normalize=False)
    S = res.Sigma
    f0 = O.mle_objective(S, U, gamma)
    h = 1e-5
    for H in _sym_dirs(S, 4, 9):
        g = (O.mle_objective(S + h * H, U, gamma) - O.mle_objective(S - h * H, U, gamma)) / (2 * h)
        assert abs(g) < 1e-6 * max(1.0, abs(f0))


def test_inverse_sqrt_property():
    U, _ = _ubar(30, 12, 5)
    S = O.cccp_fit(U, 0.1, 0.1, 1e-8, max_iter=50).Sigma
    P = O.inverse_sqrt(S)
    np.testing.assert_allclose(P @ S @ P, np.eye(30), atol=1e-10)
    np.testing.assert_allclose(P, P.T, atol=1e-14)
    assert np.linalg.eigvalsh(P)[0] > 0


def test_cccp_preconditioner_reduces_condition_number():
    """Sec. V-B: the learned P shrinks kappa by orders of magnitude while
    Jacobi barely changes it; PCG iterations order accordingly."""
    n = 512
    inst = synth.make_instance(n, 16, 1e-3, seed=21, grid=2)
    Z = synth.directions(n, synth.default_num_directions(n), 21)
    r = O.laker(inst.Q, inst.y, inst.lam, inst.scale, Z, tol=1e-8)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    kA = O.condition_number(A)
    kPA = O.condition_number(A, r.P)
    kJ = O.condition_number(A, O.jacobi_preconditioner(A))
    assert kPA < kA / 10
    assert kJ > kA / 3
    it_j = O.pcg(A, inst.y, O.jacobi_preconditioner(A), 1e-8).iterations
    assert r.pcg.iterations < it_j


# --------------------------------------------------------------------------
# Metrics and the radio map
# --------------------------------------------------------------------------

def test_direct_solution_minimises_R():
    """Sec. III / V-A: the minimiser of R(alpha) solves (G + lambda I) alpha = y
    (G is invertible here); finite differences of R vanish at alpha*."""
    inst = synth.make_instance(40, 6, 1e-1, seed=13, grid=2)
    G = O.kernel_matrix(inst.Q, inst.scale)
    A = G + inst.lam * np.eye(40)
    a = O.solve_direct(A, inst.y)
    rng = np.random.default_rng(1)
    h = 1e-4
    base = O.objective_R(G, a, inst.y, inst.lam)
    for _ in range(5):
        v = rng.normal(size=40)
        g = (O.objective_R(G, a + h * v, inst.y, inst.lam)
             - O.objective_R(G, a - h * v, inst.y, inst.lam)) / (2 * h)
        assert abs(g) < 1e-6 * max(1.0, base)
    assert O.objective_gap(G, a, a, inst.y, inst.lam) == 0.0
    assert O.prediction_discrepancy(G, a, a) == 0.0
    assert O.relative_residual(A, a, inst.y) < 1e-12


def test_radio_map_at_training_points_is_y_minus_lambda_alpha():
    """From (G + lambda I) alpha = y: r(x_i) = (G alpha)_i = y_i - lambda alpha_i."""
    inst = synth.make_instance(50, 8, 1e-2, seed=17, grid=2)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    a = O.solve_direct(A, inst.y)
    f = O.radio_map(inst.Q, inst.Q, a, inst.scale)
    np.testing.assert_allclose(f, inst.y - inst.lam * a, rtol=1e-9, atol=1e-9)


def test_rmse_nmse_closed_forms():
    t = np.array([1.0, -2.0, 3.0, 0.5])
    p = t + np.array([0.1, -0.1, 0.2, 0.0])
    assert abs(O.rmse(p, t) - math.sqrt((0.01 + 0.01 + 0.04) / 4)) < 1e-15
    assert abs(O.nmse(p, t) - 0.06 / (1 + 4 + 9 + 0.25)) < 1e-15


def test_cccp_map_at_identity_closed_form_trace():
    """At Sigma = I every quadratic form u_k^T u_k is 1, so
    tr F_gamma(I) = n (1/(1 + eps) + gamma) / (1 + gamma/n) in closed form
    (Eq. kernel_shrinkage_cccp_F)."""
    n, n_r = 15, 9
    U, _ = _ubar(n, n_r, 6)
    for gamma, eps in ((0.3, 0.5), (0.0, 2.0), (1.7, 0.0)):
        F = O.cccp_map_F(np.eye(n), U, gamma, eps)
        want = n * (1.0 / (1.0 + eps) + gamma) / (1.0 + gamma / n)
        assert abs(np.trace(F) - want) < 1e-12 * want
        # and F - gamma I/(1+gamma/n) has rank <= N_r
        R = F - gamma / (1 + gamma / n) * np.eye(n)
        assert np.linalg.matrix_rank(R, tol=1e-10) <= n_r


def test_shrinkage_rule_reading():
    assert O.shrinkage_rho(100, 100, 0.1) == 1e-3
    assert O.shrinkage_rho(100, 200, 0.1) == 1e-3
    vals = [O.shrinkage_rho(1000, m, 0.1) for m in (900, 500, 100, 10)]
    assert all(a <= b for a, b in zip(vals, vals[1:]))
    assert O.shrinkage_rho(1000, 10, 5.0) == 0.5


# --------------------------------------------------------------------------
# Metrics with hand-worked values (Sec. V-A, Eqs. objective-gap and
# prediction-discrepancy), the Jacobi baseline and the condition number
# --------------------------------------------------------------------------

def _R_exact(G, a, y, lam):
    """R(alpha) = |G alpha - y|^2 + lambda alpha^T G alpha in exact rationals,
    written as explicit loops over the entries."""
    n = len(y)
    Ga = [sum((G[i][j] * a[j] for j in range(n)), Fraction(0)) for i in range(n)]
    fit = sum(((Ga[i] - y[i]) ** 2 for i in range(n)), Fraction(0))
    reg = sum((a[i] * Ga[i] for i in range(n)), Fraction(0))
    return fit + lam * reg


def test_objective_gap_and_prediction_discrepancy_hand_worked_2x2():
    """G = [[2, 1], [1, 3]], y = (1, 2), lambda = 1/2, alpha = (1, 0),
    alpha_ref = (0, 1).  By hand: G alpha = (2, 1), |G alpha - y|^2 = 2,
    alpha^T G alpha = 2, so R(alpha) = 3; G alpha_ref = (1, 3),
    |G alpha_ref - y|^2 = 1, alpha_ref^T G alpha_ref = 3, so R(alpha_ref) = 5/2.
    Objective gap |3 - 5/2| / (5/2) = 1/5.  Prediction discrepancy
    |(2, 1) - (1, 3)| / |(1, 3)| = sqrt(5) / sqrt(10) = 1/sqrt(2).
    A dropped lambda term (gap 1), lambda alpha^T alpha in place of
    alpha^T G alpha (gap 2/3), normalising by R(alpha) (1/6), or comparing
    alpha instead of G alpha (sqrt 2) all fail."""
    G = np.array([[2.0, 1.0], [1.0, 3.0]])
    y = np.array([1.0, 2.0])
    a = np.array([1.0, 0.0])
    a_ref = np.array([0.0, 1.0])
    assert O.objective_R(G, a, y, 0.5) == 3.0
    assert O.objective_R(G, a_ref, y, 0.5) == 2.5
    assert abs(O.objective_gap(G, a, a_ref, y, 0.5) - 0.2) < 1e-15
    assert abs(O.prediction_discrepancy(G, a, a_ref) - 1.0 / math.sqrt(2.0)) < 1e-15


def test_objective_gap_and_prediction_discrepancy_exact_3x3():
    """A non-symmetric-looking but symmetric 3 x 3 G with rational entries,
    unequal alpha and alpha_ref: the oracle's float64 metrics against exact
    rational arithmetic (squared discrepancy compared, to stay rational)."""
    Gq = [[Fraction(5, 2), Fraction(1, 3), Fraction(-1, 4)],
          [Fraction(1, 3), Fraction(7, 5), Fraction(1, 6)],
          [Fraction(-1, 4), Fraction(1, 6), Fraction(9, 8)]]
    yq = [Fraction(3, 2), Fraction(-1, 2), Fraction(2, 7)]
    aq = [Fraction(1, 5), Fraction(-3, 4), Fraction(5, 3)]
    rq = [Fraction(-2, 3), Fraction(1, 2), Fraction(1, 9)]
    lam = Fraction(3, 10)
    G = np.array([[float(v) for v in row] for row in Gq])
    y, a, r = (np.array([float(v) for v in vec]) for vec in (yq, aq, rq))
    R_a, R_r = _R_exact(Gq, aq, yq, lam), _R_exact(Gq, rq, yq, lam)
    gap = abs(R_a - R_r) / abs(R_r)
    assert abs(O.objective_gap(G, a, r, y, float(lam)) - float(gap)) < 1e-14 * float(gap)
    Ga = [sum(Gq[i][j] * aq[j] for j in range(3)) for i in range(3)]
    Gr = [sum(Gq[i][j] * rq[j] for j in range(3)) for i in range(3)]
    disc2 = sum((Ga[i] - Gr[i]) ** 2 for i in range(3)) / sum(v * v for v in Gr)
    pd = O.prediction_discrepancy(G, a, r)
    assert abs(pd * pd - float(disc2)) < 1e-14 * float(disc2)


def test_jacobi_preconditioner_is_the_inverse_diagonal():
    """P_J = diag(A)^-1 (Sec. V-A baseline).  On a diagonal A with distinct
    entries P_J is A^-1 exactly, so P_J A = I and PCG stops after one product;
    on a full SPD A, P_J is diagonal and P_J A has a unit diagonal.  diag(A)
    in place of its inverse, diag(A)^-1/2, or the full inverse all fail."""
    a = np.array([0.5, 2.0, 8.0, 32.0, 0.125])          # exact binary fractions
    A = np.diag(a)
    PJ = O.jacobi_preconditioner(A)
    assert np.array_equal(PJ @ A, np.eye(5))
    res = O.pcg(A, np.array([1.0, -2.0, 3.0, 0.5, 4.0]), PJ, 1e-14)
    assert res.converged and res.iterations == 1
    inst = synth.make_instance(60, 8, 1e-2, seed=19, grid=2)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    PJ = O.jacobi_preconditioner(A)
    assert np.array_equal(PJ, np.diag(np.diag(PJ)))
    np.testing.assert_allclose(np.diag(PJ @ A), np.ones(60), rtol=2e-16, atol=0)


def test_condition_number_of_a_known_spectrum():
    """A = V diag(a) V^T and P = V diag(p) V^T share eigenvectors, so the
    eigenvalues of P A are a_k p_k and kappa(P A) = max(a p) / min(a p)
    exactly; for a P that does not commute with A, kappa(P A) equals the
    ratio of the extreme generalised eigenvalues of A x = mu P^-1 x."""
    rng = np.random.default_rng(23)
    V, _ = np.linalg.qr(rng.normal(size=(12, 12)))
    a = np.geomspace(1e-3, 1e3, 12)
    p = np.geomspace(5.0, 0.02, 12)
    A = (V * a) @ V.T
    A = 0.5 * (A + A.T)
    P = (V * p) @ V.T
    P = 0.5 * (P + P.T)
    want = float(np.max(a * p) / np.min(a * p))
    assert abs(O.condition_number(A, P) - want) < 1e-8 * want
    assert abs(O.condition_number(A) - 1e6) < 1e-6 * 1e6
    W, _ = np.linalg.qr(rng.normal(size=(12, 12)))
    P2 = (W * np.geomspace(0.1, 10.0, 12)) @ W.T
    P2 = 0.5 * (P2 + P2.T)
    mu = scipy_eigh_general(A, np.linalg.inv(P2))
    assert abs(O.condition_number(A, P2) - mu[-1] / mu[0]) < 1e-7 * (mu[-1] / mu[0])


def scipy_eigh_general(A, B):
    import scipy.linalg
    return scipy.linalg.eigh(A, 0.5 * (B + B.T), eigvals_only=True)


# --------------------------------------------------------------------------
# Gradient descent baseline (Sec. V-A) and the device generator's definition
# --------------------------------------------------------------------------

def test_gradient_of_R_matches_finite_differences():
    inst = synth.make_instance(30, 5, 1e-1, seed=29, grid=2)
    G = O.kernel_matrix(inst.Q, inst.scale)
    rng = np.random.default_rng(4)
    a = rng.normal(size=30)
    g = O.gradient_R(G, a, inst.y, inst.lam)
    h = 1e-5
    for _ in range(5):
        v = rng.normal(size=30)
        fd = (O.objective_R(G, a + h * v, inst.y, inst.lam) - O.objective_R(G, a - h * v, inst.y, inst.lam)) / (2 * h)
        assert abs(fd - g @ v) < 1e-6 * max(1.0, abs(fd))


def test_gradient_descent_contracts_each_eigencomponent_in_closed_form():
    """With G = V diag(g) V^T, A = G + lambda I and alpha* = A^-1 y, one GD step
    maps the error e = alpha - alpha* to (I - 2 eta G A) e, so after k steps
    from alpha^0 = 0 its component along v_i is (1 - 2 eta g_i (g_i + lambda))^k
    times that of -alpha*."""
    rng = np.random.default_rng(8)
    V, _ = np.linalg.qr(rng.normal(size=(9, 9)))
    g = np.array([3.0, 1.5, 1.0, 0.5, 0.25, 0.1, 0.05, 0.01, 0.0])
    G = (V * g) @ V.T
    G = 0.5 * (G + G.T)
    lam = 0.2
    y = rng.normal(size=9)
    a_star = V @ ((V.T @ y) / (g + lam))
    eta = 0.9 / (2 * g[0] * (g[0] + lam))
    k = 7
    res = O.gradient_descent(G, y, lam, eta, max_iter=k)
    want = a_star + V @ (((1 - 2 * eta * g * (g + lam)) ** k) * (V.T @ -a_star))
    assert res.steps == k and not res.converged
    np.testing.assert_allclose(res.alpha, want, rtol=0, atol=1e-12 * np.linalg.norm(a_star))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(res.R, res.R[1:]))   # eta < 1/L: R decreases


def test_philox4x32_10_known_answers():
    from oracle import philox as X
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.json")) as f:
        kat = json.load(f)
    for case in kat["cases"]:
        c = [int(v, 16) for v in case["counter"]]
        k = [int(v, 16) for v in case["key"]]
        got = [int(v) for v in X.philox4x32_10(c, k)]
        assert got == [int(v, 16) for v in case["out"]]


def test_philox_gaussian_directions_are_standard_normal():
    """Moments and tail fractions of 2^18 draws: mean 0, variance 1, fourth
    moment 3, and the one- and two-sigma fractions of N(0, 1) (0.6827, 0.9545)
    within five standard errors; the layout is reproducible and row-major."""
    from oracle import philox as X
    Z = X.gaussian_directions(1234, 512, 512)
    z = Z.ravel()
    m = z.size
    assert abs(z.mean()) < 5 / math.sqrt(m)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / m)
    assert abs(np.mean(z ** 4) - 3.0) < 5 * math.sqrt(96.0 / m)
    for s, p in ((1.0, 0.682689492), (2.0, 0.954499736)):
        frac = np.mean(np.abs(z) < s)
        assert abs(frac - p) < 5 * math.sqrt(p * (1 - p) / m)
    np.testing.assert_array_equal(X.gaussian_directions(1234, 3, 5), Z.ravel()[:15].reshape(3, 5))
    assert not np.array_equal(X.gaussian_directions(1235, 3, 5), Z.ravel()[:15].reshape(3, 5))


# --------------------------------------------------------------------------
# Streaming update (Sec. VI, future work): warm-started PCG and CCCP
# --------------------------------------------------------------------------

def _spd_exact(n, seed):
    """An SPD matrix with small-integer entries (exact in float64 and Fraction)."""
    rng = np.random.default_rng(seed)
    B = rng.integers(-3, 4, size=(n, n))
    return (B @ B.T + n * np.eye(n, dtype=np.int64)).astype(np.int64)


def test_warm_pcg_terminates_in_n_steps_from_any_start():
    """CG from any start reaches the exact solution in at most n steps in
    exact arithmetic (textbook): the solution is computed in Fraction
    arithmetic by Gaussian elimination, and the oracle's warm start from a
    far-off alpha0 must land on it after n = 4 steps (to rounding)."""
    n = 4
    Ai = _spd_exact(n, 3)
    yi = np.array([3, -1, 2, 5])
    # exact solution by Fraction Gaussian elimination
    M = [[Fraction(int(Ai[i, j])) for j in range(n)] + [Fraction(int(yi[i]))] for i in range(n)]
    for c in range(n):
        piv = M[c][c]
        for r in range(c + 1, n):
            f = M[r][c] / piv
            M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    x = [Fraction(0)] * n
    for r in range(n - 1, -1, -1):
        x[r] = (M[r][n] - sum(M[r][j] * x[j] for j in range(r + 1, n))) / M[r][r]
    exact = np.array([float(v) for v in x])
    A = Ai.astype(np.float64)
    y = yi.astype(np.float64)
    a0 = np.array([10.0, -7.0, 3.0, 0.5])
    res = O.pcg(A, y, None, 0.0, max_iter=n, alpha0=a0)
    np.testing.assert_allclose(res.alpha, exact, rtol=1e-12, atol=1e-12)
    # and with a (diagonal) preconditioner as well
    res = O.pcg(A, y, np.diag(1.0 / np.diag(A)), 0.0, max_iter=n, alpha0=a0)
    np.testing.assert_allclose(res.alpha, exact, rtol=1e-12, atol=1e-12)


def test_warm_pcg_from_the_solution_stops_before_any_product():
    n = 6
    A = _spd_exact(n, 5).astype(np.float64)
    y = np.arange(1.0, n + 1.0)
    a_star = np.linalg.solve(A, y)
    res = O.pcg(A, y, None, 1e-10, alpha0=a_star)
    assert res.iterations == 0 and res.converged
    np.testing.assert_array_equal(res.alpha, a_star)
    # a start that misses the tolerance does iterate
    res = O.pcg(A, y, None, 1e-10, alpha0=a_star + 1e-3)
    assert res.iterations >= 1 and res.converged


def test_warm_pcg_is_cold_pcg_on_the_residual_system():
    """PCG from alpha0 on A alpha = y is alpha0 plus PCG from 0 on
    A e = y - A alpha0 (translation invariance of Krylov iterates): fails if
    the warm start took r^0 = y, or kept alpha^0 = 0."""
    inst = synth.make_instance(120, 8, 1e-2, seed=9, grid=2)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    P = np.diag(1.0 / np.sqrt(np.diag(A)))
    a0 = synth.random_vector(120, 4)
    for k in (1, 5, 17):
        warm = O.pcg(A, inst.y, P, 0.0, max_iter=k, alpha0=a0).alpha
        cold = O.pcg(A, inst.y - A @ a0, P, 0.0, max_iter=k).alpha
        np.testing.assert_allclose(warm, a0 + cold, rtol=1e-9, atol=1e-9 * np.abs(a0).max())


def test_warm_sigma0_closed_form_on_orthonormal_directions():
    """With orthonormal directions, c I + U diag(D) U^T has eigenvalues c + D_k
    along u_k and c on the complement; scaled to trace n."""
    n, k = 10, 3
    U, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((n, k)))
    c, D = 0.7, np.array([2.0, 0.5, 5.0])
    S = O.warm_sigma0(U, c, D)
    s = n / (n * c + D.sum())
    assert abs(np.trace(S) - n) < 1e-12 * n
    np.testing.assert_allclose(S @ U, U * ((c + D) * s), rtol=1e-12, atol=1e-13)
    v = np.linalg.qr(np.concatenate([U, np.random.default_rng(2).standard_normal((n, 1))], axis=1))[0][:, -1]
    np.testing.assert_allclose(S @ v, c * s * v, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(O.warm_sigma0(U, 2.5, np.zeros(k)), np.eye(n), rtol=0, atol=1e-15)


def test_warm_cccp_reaches_the_cold_fixed_point():
    """The regularised MLE objective (Eq. prob:kernel-mle) is geodesically
    convex in Sigma, as Tyler's M-estimator is, and the trace penalty makes
    its minimiser unique, so CCCP reaches the same Sigma_* from any SPD start:
    a warm start from a positive (c, D) must land on the cold start's answer,
    and a start next to that answer must need fewer iterations."""
    n, n_r = 24, 10
    U, _ = _ubar(n, n_r, 2)
    gamma, rho, eps = 0.1, 0.05, 1e-8
    cold = O.cccp_fit(U, gamma, rho, eps, max_iter=500, tol=1e-12)
    rng = np.random.default_rng(3)
    warm = O.cccp_fit(U, gamma, rho, eps, max_iter=500, tol=1e-12,
                      Sigma0=O.warm_sigma0(U, 0.3, rng.uniform(0.1, 3.0, n_r)))
    assert cold.converged and warm.converged
    np.testing.assert_allclose(warm.Sigma, cold.Sigma, rtol=0, atol=1e-9 * np.abs(cold.Sigma).max())
    # started from a slightly perturbed copy of the answer: fewer iterations
    near = O.cccp_fit(U, gamma, rho, eps, max_iter=500, tol=1e-12, Sigma0=cold.Sigma + 1e-4 * np.eye(n))
    assert near.converged and near.iterations < cold.iterations


def test_cccp_step_coefficients_match_the_dense_update():
    """The coefficient form of one CCCP step equals the dense step of
    cccp_fit (cho_solve, explicit n x n sums) from an SPD start, and at the
    converged Sigma_* it reproduces Sigma_* (fixed point)."""
    n, n_r = 30, 6
    U, _ = _ubar(n, n_r, 4)
    gamma, rho, eps = 0.1, 0.05, 1e-8
    S0 = O.warm_sigma0(U, 0.4, np.array([1.0, 0.2, 3.0, 0.05, 0.7, 2.2]))
    c, D = O.cccp_step_coefficients(S0, U, gamma, rho, eps)
    step = O.cccp_fit(U, gamma, rho, eps, max_iter=1, Sigma0=S0).Sigma
    np.testing.assert_allclose(c * np.eye(n) + (U * D) @ U.T, step, rtol=0, atol=1e-12 * np.abs(step).max())
    res = O.cccp_fit(U, gamma, rho, eps, max_iter=500, tol=1e-13)
    c2, D2 = O.cccp_step_coefficients(res.Sigma, U, gamma, rho, eps)
    np.testing.assert_allclose(c2 * np.eye(n) + (U * D2) @ U.T, res.Sigma, rtol=0,
                               atol=1e-11 * np.abs(res.Sigma).max())
    assert c2 > 0 and np.all(D2 > 0)
