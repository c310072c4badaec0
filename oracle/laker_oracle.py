"""FP64 CPU oracle for LAKER's regularized attention-kernel regression.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline / reference legs may import this module.  The CUDA library never
calls it, and it shares no code with the CUDA path: the two meet only through
the seeded inputs drawn by ``paper_2604_25138_gb300.synth``.

Everything here is written as plainly as the paper states it, in float64,
with dense matrices and numpy/scipy primitives (matmul, Cholesky,
symmetric eigendecomposition) used only as single steps.  No blocking, low-rank
tricks or fusion: the point is that a reader can check each function against
the cited equation by eye.

Paper map (arXiv 2604.25138):
* Sec. III-A, Eq. (sc-exp-kernel): G_ij = exp(<e_i, e_j>).  The scale s in
  exp(s <q_i, q_j>) is a parameter here (s = 1 reproduces the paper; s = 1/sqrt(d)
  is the scaled dot-product attention form, equivalent to e_i = q_i s^(1/2)).
* Sec. III-A, Eq. (sc-final): (G + lambda I) alpha = y.
* Sec. III-A, Eq. (sc-radio-map-reconstruction): r(x) = sum_i G(x, x_i) alpha_i.
* Sec. IV-B, Eq. (random_directions): u_k = (lambda I + G) z_k, u_k/|u_k|.
* Sec. IV-B, Eq. (prob:kernel-mle): the regularized MLE objective.
* Sec. IV-C, Eq. (atten-kernel-cccp-iteration) and Sec. IV-D,
  Eqs. (kernel_shrinkage_cccp_F / _Sigma / _normalization): shrinkage CCCP.
* Sec. IV-B, Eq. (preconditioner-Sigmma): P = Sigma_*^(-1/2).
* Sec. IV-E and Algorithm 1 (PCG stage): preconditioned conjugate gradient.
* Sec. V-A, Eqs. (simu-R-definition, residual, objective-gap,
  prediction-discrepancy, rmse, nmse): evaluation metrics.
* Sec. V-A, numerical-layer baselines: gradient descent on R(alpha).
* Sec. VI (future work: measurements arriving sequentially): the streaming
  update's warm starts, ``pcg(alpha0=...)`` and ``warm_sigma0`` for
  ``cccp_fit(Sigma0=...)``.
* oracle/philox.py: the counter-based generator behind the device-drawn
  random directions (Philox4x32-10, Salmon et al. 2011).

Parity pins (see tests/test_oracle_pins.py): every function below is pinned by
a test that does not re-run its own formula -- the paper's Example 1, exact
rational brute force, closed forms, Theorem 1's invariants, the Tyler
fixed-point equation and finite-difference stationarity of the MLE objective.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg


# ---------------------------------------------------------------------------
# Kernel and system (Sec. III-A)
# ---------------------------------------------------------------------------

def kernel_matrix(E: np.ndarray, scale: float = 1.0, E2: np.ndarray | None = None) -> np.ndarray:
    """G_ij = exp(scale * <e_i, e_j>)  (Eq. sc-exp-kernel), elementwise exp of
    the Gram matrix.  With ``E2`` given, the cross kernel exp(scale E E2^T)
    used by the radio-map reconstruction."""
    E = np.asarray(E, dtype=np.float64)
    E2 = E if E2 is None else np.asarray(E2, dtype=np.float64)
    return np.exp(scale * (E @ E2.T))


def system_matrix(E: np.ndarray, scale: float, lam: float) -> np.ndarray:
    """A = lambda I + G  (Eq. sc-final)."""
    G = kernel_matrix(E, scale)
    return G + lam * np.eye(G.shape[0])


def solve_direct(A: np.ndarray, y: np.ndarray) -> np.ndarray:
    """alpha* = A^-1 y by Cholesky.  A is SPD for lambda > 0 (Sec. III-A: G is
    PSD by the Schur product theorem), and alpha* is the unique minimiser of
    R(alpha) (Eq. simu-R-definition); it stands in for the paper's convex-solver
    reference solution."""
    c, low = scipy.linalg.cho_factor(A, lower=True)
    return scipy.linalg.cho_solve((c, low), y)


def radio_map(Eg: np.ndarray, E: np.ndarray, alpha: np.ndarray, scale: float) -> np.ndarray:
    """r(x_m) = sum_i exp(scale <e(x_m), e_i>) alpha_i
    (Eq. sc-radio-map-reconstruction; Algorithm 1, reconstruction stage)."""
    return kernel_matrix(Eg, scale, E) @ alpha


# ---------------------------------------------------------------------------
# Preconditioner learning (Sec. IV-B .. IV-D)
# ---------------------------------------------------------------------------

def random_directions(A: np.ndarray, Z: np.ndarray) -> np.ndarray:
    """u_k = (lambda I + G) z_k and u_k / |u_k|_2  (Eq. random_directions).
    Z is n x N_r with column k = z_k; the result has column k = u_bar_k."""
    U = A @ Z
    return U / np.linalg.norm(U, axis=0, keepdims=True)


def shrinkage_rho(n: int, n_r: int, gamma: float, eps_rho: float = 1e-3) -> float:
    """Adaptive shrinkage (Sec. V-A, preconditioner construction): a small fixed
    rho = eps_rho when N_r >= n; otherwise rho grows with the undersampling and
    scales with gamma.  The paper gives no constants; this reading is
    rho = min(1/2, max(eps_rho, gamma (1 - N_r/n)))."""
    if n_r >= n:
        return eps_rho
    return float(min(0.5, max(eps_rho, gamma * (1.0 - n_r / n))))


def mle_objective(Sigma: np.ndarray, Ubar: np.ndarray, gamma: float) -> float:
    """(1 + gamma/n) log det Sigma + (n/N_r) sum_k log(u_k^T Sigma^-1 u_k)
    + gamma tr(Sigma^-1)   (Eq. prob:kernel-mle; the nuclear norm of the SPD
    Sigma^-1 equals its trace, per the remark that follows it)."""
    n, n_r = Ubar.shape
    sign, logdet = np.linalg.slogdet(Sigma)
    if sign <= 0:
        return np.inf
    Sinv = np.linalg.inv(Sigma)
    quad = np.einsum("ik,ij,jk->k", Ubar, Sinv, Ubar)
    return float((1.0 + gamma / n) * logdet + (n / n_r) * np.sum(np.log(quad))
                 + gamma * np.trace(Sinv))


def cccp_map_F(Sigma: np.ndarray, Ubar: np.ndarray, gamma: float, eps: float) -> np.ndarray:
    """F_gamma(Sigma) = [ (n/N_r) sum_k u_k u_k^T / (u_k^T Sigma^-1 u_k + eps)
    + gamma I ] / (1 + gamma/n)   (Eq. kernel_shrinkage_cccp_F; with eps = 0
    this is the plain CCCP update, Eq. atten-kernel-cccp-iteration)."""
    n, n_r = Ubar.shape
    c, low = scipy.linalg.cho_factor(Sigma, lower=True)
    SinvU = scipy.linalg.cho_solve((c, low), Ubar)
    quad = np.sum(Ubar * SinvU, axis=0)                  # u_k^T Sigma^-1 u_k
    S = (Ubar / (quad + eps)) @ Ubar.T                     # sum_k u_k u_k^T / (q_k + eps)
    return ((n / n_r) * S + gamma * np.eye(n)) / (1.0 + gamma / n)


@dataclasses.dataclass
class CCCPResult:
    Sigma: np.ndarray          # Sigma_* (n x n)
    iterations: int            # number of updates applied
    converged: bool
    history: list              # relative Frobenius change per iteration
    rho: float


def cccp_fit(Ubar: np.ndarray, gamma: float, rho: float, eps: float,
             max_iter: int = 200, tol: float = 1e-10, normalize: bool = True,
             Sigma0: np.ndarray | None = None) -> CCCPResult:
    """Shrinkage-regularised CCCP (Algorithm 1, preconditioner-learning stage;
    Eqs. kernel_shrinkage_cccp_F, _Sigma, _normalization):

        Sigma_0 = I
        repeat: F = F_gamma(Sigma_t)
                Sigma~ = (1 - rho) F + rho I
                Sigma_{t+1} = Sigma~ / (tr(Sigma~) / n)

    Stopping (the paper says only "until convergence"; reading):
    |Sigma_{t+1} - Sigma_t|_F / |Sigma_t|_F <= tol, or max_iter updates.
    ``normalize=False`` drops the trace normalisation (the unnormalised CCCP
    of Eq. atten-kernel-cccp-iteration), used only by the stationarity pin."""
    n = Ubar.shape[0]
    Sigma = np.eye(n) if Sigma0 is None else np.array(Sigma0, dtype=np.float64)
    hist = []
    converged = False
    t = 0
    for t in range(1, max_iter + 1):
        F = cccp_map_F(Sigma, Ubar, gamma, eps)
        St = (1.0 - rho) * F + rho * np.eye(n)
        if normalize:
            St = St / (np.trace(St) / n)
        change = np.linalg.norm(St - Sigma) / np.linalg.norm(Sigma)
        hist.append(float(change))
        Sigma = St
        if change <= tol:
            converged = True
            break
    return CCCPResult(Sigma=Sigma, iterations=t, converged=converged, history=hist, rho=rho)


def warm_sigma0(Ubar: np.ndarray, c: float, D: np.ndarray) -> np.ndarray:
    """Start of a warm-started CCCP (the streaming update): a previous fit's
    Sigma_* = c I + sum_k D_k u_k u_k^T carried to the current normalised
    directions u_k, Sigma_0 = (c I + Ubar diag(D) Ubar^T) scaled to trace n
    like every CCCP iterate (Eq. kernel_shrinkage_cccp_normalization)."""
    n = Ubar.shape[0]
    S = c * np.eye(n) + (Ubar * np.asarray(D, dtype=np.float64)) @ Ubar.T
    return S / (np.trace(S) / n)


def cccp_step_coefficients(Sigma: np.ndarray, Ubar: np.ndarray, gamma: float, rho: float,
                           eps: float) -> tuple:
    """(c, D) of the next shrinkage-CCCP iterate written as c I + Ubar diag(D)
    Ubar^T (Eqs. kernel_shrinkage_cccp_F, _Sigma, _normalization): F_gamma
    puts the weight (n/N_r) / ((1 + gamma/n)(u_k^T Sigma^-1 u_k + eps)) on
    u_k u_k^T and gamma / (1 + gamma/n) on I; the shrinkage scales the former
    by 1 - rho and adds rho to the latter; the trace normalisation divides
    both by tr / n, with tr = n a + sum_k w_k |u_k|^2.  At a converged Sigma_*
    this is the low-rank form of Sigma_* itself (a fixed point)."""
    n, n_r = Ubar.shape
    c, low = scipy.linalg.cho_factor(Sigma, lower=True)
    quad = np.sum(Ubar * scipy.linalg.cho_solve((c, low), Ubar), axis=0)
    w = (1.0 - rho) * (n / n_r) / ((1.0 + gamma / n) * (quad + eps))
    a = (1.0 - rho) * gamma / (1.0 + gamma / n) + rho
    tr = n * a + float(np.sum(w * np.sum(Ubar * Ubar, axis=0)))
    return a * n / tr, w * n / tr


def inverse_sqrt(Sigma: np.ndarray) -> np.ndarray:
    """P = Sigma^(-1/2)  (Eq. preconditioner-Sigmma), by a symmetric
    eigendecomposition Sigma = V diag(w) V^T, P = V diag(w^-1/2) V^T."""
    w, V = np.linalg.eigh(Sigma)
    return (V * (1.0 / np.sqrt(w))) @ V.T


def jacobi_preconditioner(A: np.ndarray) -> np.ndarray:
    """P_J = diag(lambda I + G)^-1  (Sec. V-A, numerical-layer baselines)."""
    return np.diag(1.0 / np.diag(A))


# ---------------------------------------------------------------------------
# PCG (Sec. IV-E, Algorithm 1)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class PCGResult:
    alpha: np.ndarray
    iterations: int            # number of products (lambda I + G) p
    converged: bool
    rel_res: list              # |r^{k+1}| / |y| after each iteration (recursive r)


def pcg(A: np.ndarray, y: np.ndarray, P: np.ndarray | None, tol: float,
        max_iter: int = 100000, callback=None, alpha0: np.ndarray | None = None) -> PCGResult:
    """Preconditioned CG exactly in the order of Algorithm 1:

        alpha^0 = 0, r^0 = y, theta^0 = P r^0, p^0 = theta^0
        for k = 0, 1, ...:
            delta = (r^k . theta^k) / (p^k . A p^k)
            alpha^{k+1} = alpha^k + delta p^k
            r^{k+1}     = r^k - delta A p^k
            stop if |r^{k+1}| / |y| <= tol
            theta^{k+1} = P r^{k+1}
            beta = (r^{k+1} . theta^{k+1}) / (r^k . theta^k)
            p^{k+1} = theta^{k+1} + beta p^k

    P = None means the identity (plain CG).  ``callback(k, alpha)``, if given,
    sees each iterate alpha^k (k = 1, 2, ...); it changes no arithmetic, and a
    true return value ends the iteration there.

    ``alpha0`` (the streaming update's warm start, the paper's future work of
    Sec. VI): the iteration starts from alpha^0 = alpha0 with r^0 = y - A alpha0
    instead of 0 and y, and a start with |r^0| / |y| <= tol returns at once
    (0 iterations); the rest is unchanged."""
    y = np.asarray(y, dtype=np.float64)
    n = y.shape[0]
    if alpha0 is None:
        alpha = np.zeros(n)
        r = y.copy()
    else:
        alpha = np.array(alpha0, dtype=np.float64)
        r = y - A @ alpha
    theta = r.copy() if P is None else P @ r
    p = theta.copy()
    rtheta = float(r @ theta)
    ny = float(np.linalg.norm(y))
    hist = []
    if ny == 0.0:
        return PCGResult(alpha=alpha, iterations=0, converged=True, rel_res=hist)
    if alpha0 is not None and float(np.linalg.norm(r)) / ny <= tol:
        return PCGResult(alpha=alpha, iterations=0, converged=True, rel_res=hist)
    for k in range(max_iter):
        Ap = A @ p
        delta = rtheta / float(p @ Ap)
        alpha = alpha + delta * p
        r = r - delta * Ap
        if callback is not None and callback(k + 1, alpha):
            return PCGResult(alpha=alpha, iterations=k + 1, converged=False, rel_res=hist)
        rel = float(np.linalg.norm(r)) / ny
        hist.append(rel)
        if rel <= tol:
            return PCGResult(alpha=alpha, iterations=k + 1, converged=True, rel_res=hist)
        theta = r.copy() if P is None else P @ r
        rtheta_new = float(r @ theta)
        beta = rtheta_new / rtheta
        rtheta = rtheta_new
        p = theta + beta * p
    return PCGResult(alpha=alpha, iterations=max_iter, converged=False, rel_res=hist)


# ---------------------------------------------------------------------------
# Metrics (Sec. V-A)
# ---------------------------------------------------------------------------

def objective_R(G: np.ndarray, alpha: np.ndarray, y: np.ndarray, lam: float) -> float:
    """R(alpha) = |G alpha - y|^2 + lambda alpha^T G alpha  (Eq. simu-R-definition)."""
    Ga = G @ alpha
    return float(np.sum((Ga - y) ** 2) + lam * alpha @ Ga)


def relative_residual(A: np.ndarray, alpha: np.ndarray, y: np.ndarray) -> float:
    """Res. = |(lambda I + G) alpha - y| / |y|  (Eq. residual)."""
    return float(np.linalg.norm(A @ alpha - y) / np.linalg.norm(y))


def objective_gap(G, alpha, alpha_ref, y, lam) -> float:
    """|R(alpha) - R(alpha_ref)| / |R(alpha_ref)|  (Eq. objective-gap)."""
    r0 = objective_R(G, alpha_ref, y, lam)
    return abs(objective_R(G, alpha, y, lam) - r0) / abs(r0)


def prediction_discrepancy(G, alpha, alpha_ref) -> float:
    """|G alpha - G alpha_ref| / |G alpha_ref|  (Eq. prediction-discrepancy)."""
    g0 = G @ alpha_ref
    return float(np.linalg.norm(G @ alpha - g0) / np.linalg.norm(g0))


def rmse(pred: np.ndarray, truth: np.ndarray) -> float:
    """Eq. rmse."""
    return float(np.sqrt(np.mean((pred - truth) ** 2)))


def nmse(pred: np.ndarray, truth: np.ndarray) -> float:
    """Eq. nmse."""
    return float(np.sum((pred - truth) ** 2) / np.sum(truth ** 2))


def gradient_R(G: np.ndarray, alpha: np.ndarray, y: np.ndarray, lam: float) -> np.ndarray:
    """grad R(alpha) = 2 G (G alpha - y) + 2 lambda G alpha: the gradient of
    R(alpha) = |G alpha - y|^2 + lambda alpha^T G alpha (Eq. simu-R-definition)
    for a symmetric G."""
    Ga = G @ alpha
    return 2.0 * (G @ (Ga - y)) + 2.0 * lam * Ga


@dataclasses.dataclass
class GDResult:
    alpha: np.ndarray
    steps: int                 # gradient steps taken
    converged: bool
    rel_res: list              # |y - (lambda I + G) alpha^k| / |y| for k = 1 .. steps
    R: list                    # R(alpha^k) for k = 1 .. steps


def gradient_descent(G: np.ndarray, y: np.ndarray, lam: float, eta: float, max_iter: int,
                     tol: float = 0.0) -> GDResult:
    """The first-order baseline of Sec. V-A: alpha^0 = 0 and
    alpha^{k+1} = alpha^k - eta grad R(alpha^k); stop once the relative
    residual |y - (lambda I + G) alpha^k| / |y| <= tol or after max_iter
    steps.  (The paper tunes eta by grid search.)"""
    n = y.shape[0]
    alpha = np.zeros(n)
    A = G + lam * np.eye(n)
    ny = float(np.linalg.norm(y))
    res, Rs = [], []
    if ny == 0.0 or float(np.linalg.norm(y - A @ alpha)) <= tol * ny:
        return GDResult(alpha=alpha, steps=0, converged=True, rel_res=res, R=Rs)
    for k in range(1, max_iter + 1):
        alpha = alpha - eta * gradient_R(G, alpha, y, lam)
        rel = float(np.linalg.norm(y - A @ alpha)) / ny
        res.append(rel)
        Rs.append(objective_R(G, alpha, y, lam))
        if rel <= tol:
            return GDResult(alpha=alpha, steps=k, converged=True, rel_res=res, R=Rs)
    return GDResult(alpha=alpha, steps=max_iter, converged=False, rel_res=res, R=Rs)


def condition_number(A: np.ndarray, P: np.ndarray | None = None) -> float:
    """kappa(P A) (Sec. III-B, preconditioning objective).  For SPD P the
    eigenvalues of P A equal those of P^(1/2) A P^(1/2), which are real."""
    if P is None:
        w = np.linalg.eigvalsh(A)
    else:
        Ph = inverse_sqrt(np.linalg.inv(P))      # P^(1/2)
        w = np.linalg.eigvalsh(Ph @ A @ Ph)
    return float(w[-1] / w[0])


# ---------------------------------------------------------------------------
# The whole method on one instance (Algorithm 1)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class LakerResult:
    alpha: np.ndarray
    pcg: PCGResult
    cccp: CCCPResult | None
    P: np.ndarray | None
    map: np.ndarray | None


def laker(E: np.ndarray, y: np.ndarray, lam: float, scale: float, Z: np.ndarray,
          gamma: float = 0.1, rho: float | None = None, eps: float = 1e-8,
          tol: float = 1e-8, cccp_tol: float = 1e-10, cccp_max_iter: int = 200,
          Eg: np.ndarray | None = None, precond: str = "cccp") -> LakerResult:
    """Algorithm 1 end to end: kernel construction, preconditioner learning
    from the given directions Z (n x N_r), PCG, radio-map reconstruction."""
    n, n_r = Z.shape
    A = system_matrix(E, scale, lam)
    cc = None
    if precond == "cccp":
        Ubar = random_directions(A, Z)
        if rho is None:
            rho = shrinkage_rho(n, n_r, gamma)
        cc = cccp_fit(Ubar, gamma, rho, eps, max_iter=cccp_max_iter, tol=cccp_tol)
        P = inverse_sqrt(cc.Sigma)
    elif precond == "jacobi":
        P = jacobi_preconditioner(A)
    elif precond == "none":
        P = None
    else:
        raise ValueError(precond)
    res = pcg(A, y, P, tol)
    fmap = None if Eg is None else radio_map(Eg, E, res.alpha, scale)
    return LakerResult(alpha=res.alpha, pcg=res, cccp=cc, P=P, map=fmap)
