"""Host arithmetic of the paper's numerical-layer metrics (Sec. V-A) on a PCG
trace: the condition-number estimate from the Lanczos tridiagonal of the CG
coefficients, and the iterations to an objective gap.

The trace layout is that of laker_pcg_solve_trace (per product: delta,
|r|^2/|y|^2, R(alpha), beta).  The coefficients here come from plain CG on
diagonal matrices with a known spectrum, which pins the estimate: its Ritz
values lie inside the spectrum, move outwards with k, and equal the extreme
eigenvalues once CG has terminated (finite termination on the distinct
eigenvalues, reached in floating point a few products later).  No GPU is
used; the library is loaded for its host functions.
"""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def L():
    from paper_2604_25138_gb300 import build, laker
    build.build()
    return laker


def _cg_trace(eigs, b, iters):
    """Textbook CG on diag(eigs) x = b; rows (delta, |r|^2/|b|^2, 0, beta)."""
    A = np.asarray(eigs, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = r @ r
    rows = []
    for _ in range(iters):
        Ap = A * p
        delta = rr / (p @ Ap)
        x = x + delta * p
        r = r - delta * Ap
        rr_new = r @ r
        beta = rr_new / rr
        rows.append((delta, rr_new / (b @ b), 0.0, beta))
        if rr_new == 0.0:
            break
        p = r + beta * p
        rr = rr_new
    return np.array(rows)


def test_lanczos_extremes_reach_the_spectrum(L):
    eigs_distinct = np.array([1.0, 2.0, 5.0, 11.0, 40.0, 90.0, 300.0, 1e3, 4e3, 1e4])
    rng = np.random.default_rng(3)
    eigs = np.repeat(eigs_distinct, 3)               # 30 unknowns, 10 distinct eigenvalues
    b = rng.normal(size=eigs.size)
    # in floating point CG needs a few products beyond the 10 distinct
    # eigenvalues to drive the residual to rounding level
    trace = _cg_trace(eigs, b, 16)
    assert trace[-1, 1] < 1e-20
    lo, hi = L.laker_lanczos_extremes(trace)
    assert abs(lo - 1.0) < 1e-9 and abs(hi - 1e4) < 1e-9 * 1e4
    prev = (np.inf, 0.0)
    for k in range(1, trace.shape[0] + 1):
        lo_k, hi_k = L.laker_lanczos_extremes(trace, k)
        assert 1.0 - 1e-9 <= lo_k <= prev[0] + 1e-12 and prev[1] - 1e-9 <= hi_k <= 1e4 * (1 + 1e-12)
        prev = (lo_k, hi_k)


def test_lanczos_one_step_is_the_rayleigh_quotient(L):
    eigs = np.array([2.0, 3.0, 7.0])
    b = np.array([1.0, -2.0, 0.5])
    trace = _cg_trace(eigs, b, 1)
    lo, hi = L.laker_lanczos_extremes(trace, 1)
    rq = (b @ (eigs * b)) / (b @ b)                   # 1 / delta_0
    assert abs(lo - rq) < 1e-12 and abs(hi - rq) < 1e-12


def test_lanczos_rejects_bad_coefficients(L):
    bad = np.array([[0.0, 1.0, 0.0, 0.5]])
    with pytest.raises(L.LakerError):
        L.laker_lanczos_extremes(bad)


def test_gap_iterations(L):
    R = np.array([10.0, 3.0, 1.2, 1.01, 1.0005, 1.0])
    trace = np.zeros((R.size, 4))
    trace[:, 2] = R
    assert L.laker_trace_gap_iterations(trace, 1.0, 1e-3) == 5
    assert L.laker_trace_gap_iterations(trace, 1.0, 1e-1) == 4
    assert L.laker_trace_gap_iterations(trace, 2.0, 1e-6) == -1
