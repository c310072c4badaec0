"""Rounding envelopes of the oracle's PCG (test helper).

Where an iteration index is decided by rounding -- CG's stopping index at a
tight tolerance, or the first product whose objective gap R(alpha_k) - R_ref
crosses TAR.TOL while the gap oscillates around it -- parity is checked
against the spread of the oracle's own index under changes that only move
rounding: random orderings of the summation in A p, and relative noise in
every preconditioner apply at the level at which two float64 constructions
of it agree (1e-9).
"""
import numpy as np

from oracle import laker_oracle as O


class _PermutedA:
    """A p summed in the order of a random permutation of the indices."""

    def __init__(self, A, perm):
        self.Ap = A[np.ix_(perm, perm)]
        self.perm, self.inv = perm, np.argsort(perm)

    def __matmul__(self, v):
        return (self.Ap @ v[self.perm])[self.inv]


class _NoisyP:
    """P r with fresh relative noise of size eps on every application: the
    rounding of an apply whose error is ~eps |P r| (the GPU's float64
    low-rank apply c^-1/2 r + U B U^T r agrees with a dense P r to ~1e-9)."""

    def __init__(self, P, eps, rng):
        self.P, self.eps, self.rng = P, eps, rng

    def __matmul__(self, r):
        z = self.P @ r
        noise = self.rng.normal(size=z.shape)
        return z + noise * (self.eps * np.linalg.norm(z) / np.linalg.norm(noise))


def gap_crossing(A, G, y, P, lam, R_ref, gap, kmax):
    """First k (1-based) with |R(alpha_k) - R_ref| <= gap |R_ref| along the
    oracle's PCG iterates, or None within kmax products."""
    hit = []

    def cb(k, alpha):
        if abs(O.objective_R(G, alpha, y, lam) - R_ref) <= gap * abs(R_ref):
            hit.append(k)
            return True
        return False
    O.pcg(A, y, P, 0.0, max_iter=kmax, callback=cb)
    return hit[0] if hit else None


def gap_envelope(A, G, y, P, lam, R_ref, gap, kmax, n_perm=6, p_rel=1e-9, n_pert=6, seed=0):
    """(min, max) of the gap-crossing index over the plain oracle, n_perm
    permuted summation orders of A p and, for a preconditioner, n_pert runs
    whose every apply carries fresh relative noise p_rel.  The default p_rel
    is the level at which the GPU's float64 apply agrees with the oracle's
    dense Sigma^-1/2 r (1e-9 in the fit's parity tests): rounding at that
    level parts two CG runs after a few tens of products."""
    rng = np.random.default_rng(seed)
    ks = [gap_crossing(A, G, y, P, lam, R_ref, gap, kmax)]
    for _ in range(n_perm):
        ks.append(gap_crossing(_PermutedA(A, rng.permutation(len(y))), G, y, P, lam, R_ref, gap, kmax))
    if P is not None:
        for _ in range(n_pert):
            ks.append(gap_crossing(A, G, y, _NoisyP(P, p_rel, rng), lam, R_ref, gap, kmax))
    ks = [k for k in ks if k is not None]
    return (min(ks), max(ks)) if ks else None


def within_envelope(k, env):
    """k inside the envelope widened by its own width (at least 1): the range
    of a dozen rounding samples covers only part of the index's spread."""
    w = max(1, env[1] - env[0])
    return env[0] - w <= k <= env[1] + w


def tol_envelope(A, y, P, tol, n_perm=6, p_rel=1e-9, n_pert=6, seed=0, max_iter=100000):
    """(min, max) of the oracle's stopping index at a tolerance (the number
    of products of O.pcg) over the plain run, n_perm permuted summation
    orders of A p and n_pert runs with relative noise p_rel in every
    preconditioner apply."""
    rng = np.random.default_rng(seed)
    ks = [O.pcg(A, y, P, tol, max_iter=max_iter).iterations]
    for _ in range(n_perm):
        ks.append(O.pcg(_PermutedA(A, rng.permutation(len(y))), y, P, tol, max_iter=max_iter).iterations)
    if P is not None:
        for _ in range(n_pert):
            ks.append(O.pcg(A, y, _NoisyP(P, p_rel, rng), tol, max_iter=max_iter).iterations)
    return min(ks), max(ks)
