"""Rounding envelopes of the oracle's PCG (test helper).

Where an iteration index is decided by rounding -- CG's stopping index at a
tight tolerance, or the first product whose objective gap R(alpha_k) - R_ref
crosses TAR.TOL while the gap oscillates around it -- parity is checked
against the spread of the oracle's own index under changes that only move
rounding: random orderings of the summation in A p, and a symmetric 1e-12
relative perturbation of P.
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


def gap_envelope(A, G, y, P, lam, R_ref, gap, kmax, n_perm=8, seed=0):
    """(min, max) of the gap-crossing index over the plain oracle, n_perm
    permuted summation orders and a 1e-12 perturbation of P."""
    rng = np.random.default_rng(seed)
    ks = [gap_crossing(A, G, y, P, lam, R_ref, gap, kmax)]
    for _ in range(n_perm):
        ks.append(gap_crossing(_PermutedA(A, rng.permutation(len(y))), G, y, P, lam, R_ref, gap, kmax))
    if P is not None:
        E = rng.normal(size=P.shape)
        E = (E + E.T) * (1e-12 * np.linalg.norm(P) / np.linalg.norm(E + E.T))
        ks.append(gap_crossing(A, G, y, P + E, lam, R_ref, gap, kmax))
    ks = [k for k in ks if k is not None]
    return (min(ks), max(ks)) if ks else None
