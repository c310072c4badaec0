"""Rounding envelopes of the oracle's PCG (test helper).

Where an iteration index is decided by rounding -- CG's stopping index at a
tight tolerance, or the first product whose objective gap R(alpha_k) - R_ref
crosses TAR.TOL while the gap oscillates around it -- parity is checked
against the spread of the oracle's own index under changes that only move
rounding: random orderings of the summation in A p, and symmetric
perturbations of P at the level at which two float64 constructions of it
agree (1e-9 relative).
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


def gap_envelope(A, G, y, P, lam, R_ref, gap, kmax, n_perm=8, p_rel=1e-9, n_pert=3, seed=0):
    """(min, max) of the gap-crossing index over the plain oracle, n_perm
    permuted summation orders and n_pert symmetric perturbations of P of
    relative size p_rel.  The default p_rel is the level at which the GPU's
    float64 P (low-rank CCCP form, Jacobi eigenvectors) agrees with the
    oracle's dense Sigma^-1/2 (|P v| to 1e-9 in the fit's parity tests)."""
    rng = np.random.default_rng(seed)
    ks = [gap_crossing(A, G, y, P, lam, R_ref, gap, kmax)]
    for _ in range(n_perm):
        ks.append(gap_crossing(_PermutedA(A, rng.permutation(len(y))), G, y, P, lam, R_ref, gap, kmax))
    if P is not None:
        for _ in range(n_pert):
            E = rng.normal(size=P.shape)
            E = E + E.T
            E *= p_rel * np.linalg.norm(P) / np.linalg.norm(E)
            ks.append(gap_crossing(A, G, y, P + E, lam, R_ref, gap, kmax))
    ks = [k for k in ks if k is not None]
    return (min(ks), max(ks)) if ks else None
