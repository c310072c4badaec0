"""The split form of the radio map, modelled on the CPU.

For mixed operators the library evaluates r(x) = sum_i alpha_i exp(L_i),
L_i = s <q(x), q_i> (Eq. sc-radio-map-reconstruction), as

    m0 + s q(x).m1 + (s^2/2) q(x)^T M2 q(x) + sum_i alpha_i L_i^3 g(L_i),
    g(L) = sum_k L^k / (k+3)!,

with float64 moments m0 = sum alpha_i, m1 = sum alpha_i q_i,
M2 = sum alpha_i q_i q_i^T, and the remainder from float32 logits (three-piece
bf16 split of q sqrt(s), six cross products), a degree-5 float32 polynomial
for g and float32 row sums over 64 columns.  These tests model that arithmetic
in numpy on a small instance and check it against the float64 oracle map:
the identity itself, the accuracy of the polynomial, and that the split keeps
the map far inside 0.01 dB where a plain float32 map does not.
"""
import math

import numpy as np

from oracle import laker_oracle as O
from paper_2604_25138_gb300 import synth


def _bf16(x):
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def _split3(x):
    """x (float64) -> three bf16 pieces h + m + l."""
    h = _bf16(x.astype(np.float32))
    r = x - h.astype(np.float64)
    m = _bf16(r.astype(np.float32))
    l = _bf16((r - m.astype(np.float64)).astype(np.float32))
    return h, m, l


def _remainder_poly(deg=5, half_width=0.5):
    """Monomial coefficients of the interpolant of g at the Chebyshev nodes."""
    k = np.arange(deg + 1)
    x = half_width * np.cos((2 * k + 1) * math.pi / (2 * (deg + 1)))
    g = sum(x ** j / math.factorial(j + 3) for j in range(40))
    return np.linalg.solve(np.vander(x, deg + 1, increasing=True), g)


def _instance(n=2048, m=256, seed=3101):
    inst = synth.make_instance(n, 32, 1e-4, n_tx=8, seed=seed, layout="clustered", grid=64)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    alpha = O.solve_direct(A, inst.y)
    rng = np.random.default_rng(1)
    Qs = inst.Qg[np.sort(rng.choice(inst.Qg.shape[0], m, replace=False))]
    return inst, alpha, Qs


def test_split_identity_in_float64():
    """In float64 the split form is the map itself (a rearrangement of exp)."""
    inst, alpha, Qs = _instance(n=512, m=64)
    s = inst.scale
    L = s * (Qs @ inst.Q.T)
    r3 = np.exp(L) - 1.0 - L - 0.5 * L * L
    m1 = inst.Q.T @ alpha
    M2 = (inst.Q * alpha[:, None]).T @ inst.Q
    split = alpha.sum() + s * (Qs @ m1) + 0.5 * s * s * np.einsum("ia,ab,ib->i", Qs, M2, Qs) + r3 @ alpha
    exact = O.radio_map(Qs, inst.Q, alpha, s)
    assert np.max(np.abs(split - exact)) <= 1e-9 * np.max(np.abs(alpha)) * len(alpha) ** 0.5


def test_remainder_polynomial_accuracy():
    """Degree 5 at the Chebyshev nodes of [-1/2, 1/2]: relative error below
    1e-8 on the interval, well under float32 rounding."""
    c = _remainder_poly()
    x = np.linspace(-0.5, 0.5, 20001)
    g = sum(x ** j / math.factorial(j + 3) for j in range(40))
    p = np.polynomial.polynomial.polyval(x, c)
    assert np.max(np.abs(p - g) / g) < 1e-8
    # the leading coefficients are those of the series, 1/3! and 1/4!
    assert abs(c[0] - 1 / 6) < 1e-8 and abs(c[1] - 1 / 24) < 1e-8


def test_split_model_stays_inside_the_map_tolerance():
    """The float32 model of the tensor-core arithmetic against the float64 map
    of the same large, oscillating alpha: dB RMSE far below 0.01 dB, where a
    plain float32 map (float32 logits and exp) is off by more than 0.1 dB."""
    inst, alpha, Qs = _instance()
    s = inst.scale
    exact = O.radio_map(Qs, inst.Q, alpha, s)
    # remainder from six bf16 cross products with float32 accumulation
    xh, xm, xl = _split3(Qs * math.sqrt(s))
    yh, ym, yl = _split3(inst.Q * math.sqrt(s))
    f32 = lambda a, b: a.astype(np.float32) @ b.astype(np.float32).T
    L = (f32(xh, yh) + f32(xh, ym) + f32(xm, yh) + f32(xh, yl) + f32(xm, ym) + f32(xl, yh)).astype(np.float32)
    assert np.max(np.abs(L)) <= 0.5
    c = _remainder_poly().astype(np.float32)
    g = np.full_like(L, c[-1])
    for ck in c[-2::-1]:
        g = g * L + ck
    a32 = alpha.astype(np.float32)
    terms = (a32[None, :] * L) * (L * L) * g                      # alpha_j L^3 g(L), float32
    acc = np.zeros(len(Qs))
    for j0 in range(0, terms.shape[1], 64):                          # float32 sums over 64 columns
        part = np.zeros(len(Qs), dtype=np.float32)
        for j in range(j0, min(terms.shape[1], j0 + 64)):
            part = part + terms[:, j]
        acc += part.astype(np.float64)
    m1 = inst.Q.T @ alpha
    M2 = (inst.Q * alpha[:, None]).T @ inst.Q
    model = alpha.sum() + s * (Qs @ m1) + 0.5 * s * s * np.einsum("ia,ab,ib->i", Qs, M2, Qs) + acc
    db = inst.y_sigma * (model - exact)
    assert math.sqrt(np.mean(db ** 2)) < 1e-3, math.sqrt(np.mean(db ** 2))
    plain = np.exp(L).astype(np.float32) @ a32
    db_plain = inst.y_sigma * (plain.astype(np.float64) - exact)
    assert math.sqrt(np.mean(db_plain ** 2)) > 0.1
