"""CUDA path vs the FP64 oracle, element by element on the same seeded inputs.

Tolerances: float64 operator products 1e-13 relative (summation order only);
float64 PCG alpha 1e-9 relative and iterations +-1 against the oracle's PCG
with the same preconditioner; float32 products 1e-6 relative.
"""
import math

import numpy as np
import pytest

from oracle import laker_oracle as O
from paper_2604_25138_gb300 import synth
from tests.pcg_envelope import tol_envelope, within_envelope

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2604_25138_gb300 import build, laker
    build.build()
    return laker


@pytest.fixture(scope="module")
def ctx(L):
    return L.Context(0)


def _inst(n, d, lam, seed, **kw):
    return synth.make_instance(n, d, lam, seed=seed, grid=kw.pop("grid", 8), **kw)


@pytest.mark.parametrize("n,d", [(1, 3), (7, 5), (64, 16), (100, 33), (1000, 16), (1031, 64)])
def test_matvec_fp64_matches_oracle(L, ctx, n, d):
    from tests.gpu_util import dev, host, rel
    inst = _inst(n, d, 1e-3, 100 + n)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.FP64)
    x = synth.random_vector(n, n)
    w = host(L.laker_op_matvec(ctx, op, dev(x)))
    assert rel(w, A @ x) < 1e-13


@pytest.mark.parametrize("n,d", [(5, 4), (300, 16), (2049, 32)])
def test_matvec_fp32_matches_oracle(L, ctx, n, d):
    from tests.gpu_util import dev, host, rel
    inst = _inst(n, d, 1e-3, 200 + n)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.FP32)
    x = synth.random_vector(n, n)
    assert rel(host(L.laker_op_matvec(ctx, op, dev(x))), A @ x) < 2e-6
    assert rel(host(L.laker_op_matvec(ctx, op, dev(x), fp64=True)), A @ x) < 1e-13


def _perm_ensemble(A, y, P, tol, k=6, seed=0):
    """The oracle's PCG under k random row/column orderings of the matvec sum:
    the spread of its own iteration counts under rounding-order changes."""
    rng = np.random.default_rng(seed)
    n = len(y)
    its = []
    for _ in range(k):
        perm = rng.permutation(n)
        Ap, inv = A[np.ix_(perm, perm)], np.argsort(perm)

        class PA:
            def __matmul__(self, p):
                return (Ap @ p[perm])[inv]
        its.append(O.pcg(PA(), y, P, tol).iterations)
    return min(its), max(its)


def _gap_tolerance(hist, target=1e-8, ratio=3.0):
    """A tolerance near `target` placed in a clean gap of a residual history:
    the first index k with hist[k] < 10 target whose residual is at least
    `ratio` times below every earlier one; tol = sqrt(min(hist[:k]) hist[k]).
    The stopping index is then not decided by rounding-level differences."""
    for k in range(1, len(hist)):
        lo = min(hist[:k])
        if hist[k] < 10 * target and lo >= ratio * hist[k]:
            return math.sqrt(lo * hist[k])
    return None


@pytest.mark.parametrize("n,lam", [(400, 1.0), (400, 1e-1), (1024, 1e-1)])
def test_pcg_fp64_cccp_iterations_exact(L, ctx, n, lam):
    """CCCP-preconditioned float64 PCG: the same number of products (+-1) as the
    oracle at a tolerance in a clean gap of the oracle's residual history;
    alpha within 1e-9 of the oracle's after 10 products and at tol 1e-10.
    (Later iterates of two equally exact float64 constructions of the same P
    drift apart by up to ~3e-8 before they converge again.)"""
    from tests.gpu_util import dev, host, rel
    inst = _inst(n, 16, lam, 31, grid=4)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    Z = synth.directions(n, 64, 31)
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.FP64)
    P = L.laker_fit_preconditioner(ctx, op, dev(Z))
    Pd = O.inverse_sqrt(O.cccp_fit(O.random_directions(A, Z), 0.1, O.shrinkage_rho(n, 64, 0.1), 1e-8).Sigma)
    full = O.pcg(A, inst.y, Pd, 1e-12)
    tol = _gap_tolerance(full.rel_res)
    assert tol is not None
    ref = O.pcg(A, inst.y, Pd, tol)
    alpha, info = L.laker_pcg_solve(ctx, op, P, dev(inst.y), tol)
    assert abs(info["iterations"] - ref.iterations) <= 1, (info, ref.iterations, tol)
    aK, _ = L.laker_pcg_solve(ctx, op, P, dev(inst.y), 0.0, max_iter=10, allow_maxiter=True)
    assert rel(host(aK), O.pcg(A, inst.y, Pd, 0.0, max_iter=10).alpha) < 1e-9
    a_t, _ = L.laker_pcg_solve(ctx, op, P, dev(inst.y), 1e-10)
    assert rel(host(a_t), O.pcg(A, inst.y, Pd, 1e-10).alpha) < 1e-9


@pytest.mark.parametrize("precond", ["none", "jacobi"])
def test_pcg_fp64_matches_oracle_envelope(L, ctx, precond):
    """kappa ~ 5e4 without a learned preconditioner: CG's stopping iteration moves
    by several steps under rounding-order changes alone, so the GPU count must
    lie in the oracle's own permutation envelope; alpha parity <= 1e-9 is
    checked at tol 1e-10 where it is well posed."""
    from tests.gpu_util import dev, host, rel
    inst = _inst(500, 16, 1e-2, 7)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.FP64)
    Po = None if precond == "none" else O.jacobi_preconditioner(A)
    Pg = None if precond == "none" else L.laker_precond_jacobi(ctx, op)
    lo, hi = _perm_ensemble(A, inst.y, Po, 1e-8)
    alpha, info = L.laker_pcg_solve(ctx, op, Pg, dev(inst.y), 1e-8)
    assert lo - 1 <= info["iterations"] <= hi + 1, (info, lo, hi)
    assert info["rel_res"] <= 1e-8
    assert abs(info["rel_res_true"] - O.relative_residual(A, host(alpha), inst.y)) < 1e-12
    ref = O.pcg(A, inst.y, Po, 1e-10)
    alpha, info = L.laker_pcg_solve(ctx, op, Pg, dev(inst.y), 1e-10)
    assert rel(host(alpha), ref.alpha) < 1e-9


def test_cccp_fit_matches_dense_oracle(L, ctx):
    from tests.gpu_util import dev, host, rel
    n, n_r = 256, 40
    inst = _inst(n, 8, 1e-2, 3)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    Z = synth.directions(n, n_r, 3)
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.FP64)
    P = L.laker_fit_preconditioner(ctx, op, dev(Z), gamma=0.1, rho=-1.0, eps=1e-8, max_iter=200, tol=1e-10)
    Ubar = O.random_directions(A, Z)
    rho = O.shrinkage_rho(n, n_r, 0.1)
    ref = O.cccp_fit(Ubar, 0.1, rho, 1e-8, max_iter=200, tol=1e-10)
    c, D, U = L.laker_precond_export(ctx, P)
    U = host(U)
    assert rel(U, Ubar) < 1e-13
    Sigma = c * np.eye(n) + (U * host(D)) @ U.T
    assert rel(Sigma, ref.Sigma) < 1e-9
    assert abs(P.info["iterations"] - ref.iterations) <= 1
    # Theorem 1: tr Sigma_* = n
    assert abs(np.trace(Sigma) - n) < 1e-9 * n
    # the preconditioner apply equals Sigma_*^-1/2 v
    Pd = O.inverse_sqrt(ref.Sigma)
    v = synth.random_vector(n, 11)
    assert rel(host(L.laker_precond_apply(ctx, P, dev(v))), Pd @ v) < 1e-9


def test_c1_end_to_end_fp64(L, ctx):
    """Plain FP64 single instance (n=1024, d=16, lambda=1e-3, 3 Tx, N_r=64,
    PCG to 1e-8, 64x64 map).  kappa(A) ~ 1e6: the fit must match the dense
    oracle; the PCG arithmetic is checked on a fixed number of steps and alpha
    at tol 1e-10; at tol 1e-8 the stopping iteration is decided by rounding
    (equivalent float64 constructions of the same P stop anywhere in
    322..360), so that count is checked against the oracle's own envelope
    (summation-order permutations and per-apply noise at the measured
    difference of the GPU's apply) and alpha against the exact solution."""
    from tests.gpu_util import dev, host, rel
    cfg = synth.CONFIGS["n1024_fp64"]
    inst = synth.make_instance(cfg["n"], cfg["d"], cfg["lam"], n_tx=cfg["n_tx"], seed=1001, grid=cfg["grid"])
    n = inst.n
    n_r = synth.default_num_directions(n)
    Z = synth.directions(n, n_r, 1001)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    ref = O.laker(inst.Q, inst.y, inst.lam, inst.scale, Z, tol=cfg["tol"], Eg=inst.Qg)
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.FP64)
    P = L.laker_fit_preconditioner(ctx, op, dev(Z))
    c, D, U = L.laker_precond_export(ctx, P)
    U = host(U)
    Sigma = c * np.eye(n) + (U * host(D)) @ U.T
    assert rel(Sigma, ref.cccp.Sigma) < 1e-11
    assert P.info["iterations"] == ref.cccp.iterations
    # fixed number of PCG steps: identical arithmetic up to rounding
    a10, _ = L.laker_pcg_solve(ctx, op, P, dev(inst.y), 0.0, max_iter=10, allow_maxiter=True)
    assert rel(host(a10), O.pcg(A, inst.y, ref.P, 0.0, max_iter=10).alpha) < 1e-9
    # converged to 1e-10: alpha parity
    a_t, _ = L.laker_pcg_solve(ctx, op, P, dev(inst.y), 1e-10)
    assert rel(host(a_t), O.pcg(A, inst.y, ref.P, 1e-10).alpha) < 1e-9
    # the configuration's tolerance: the stopping index against the oracle's
    # own rounding envelope (see test_c1_stopping_index_five_seeds)
    alpha, info = L.laker_pcg_solve(ctx, op, P, dev(inst.y), cfg["tol"])
    a = host(alpha)
    v = synth.random_vector(n, 2)
    pv_err = rel(host(L.laker_precond_apply(ctx, P, dev(v))), ref.P @ v)
    env = tol_envelope(A, inst.y, ref.P, cfg["tol"], p_rel=max(pv_err, 1e-15))
    assert within_envelope(info["iterations"], env), (info["iterations"], env)
    assert O.relative_residual(A, a, inst.y) <= 1e-8 * 1.01
    a_star = O.solve_direct(A, inst.y)
    assert rel(a, a_star) < 1e-8
    assert rel(ref.alpha, a_star) < 1e-8
    fmap = host(L.laker_eval_map(ctx, op, dev(inst.Qg), alpha))
    fref = O.radio_map(inst.Qg, inst.Q, a, inst.scale)
    assert rel(fmap, fref) < 1e-10
    db = inst.y_sigma * (fmap - ref.map)
    assert math.sqrt(np.mean(db ** 2)) < 1e-3


def test_zero_rhs_and_bad_inputs(L, ctx):
    from tests.gpu_util import dev, host
    inst = _inst(50, 4, 1e-2, 5)
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.FP64)
    alpha, info = L.laker_pcg_solve(ctx, op, None, dev(np.zeros(50)), 1e-8)
    assert info["iterations"] == 0 and np.all(host(alpha) == 0)
    bad = inst.y.copy()
    bad[3] = np.nan
    with pytest.raises(L.LakerError) as e:
        L.laker_pcg_solve(ctx, op, None, dev(bad), 1e-8)
    assert e.value.status == L.ERR_NONFINITE
    with pytest.raises(L.LakerError) as e:
        L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, -1.0, L.FP64)
    assert e.value.status == L.ERR_ARG
    # max_iter reached still writes the iterate
    alpha, info = L.laker_pcg_solve(ctx, op, None, dev(inst.y), 1e-30, max_iter=3, allow_maxiter=True)
    assert info["iterations"] == 3 and not info["converged"]


@pytest.mark.parametrize("prec", ["FP32", "BF16X3"])
def test_mixed_precond_apply_matches_oracle(L, ctx, prec):
    """Mixed operators keep the preconditioner in the orthonormal form
    P = c^-1/2 I + U~ diag(phi) U~^T (float32 U~) from an eigendecomposition
    stopped once its off-diagonal remainder is below c / 100; P v must match
    the oracle's dense Sigma_*^-1/2 v to well under that bound and stay
    positive definite.  Their directions are z_k rounded to bf16, so both
    sides get bf16-representable directions."""
    from tests.gpu_util import bf16_round, dev, host, rel
    n, n_r = 1024, 128
    inst = _inst(n, 16, 1e-3, 51)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    Z = bf16_round(synth.directions(n, n_r, 51))   # mixed fits use bf16 directions
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, getattr(L, prec))
    P = L.laker_fit_preconditioner(ctx, op, dev(Z))
    Pd = O.inverse_sqrt(O.cccp_fit(O.random_directions(A, Z), 0.1, O.shrinkage_rho(n, n_r, 0.1), 1e-8).Sigma)
    worst = 0.0
    for s in range(4):
        v = synth.random_vector(n, 60 + s)
        pv = host(L.laker_precond_apply(ctx, P, dev(v)))
        worst = max(worst, rel(pv, Pd @ v))
        assert float(v @ pv) > 0.0
    assert worst < 2e-3, worst
    # along the dominant eigenvector of Sigma_* (the smallest factor of P)
    w, V = np.linalg.eigh(np.linalg.inv(Pd @ Pd))
    top = V[:, -1]
    assert rel(host(L.laker_precond_apply(ctx, P, dev(top))), Pd @ top) < 2e-3


def test_fp32_mixed_refinement_reaches_true_tolerance(L, ctx):
    """Mixed form: float32 operator inside PCG, float64-accurate residual every
    20 products; the returned alpha meets the TRUE relative residual 1e-6
    (checked by the oracle's float64 operator)."""
    from tests.gpu_util import dev, host, rel
    n = 2048
    inst = _inst(n, 32, 1e-4, 17, layout="clustered")
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    Z = synth.directions(n, 128, 17)
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.FP32)
    P = L.laker_fit_preconditioner(ctx, op, dev(Z))
    alpha, info = L.laker_pcg_solve(ctx, op, P, dev(inst.y), 1e-6, refine_every=20)
    a = host(alpha)
    res = O.relative_residual(A, a, inst.y)
    assert res <= 1e-6 * (1 + 1e-6), (res, info)
    assert abs(info["rel_res_true"] - res) < 1e-9
    assert info["true_residuals"] >= 1
    a_star = O.solve_direct(A, inst.y)
    kappa_bound = 1.0 + n * np.mean(O.kernel_matrix(inst.Q, inst.scale)) / inst.lam
    assert rel(a, a_star) <= kappa_bound * 1e-6


@pytest.mark.parametrize("n,d,m", [(1000, 16, 333), (2048, 32, 4096), (777, 64, 1025)])
def test_map_double_float_matches_oracle(L, ctx, n, d, m):
    """Mixed operators evaluate the radio map in double-float arithmetic on the
    float32 pipes.  With |alpha| ~ |y| / lambda the map needs ~1e-10 relative
    accuracy per kernel value to stay well under 0.01 dB; checked against the
    float64 oracle map of the same alpha."""
    from tests.gpu_util import dev, host, rel
    inst = _inst(n, d, 1e-4, 40 + d, grid=int(math.ceil(math.sqrt(m))))
    Qg = inst.Qg[:m]
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    alpha = O.solve_direct(A, inst.y)           # large, oscillating coefficients
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.FP32)
    f = host(L.laker_eval_map(ctx, op, dev(Qg), dev(alpha), method=L.MAP_DOUBLE_FLOAT))
    fref = O.radio_map(Qg, inst.Q, alpha, inst.scale)
    db = inst.y_sigma * (f - fref)
    assert math.sqrt(np.mean(db ** 2)) < 1e-4
    assert rel(f, fref) < 1e-8


@pytest.mark.parametrize("n,d,m,prec", [(1000, 16, 333, 1), (2048, 32, 4096, 2), (777, 64, 1025, 1),
                                        (100, 32, 70, 2), (4097, 32, 20000, 2), (500, 33, 1000, 1)])
def test_map_tensor_split_matches_oracle(L, ctx, n, d, m, prec):
    """The tensor-core map: float64 moments for 1 + L + L^2/2 and tcgen05
    logits for the remainder L^3 g(L).  Against the float64 oracle map of the
    same (large, oscillating) alpha: the remainder's float32 errors weigh ~1e-3
    of a plain float32 map's, so the map stays far inside 0.01 dB (measured on
    the CPU model of the kernel: ~1e-4 dB at n = 8192).  Ragged m and n (not
    multiples of 256 and 128), one tile, and d = 16 / 32 / 64 cover the tile
    shapes; LAKER_MAP_AUTO takes the same path for mixed operators."""
    from tests.gpu_util import dev, host
    inst = _inst(n, d, 1e-4, 60 + d, grid=int(math.ceil(math.sqrt(m))))
    Qg = inst.Qg[:m]
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    alpha = O.solve_direct(A, inst.y)
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, prec)
    f = host(L.laker_eval_map(ctx, op, dev(Qg), dev(alpha), method=L.MAP_TENSOR))
    fref = O.radio_map(Qg, inst.Q, alpha, inst.scale)
    db = inst.y_sigma * (f - fref)
    assert math.sqrt(np.mean(db ** 2)) < 1e-3, math.sqrt(np.mean(db ** 2))
    assert np.max(np.abs(db)) < 5e-3
    auto = host(L.laker_eval_map(ctx, op, dev(Qg), dev(alpha)))
    assert np.array_equal(auto, f)


def test_map_tensor_split_on_a_float64_operator_and_its_bound(L, ctx):
    """The split form on request for a float64 operator (the default there is
    the float64 kernel), and its logit bound: with scale * max|q|^2 > 1/2 the
    tensor method is refused and AUTO falls back to the double-float kernel."""
    from tests.gpu_util import dev, host
    n, d, m = 1500, 32, 2000
    inst = _inst(n, d, 1e-3, 91, grid=45)
    Qg = inst.Qg[:m]
    alpha = O.solve_direct(O.system_matrix(inst.Q, inst.scale, inst.lam), inst.y)
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.FP64)
    fref = O.radio_map(Qg, inst.Q, alpha, inst.scale)
    f64 = host(L.laker_eval_map(ctx, op, dev(Qg), dev(alpha)))
    assert np.array_equal(f64, host(L.laker_eval_map(ctx, op, dev(Qg), dev(alpha), method=L.MAP_DOUBLE_FLOAT)))
    ft = host(L.laker_eval_map(ctx, op, dev(Qg), dev(alpha), method=L.MAP_TENSOR))
    assert math.sqrt(np.mean((inst.y_sigma * (ft - fref)) ** 2)) < 1e-3
    big = 4.0                                     # scale * max|q|^2 ~ 4 * 1.5 > 1/2
    op2 = L.laker_build_kernel(ctx, dev(inst.Q), big, inst.lam, L.FP32)
    with pytest.raises(L.LakerError):
        L.laker_eval_map(ctx, op2, dev(Qg), dev(alpha), method=L.MAP_TENSOR)
    fa = host(L.laker_eval_map(ctx, op2, dev(Qg), dev(alpha)))
    fr2 = O.radio_map(Qg, inst.Q, alpha, big)
    assert np.linalg.norm(fa - fr2) / np.linalg.norm(fr2) < 1e-8


@pytest.mark.parametrize("n,d", [(100, 16), (1000, 32), (4097, 32), (777, 64), (6000, 64)])
def test_matvec_bf16x3_matrix_free_matches_oracle(L, ctx, n, d):
    """tcgen05 matrix-free product: split-bf16 logits (float32 accumulate),
    ex2.approx, float32 row sums; ~1e-6 relative per kernel value.  At
    n = 6000, d = 64 each CTA takes ~7 tiles across block-row boundaries, so
    diagonal tiles fall between off-diagonal ones in the column-sum
    reduction, and the last block is ragged (112 rows)."""
    from tests.gpu_util import dev, host, rel
    inst = _inst(n, d, 1e-3, 300 + n)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.BF16X3)
    x = synth.random_vector(n, n)
    assert rel(host(L.laker_op_matvec(ctx, op, dev(x))), A @ x) < 1e-5
    assert rel(host(L.laker_op_matvec(ctx, op, dev(x), fp64=True)), A @ x) < 1e-13


def test_bf16x3_mixed_solve_reaches_true_tolerance(L, ctx):
    from tests.gpu_util import dev, host, rel
    n = 2048
    inst = _inst(n, 32, 1e-4, 18, layout="clustered")
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    Z = synth.directions(n, 128, 18)
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.BF16X3)
    P = L.laker_fit_preconditioner(ctx, op, dev(Z))
    alpha, info = L.laker_pcg_solve(ctx, op, P, dev(inst.y), 1e-6, refine_every=20)
    res = O.relative_residual(A, host(alpha), inst.y)
    assert res <= 1e-6 * (1 + 1e-6), (res, info)
    assert info["true_residuals"] >= 1


@pytest.mark.parametrize("prec,n,d,n_r", [("BF16X3", 1000, 16, 128), ("FP32", 777, 64, 200), ("BF16X3", 4097, 32, 131),
                                          ("FP32", 300, 33, 40)])
def test_mixed_directions_match_oracle(L, ctx, prec, n, d, n_r):
    """The fit's random directions u_k = (lambda I + G) z~_k / |.| for mixed
    operators: the tensor-core kernel (d <= 64; ragged n and a ragged last
    chunk of directions) and the SIMT fallback (d = 33), against the oracle's
    dense product with the same bf16 directions.  The kernel keeps each
    element of P = G_IJ in [1/2, 2) as bf16 hi + lo, ~2^-18 absolute, so the
    error of A z~_k grows like 2^-18 sqrt(n) |z~_k| (rounding errors of
    random sign), and relative to |A z~_k| it is largest for directions with a
    small component along A's dominant eigenvector: each column must be within
    8 times that bound, and the median column within 2e-5."""
    from tests.gpu_util import bf16_round, dev, host
    inst = _inst(n, d, 1e-3, 70 + n)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    Z = bf16_round(synth.directions(n, n_r, 70 + n))
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, getattr(L, prec))
    P = L.laker_fit_preconditioner(ctx, op, dev(Z), max_iter=1)
    _, _, U = L.laker_precond_export(ctx, P)
    Uo = O.random_directions(A, Z)
    err = np.linalg.norm(host(U) - Uo, axis=0)
    bound = 8 * 2.0 ** -18 * np.sqrt(n) * np.linalg.norm(Z, axis=0) / np.linalg.norm(A @ Z, axis=0)
    assert np.all(err <= bound + 1e-9), np.max(err / bound)
    assert np.median(err) < 2e-5, np.median(err)


@pytest.mark.parametrize("n,d", [(700, 16), (4097, 32), (2048, 64)])
def test_fp32_matrix_free_variant_matches_oracle(L, ctx, n, d):
    """FP32 operators (d <= 64) also have the matrix-free variant: the
    split-bf16 tensor-core product (~1e-6 relative) with the full float32
    pair kept for the float64-accurate product; a mixed solve on it reaches
    the true tolerance by the oracle's operator."""
    from tests.gpu_util import dev, host, rel
    inst = _inst(n, d, 1e-4, 500 + n, layout="clustered")
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.FP32, L.MATRIX_FREE)
    assert L.laker_op_describe(op)["variant"] == L.MATRIX_FREE
    x = synth.random_vector(n, n)
    assert rel(host(L.laker_op_matvec(ctx, op, dev(x))), A @ x) < 1e-5
    assert rel(host(L.laker_op_matvec(ctx, op, dev(x), fp64=True)), A @ x) < 1e-13
    P = L.laker_fit_preconditioner(ctx, op, dev(synth.directions(n, synth.default_num_directions(n), n)))
    alpha, info = L.laker_pcg_solve(ctx, op, P, dev(inst.y), 1e-6, max_iter=20000, refine_every=20)
    assert O.relative_residual(A, host(alpha), inst.y) <= 1e-6 * (1 + 1e-6)


@pytest.mark.parametrize("n", [1024, 16384])
def test_auto_variant_keeps_the_faster_product(L, ctx, n):
    """LAKER_AUTO on an FP32 operator times one product of each variant after
    the build and keeps the faster; the product of the kept variant is
    correct."""
    from tests.gpu_util import dev, host, rel
    inst = _inst(n, 32, 1e-4, 600 + n)
    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.FP32, L.AUTO)
    dsc = L.laker_op_describe(op)
    assert dsc["t_materialised_ms"] > 0 and dsc["t_matrix_free_ms"] > 0
    faster = L.MATRIX_FREE if dsc["t_matrix_free_ms"] < dsc["t_materialised_ms"] else L.MATERIALISED
    assert dsc["variant"] == faster, dsc
    print(f"n={n}: materialised {dsc['t_materialised_ms']:.3f} ms, matrix-free {dsc['t_matrix_free_ms']:.3f} ms")
    x = synth.random_vector(n, 3)
    rows = np.arange(0, n, max(1, n // 64))
    Gx = O.kernel_matrix(inst.Q[rows], inst.scale, inst.Q) @ x + inst.lam * x[rows]
    w = host(L.laker_op_matvec(ctx, op, dev(x)))[rows]
    assert rel(w, Gx) < 1e-5


def test_c1_stopping_index_five_seeds(L, ctx):
    """The small float64 workload (n = 1024, d = 16, lambda = 1e-3, 3 Tx, N_r = 64,
    tol 1e-8) on five seeds: the GPU's number of products lies within the
    oracle's own envelope of it (plain run, six summation-order permutations,
    six runs with per-apply noise at the measured difference between the
    GPU's float64 apply and the oracle's dense Sigma^-1/2 r), widened by the
    envelope's width.  Prints the distribution of GPU - oracle."""
    from tests.gpu_util import dev, host, rel
    cfg = synth.CONFIGS["n1024_fp64"]
    deltas = []
    for seed in (1001, 1002, 1003, 1004, 1005):
        inst = synth.make_instance(cfg["n"], cfg["d"], cfg["lam"], n_tx=cfg["n_tx"], seed=seed, grid=2)
        n = inst.n
        Z = synth.directions(n, synth.default_num_directions(n), seed)
        A = O.system_matrix(inst.Q, inst.scale, inst.lam)
        Pd = O.inverse_sqrt(O.cccp_fit(O.random_directions(A, Z), 0.1,
                                       O.shrinkage_rho(n, Z.shape[1], 0.1), 1e-8).Sigma)
        op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.FP64)
        P = L.laker_fit_preconditioner(ctx, op, dev(Z))
        alpha, info = L.laker_pcg_solve(ctx, op, P, dev(inst.y), cfg["tol"])
        v = synth.random_vector(n, seed)
        pv_err = rel(host(L.laker_precond_apply(ctx, P, dev(v))), Pd @ v)
        env = tol_envelope(A, inst.y, Pd, cfg["tol"], p_rel=max(pv_err, 1e-15), seed=seed)
        k0 = O.pcg(A, inst.y, Pd, cfg["tol"]).iterations
        deltas.append(info["iterations"] - k0)
        print(f"seed {seed}: GPU {info['iterations']}, oracle {k0}, envelope {env}, apply difference {pv_err:.1e}")
        assert within_envelope(info["iterations"], env), (seed, info["iterations"], env)
        assert O.relative_residual(A, host(alpha), inst.y) <= 1e-8 * 1.01
    print("GPU - oracle products over the seeds:", deltas)
