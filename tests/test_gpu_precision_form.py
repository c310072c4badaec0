"""The precision form at its full size: n = 65536 uniform locations, d = 64,
lambda = 1e-4, 8 transmitters, matrix-free split-bf16 operator with the
float64-accurate residual every 20 products, N_r from the default schedule
(1024), tolerance 1e-6 on the true residual; compared with a float64 GPU run
of the same instance (materialised float64 operator, float64 PCG), and the
same generator at n = 8192 against the float64 oracle.

At these sizes the oracle cannot run the path, so the full-size checks are
properties and sampled outputs: the float64-accurate residual of the mixed
alpha (recomputed by the library's float64 operator), the mixed alpha against
the float64 GPU alpha, and the radio maps of both on sampled grid points in dB.
"""
import math

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


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def test_precision_form_n8192_against_oracle(L):
    """Same generator at n = 8192: the mixed GPU alpha meets the true relative
    residual 1e-6 by the oracle's dense float64 operator, lies within the
    residual's condition-number bound of the oracle's Cholesky solution, and
    its radio map on sampled grid points is within 0.01 dB of the map of the
    oracle's exact solution."""
    ctx = L.Context(0)
    c = synth.CONFIGS["n65536_d64"]
    n = 8192
    inst = synth.make_instance(n, c["d"], c["lam"], n_tx=c["n_tx"], seed=3101, layout=c["layout"], grid=64)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    a_star = O.solve_direct(A, inst.y)
    op = L.laker_build_kernel(ctx, _dev(inst.Q), inst.scale, inst.lam, L.BF16X3)
    Z = synth.directions(n, synth.default_num_directions(n), 3101)
    P = L.laker_fit_preconditioner(ctx, op, _dev(Z))
    alpha, info = L.laker_pcg_solve(ctx, op, P, _dev(inst.y), c["tol"], max_iter=40000, refine_every=20)
    a = alpha.cpu().numpy()
    res = O.relative_residual(A, a, inst.y)
    assert res <= c["tol"] * (1 + 1e-6), (res, info)
    assert abs(info["rel_res_true"] - res) <= 1e-8
    # |alpha - alpha*| <= |A^-1| |r| <= |r| / lambda
    assert np.linalg.norm(a - a_star) <= np.linalg.norm(A @ a - inst.y) / inst.lam * (1 + 1e-6)
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(inst.Qg.shape[0], 512, replace=False))
    Qs = inst.Qg[idx]
    f = L.laker_eval_map(ctx, op, _dev(Qs), alpha).cpu().numpy()
    f_star = O.radio_map(Qs, inst.Q, a_star, inst.scale)
    db = math.sqrt(np.mean((inst.y_sigma * (f - f_star)) ** 2))
    assert db <= 0.01, db


def test_precision_form_full_size_against_float64_gpu(L):
    """n = 65536, d = 64: the mixed form (tcgen05 operator, N_r = 1024) against
    a float64 GPU run of the same instance (float64 operator and PCG, CCCP with
    N_r = 512 for time): both meet the true tolerance by the float64 operator;
    alpha error of the mixed run relative to the float64 run and the map
    difference on 4096 sampled grid points (dB RMSE <= 0.01 dB)."""
    import torch
    ctx = L.Context(0)
    c = synth.CONFIGS["n65536_d64"]
    inst = synth.make_instance(c["n"], c["d"], c["lam"], n_tx=c["n_tx"], seed=3003, layout=c["layout"],
                               grid=c["grid"])
    n = inst.n
    rng = np.random.default_rng(2)
    Qs = _dev(inst.Qg[np.sort(rng.choice(inst.Qg.shape[0], 4096, replace=False))])
    y = _dev(inst.y)
    # mixed form
    op = L.laker_build_kernel(ctx, _dev(inst.Q), inst.scale, inst.lam, L.BF16X3)
    n_r = synth.default_num_directions(n)
    assert n_r == 1024
    P = L.laker_fit_preconditioner(ctx, op, _dev(synth.directions(n, n_r, 3003)))
    am, im = L.laker_pcg_solve(ctx, op, P, y, c["tol"], max_iter=40000, refine_every=20)
    w = torch.empty_like(am)
    L.laker_op_matvec(ctx, op, am, w, fp64=True)          # float64-accurate (lambda I + G) alpha
    res_m = float(torch.linalg.norm(y - w) / torch.linalg.norm(y))
    assert res_m <= c["tol"] * (1 + 1e-6), (res_m, im)
    fm = L.laker_eval_map(ctx, op, Qs, am)
    P.close()
    op.close()
    # float64 reference run
    op64 = L.laker_build_kernel(ctx, _dev(inst.Q), inst.scale, inst.lam, L.FP64)
    P64 = L.laker_fit_preconditioner(ctx, op64, _dev(synth.directions(n, 512, 3004)))
    a64, i64 = L.laker_pcg_solve(ctx, op64, P64, y, c["tol"], max_iter=40000)
    L.laker_op_matvec(ctx, op64, a64, w)
    res_64 = float(torch.linalg.norm(y - w) / torch.linalg.norm(y))
    assert res_64 <= c["tol"] * (1 + 1e-6), (res_64, i64)
    f64 = L.laker_eval_map(ctx, op64, Qs, a64)
    da = float(torch.linalg.norm(am - a64) / torch.linalg.norm(a64))
    db = math.sqrt(float(torch.mean((inst.y_sigma * (fm - f64)) ** 2)))
    print(f"n=65536 mixed: {im['iterations']} products, float64: {i64['iterations']} products, "
          f"alpha rel. diff {da:.2e}, map dB RMSE {db:.2e}")
    # |alpha_m - alpha_64| <= (|r_m| + |r_64|) / lambda
    bound = (res_m + res_64) * float(torch.linalg.norm(y)) / inst.lam / float(torch.linalg.norm(a64))
    assert da <= bound * (1 + 1e-6)
    assert db <= 0.01, db
