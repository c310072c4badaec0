"""Full-size checks at the benchmark's workload (n = 16384 clustered
locations, d = 32, lambda = 1e-4, 8 transmitters, 512 x 512 grid), in the
launch configuration the benchmark times.  The oracle cannot run the whole
path at this size, so the checks are properties and sampled outputs: the
float64-accurate residual of every returned alpha (evaluated by the oracle's
dense float64 operator), and the radio map on sampled grid points computed
one by one by the oracle, compared in dB.
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


def test_c2_solves_and_map_full_size(L):
    import torch

    def dev(x):
        return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")

    ctx = L.Context(0)
    c = synth.CONFIGS["n16384_d32"]
    inst = synth.make_instance(c["n"], c["d"], c["lam"], n_tx=c["n_tx"], seed=2000, layout=c["layout"],
                               grid=c["grid"])
    n = inst.n
    Z = synth.directions(n, synth.default_num_directions(n), 2000)
    A = O.system_matrix(inst.Q, inst.scale, inst.lam)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(inst.Qg.shape[0], 256, replace=False))
    Qs = inst.Qg[idx]
    alphas = {}
    for prec, refine in ((L.FP64, 0), (L.FP32, 20), (L.BF16X3, 20)):
        op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, prec)
        P = L.laker_fit_preconditioner(ctx, op, dev(Z))
        alpha, info = L.laker_pcg_solve(ctx, op, P, dev(inst.y), c["tol"], max_iter=20000, refine_every=refine)
        a = alpha.cpu().numpy()
        res = O.relative_residual(A, a, inst.y)
        assert res <= c["tol"] * (1 + 1e-6), (prec, res, info)
        assert abs(info["rel_res_true"] - res) <= 1e-8
        # the GPU map on sampled grid points against the oracle's, same alpha
        f = L.laker_eval_map(ctx, op, dev(Qs), alpha).cpu().numpy()
        fo = O.radio_map(Qs, inst.Q, a, inst.scale)
        assert math.sqrt(np.mean((inst.y_sigma * (f - fo)) ** 2)) < 1e-3
        alphas[prec] = a
    # mixed solutions against the float64 solution: map difference in dB
    f64 = O.radio_map(Qs, inst.Q, alphas[L.FP64], inst.scale)
    for prec in (L.FP32, L.BF16X3):
        fm = O.radio_map(Qs, inst.Q, alphas[prec], inst.scale)
        db = math.sqrt(np.mean((inst.y_sigma * (fm - f64)) ** 2))
        assert db <= 0.01, (prec, db)
