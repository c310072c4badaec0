"""The allocation-free radio map (laker_eval_map_noalloc).

Callers that cannot call cudaMalloc -- because another allocator owns the
device memory, or because they must not synchronise the device -- use this
entry point; it takes its scratch from a static device array inside the
library.  These tests call it through the C ABI and check it against the
allocating map with the same (double-float / float64) method on the same inputs, twice in a row (the second call
runs on the scratch the first one left behind), for a float64 operator and a
double-float (FP32) one, and check that oversized requests are refused.
This file is collected last so that a stop-at-first-failure run has already
run every other test.
"""
import math

import numpy as np
import pytest

from paper_2604_25138_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2604_25138_gb300 import build, laker
    build.build()
    return laker


@pytest.mark.parametrize("precision,n,d,m", [(0, 700, 16, 1000), (1, 1500, 32, 2049)])
def test_noalloc_map_matches_allocating_map_twice(L, precision, n, d, m):
    import torch
    ctx = L.Context(0)
    inst = synth.make_instance(n, d, 1e-3, seed=70 + d, grid=int(math.ceil(math.sqrt(m))))

    def dev(x):
        return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")

    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, precision)
    Qg = dev(inst.Qg[:m])
    for call in range(2):
        alpha = dev(synth.random_vector(n, 100 * call + d) * 1e3)
        ref = L.laker_eval_map(ctx, op, Qg, alpha, method=L.MAP_DOUBLE_FLOAT).cpu().numpy()
        out = torch.full((m,), float("nan"), dtype=torch.float64, device="cuda")
        got = L.laker_eval_map_noalloc(ctx, op, Qg, alpha, out).cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-10, call


def test_noalloc_map_refuses_oversized_requests(L):
    import torch
    ctx = L.Context(0)
    inst = synth.make_instance(64, 64, 1e-3, seed=3, grid=2)

    def dev(x):
        return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")

    op = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.FP32)
    m = 70000                      # 70000 * 64 * 8 bytes of double-float Qg alone exceed 32 MiB
    Qg = torch.zeros(m, 64, dtype=torch.float64, device="cuda")
    out = torch.zeros(m, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LakerError) as e:
        L.laker_eval_map_noalloc(ctx, op, Qg, dev(np.ones(64)), out)
    assert e.value.status == L.ERR_ARG
