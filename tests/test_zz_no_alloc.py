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


def test_noalloc_map_at_the_scratch_edge_caps_the_slices(L):
    """A double-float request that fills the static scratch to within 192
    bytes: (m d + n d + n) * 8 bytes of inputs with m = 1000, d = 64,
    n = 63527 is 33546040 bytes, 33546240 after 256-byte alignment, and the
    partial sums take 8 m = 8000 more, 33554240 <= 32 MiB = 33554432.  Only one
    slice of partial sums fits, so the slice count is capped by the scratch
    (the allocating map takes ~76 slices here); the result must still match
    the allocating map.  One more training point (n = 63528) needs
    33554752 bytes and is refused."""
    import torch
    ctx = L.Context(0)
    d, m = 64, 1000

    def dev(x):
        return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")

    inst = synth.make_instance(63528, d, 1e-3, seed=77, grid=32)
    Qg = dev(inst.Qg[:m])
    out = torch.full((m,), float("nan"), dtype=torch.float64, device="cuda")
    op_over = L.laker_build_kernel(ctx, dev(inst.Q), inst.scale, inst.lam, L.FP32)
    alpha_over = dev(synth.random_vector(63528, 5))
    with pytest.raises(L.LakerError) as e:
        L.laker_eval_map_noalloc(ctx, op_over, Qg, alpha_over, out)
    assert e.value.status == L.ERR_ARG
    op_over.close()
    n = 63527
    op = L.laker_build_kernel(ctx, dev(inst.Q[:n]), inst.scale, inst.lam, L.FP32)
    alpha = dev(synth.random_vector(n, 6) * 1e3)
    ref = L.laker_eval_map(ctx, op, Qg, alpha, method=L.MAP_DOUBLE_FLOAT).cpu().numpy()
    for call in range(2):
        got = L.laker_eval_map_noalloc(ctx, op, Qg, alpha, out).cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-10, call


def test_noalloc_map_refuses_a_float64_request_over_4mi_rows(L):
    """For a float64 operator the scratch holds only the partial sums, at
    least 8 m bytes: m = 4 Mi + 1 query points need more than 32 MiB and are
    refused before any work is issued."""
    import torch
    ctx = L.Context(0)
    inst = synth.make_instance(64, 16, 1e-3, seed=4, grid=2)
    op = L.laker_build_kernel(ctx, torch.as_tensor(inst.Q, device="cuda"), inst.scale, inst.lam, L.FP64)
    m = (4 << 20) + 1
    Qg = torch.zeros(m, 16, dtype=torch.float64, device="cuda")
    out = torch.zeros(m, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LakerError) as e:
        L.laker_eval_map_noalloc(ctx, op, Qg, torch.ones(64, dtype=torch.float64, device="cuda"), out)
    assert e.value.status == L.ERR_ARG
