"""The seeded synthetic inputs (paper_2604_25138_gb300/synth.py) against the
input recipe they state: the N_r schedule at the sizes the measurements use,
the single-instance workloads, the ranges of the batching workload, the
embedding and the standardised observations, the clustered layout, and
determinism by seed.  Host logic only: no GPU, no method arithmetic."""
import math

import numpy as np
import pytest

from paper_2604_25138_gb300 import synth


@pytest.mark.parametrize("n,n_r", [(4, 4), (50, 15), (200, 29), (500, 45), (1000, 64), (1024, 64), (2000, 90),
                                   (2048, 91), (4000, 127), (4096, 128), (8000, 179), (16384, 256),
                                   (65536, 1024), (1 << 20, 1024)])
def test_num_directions_schedule(n, n_r):
    """min(n, 1024, max(ceil(2 sqrt n), ceil(n / 64))): the square-root branch
    below n = 16384, the linear one above, capped at 1024 and at n."""
    assert synth.default_num_directions(n) == n_r


def test_single_instance_workloads():
    C = synth.CONFIGS
    head = C["n65536_d64"]
    assert (head["n"], head["d"], head["lam"], head["layout"], head["grid"], head["tol"]) == \
        (65536, 64, 1e-4, "uniform", 512, 1e-6)
    mid = C["n16384_d32"]
    assert (mid["n"], mid["d"], mid["lam"], mid["layout"], mid["grid"], mid["tol"]) == \
        (16384, 32, 1e-4, "clustered", 512, 1e-6)
    small = C["n1024_fp64"]
    assert (small["n"], small["d"], small["lam"], small["n_tx"], small["tol"]) == (1024, 16, 1e-3, 3, 1e-8)
    assert synth.default_num_directions(head["n"]) == 1024
    assert synth.default_num_directions(mid["n"]) == 256
    assert synth.default_num_directions(small["n"]) == 64


def test_batch_specs_ranges_and_determinism():
    c = synth.CONFIGS["batch256"]
    a = synth.batch_specs(c["count"], 4000)
    assert len(a) == c["count"] == 256
    for s in a:
        assert c["n_lo"] <= s["n"] <= c["n_hi"]
        assert s["d"] in c["d_choices"]
        assert c["lam_lo"] <= s["lam"] <= c["lam_hi"]
        assert c["tx_lo"] <= s["n_tx"] <= c["tx_hi"]
        assert c["f_lo"] <= s["freq_hz"] <= c["f_hi"]
    # log-uniform n: the median sits near the geometric mean of the range
    med = float(np.median([s["n"] for s in a]))
    assert 0.6 < med / math.sqrt(c["n_lo"] * c["n_hi"]) < 1.6
    assert {s["d"] for s in a} == set(c["d_choices"])
    assert len({s["seed"] for s in a}) == len(a)
    assert a == synth.batch_specs(c["count"], 4000)
    assert a != synth.batch_specs(c["count"], 4001)


@pytest.mark.parametrize("layout", ["uniform", "clustered"])
def test_instance_shapes_embedding_and_standardised_y(layout):
    inst = synth.make_instance(600, 16, 1e-3, n_tx=3, seed=11, layout=layout, grid=8)
    assert inst.Q.shape == (600, 16) and inst.X.shape == (600, 2)
    assert inst.Qg.shape == (64, 16) and inst.Xg.shape == (64, 2) and inst.rss_grid.shape == (64,)
    assert np.all((inst.X >= 0.0) & (inst.X <= 1000.0))
    # standardised observations
    assert abs(inst.y.mean()) < 1e-12 and abs(inst.y.std() - 1.0) < 1e-12
    # random-feature rows sqrt(2/d) cos(.): |q|^2 <= 2, mean ~1
    nq = (inst.Q ** 2).sum(axis=1)
    assert np.all(nq <= 2.0 + 1e-12) and 0.7 < nq.mean() < 1.3
    assert inst.scale == pytest.approx(1.0 / math.sqrt(16))
    again = synth.make_instance(600, 16, 1e-3, n_tx=3, seed=11, layout=layout, grid=8)
    assert np.array_equal(inst.Q, again.Q) and np.array_equal(inst.y, again.y)
    other = synth.make_instance(600, 16, 1e-3, n_tx=3, seed=12, layout=layout, grid=8)
    assert not np.array_equal(inst.Q, other.Q)


def test_clustered_layout_concentrates_points():
    """30 % of the points in five blobs of sigma = 50 m: the fullest 50 m
    cell holds several times what a uniform layout's fullest cell holds."""
    def fullest(layout):
        X = synth._locations(np.random.default_rng(3), 10000, 1000.0, layout)
        h, _, _ = np.histogram2d(X[:, 0], X[:, 1], bins=20, range=[[0, 1000], [0, 1000]])
        return h.max()
    assert fullest("clustered") > 2.5 * fullest("uniform")


def test_directions_and_vectors_are_seeded_standard_normals():
    Z = synth.directions(4000, 50, 5)
    assert Z.shape == (4000, 50) and Z.flags["C_CONTIGUOUS"]
    assert abs(Z.mean()) < 0.01 and abs(Z.var() - 1.0) < 0.01
    assert np.array_equal(Z, synth.directions(4000, 50, 5))
    assert not np.array_equal(Z, synth.directions(4000, 50, 6))
    v = synth.random_vector(10000, 1)
    assert v.shape == (10000,) and np.array_equal(v, synth.random_vector(10000, 1))
