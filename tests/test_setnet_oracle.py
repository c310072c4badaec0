"""Pins of the set-network oracle (CPU): hand-derived gradients against
central finite differences, the set invariances the architecture fixes
(mean pooling over points, a shared per-direction head), and the Adam update
against its closed form on a quadratic."""
import numpy as np
import pytest

from oracle import setnet_oracle as S


def _tiny(seed=0, in_dim=5, H=8, Hd=4, n=7, K=3):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0.0, 0.4, size=S.num_params(in_dim, H, Hd))
    X = rng.normal(size=(n, in_dim))
    F = rng.normal(size=(K, 2))
    return theta, X, F, (in_dim, H, Hd)


def test_num_params_matches_layout():
    assert S.num_params(35) == 35 * 256 + 256 + 2 * (256 * 256 + 256) + 256 * 256 + 256 + 256 + 1 \
        + 258 * 64 + 64 + 64 + 1
    theta = np.arange(S.num_params(5, 8, 4), dtype=float)
    assert np.array_equal(S.pack(S.unpack(theta, 5, 8, 4), 5, 8, 4), theta)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_backward_matches_finite_differences(seed):
    theta, X, F, dims = _tiny(seed)
    rng = np.random.default_rng(100 + seed)
    batch = [(X, F, 0.3, rng.normal(size=F.shape[0])),
             (rng.normal(size=(4, dims[0])), rng.normal(size=(5, 2)), -1.2, rng.normal(size=5))]
    L, g = S.loss_and_grad(theta, batch, *dims)
    h = 1e-6
    fd = np.empty_like(theta)
    for k in range(theta.size):
        e = np.zeros_like(theta)
        e[k] = h
        fd[k] = (S.loss_and_grad(theta + e, batch, *dims)[0] - S.loss_and_grad(theta - e, batch, *dims)[0]) / (2 * h)
    assert np.linalg.norm(g - fd) / np.linalg.norm(fd) < 1e-6


def test_point_permutation_invariance_and_direction_equivariance():
    theta, X, F, dims = _tiny(3)
    c0, D0, _ = S.forward(theta, X, F, *dims)
    perm = np.random.default_rng(4).permutation(X.shape[0])
    c1, D1, _ = S.forward(theta, X[perm], F, *dims)
    assert abs(c0 - c1) < 1e-13 and np.allclose(D0, D1, atol=1e-13)
    pk = np.array([2, 0, 1])
    c2, D2, _ = S.forward(theta, X, F[pk], *dims)
    assert abs(c0 - c2) < 1e-13 and np.allclose(D2, D0[pk], atol=1e-13)
    # duplicating every point leaves the mean-pooled code unchanged
    c3, D3, _ = S.forward(theta, np.concatenate([X, X]), F, *dims)
    assert abs(c0 - c3) < 1e-13 and np.allclose(D0, D3, atol=1e-13)


def test_loss_is_zero_at_its_own_predictions():
    theta, X, F, dims = _tiny(5)
    c, D, _ = S.forward(theta, X, F, *dims)
    L, g = S.loss_and_grad(theta, [(X, F, c, D)], *dims)
    assert L < 1e-28 and np.linalg.norm(g) < 1e-12


def test_adam_first_step_moves_each_coordinate_by_lr():
    # after one step the bias-corrected ratio m^/sqrt(v^) is sign(g) (eps aside)
    theta = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    t1, m, v = S.adam_step(theta, np.zeros(3), np.zeros(3), g, 1, lr=0.1, eps=0.0)
    assert np.allclose(t1, theta - 0.1 * np.sign(g), atol=1e-15)
