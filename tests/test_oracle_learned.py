"""Pins of the learned-smoother network oracle (FP64)."""
import numpy as np
import pytest

from oracle import learned


def test_single_channel_conv_matches_library_correlation():
    nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(0)
    X = rng.standard_normal((5, 6, 7, 1))
    W = rng.standard_normal((3, 3, 3, 1, 1))
    ref = nd.correlate(X[..., 0], W[..., 0, 0], mode="constant", cval=0.0)
    assert np.allclose(learned.conv(X, W)[..., 0], ref, atol=1e-12)


def test_delta_kernel_shifts():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((4, 5, 6, 2))
    W = np.zeros((3, 3, 3, 2, 2))
    W[1, 1, 2, 0, 1] = 1.0          # out channel 1 <- in channel 0 at +1 in i
    Y = learned.conv(X, W)
    assert np.allclose(Y[:, :, :-1, 1], X[:, :, 1:, 0])
    assert np.allclose(Y[:, :, -1, 1], 0.0)
    assert np.allclose(Y[..., 0], 0.0)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((3, 4, 5, 7))
    E = rng.standard_normal((3, 4, 5, 3))
    M = (rng.random((3, 4, 5, 3)) > 0.3).astype(float)
    Ws = learned.init_weights(rng, 7, 4, 3)
    Ws[2] = Ws[2] * 10
    loss, Gs, dX = learned.loss_and_grads(X, E, M, Ws)
    eps = 1e-6
    for li in range(3):
        W = Ws[li]
        for idx in [tuple(rng.integers(0, s) for s in W.shape) for _ in range(6)]:
            Wp = [w.copy() for w in Ws]; Wp[li][idx] += eps
            Wm = [w.copy() for w in Ws]; Wm[li][idx] -= eps
            fd = (learned.loss_and_grads(X, E, M, Wp)[0] - learned.loss_and_grads(X, E, M, Wm)[0]) / (2 * eps)
            assert abs(fd - Gs[li][idx]) <= 1e-6 * max(1.0, abs(fd)), (li, idx, fd, Gs[li][idx])
    for idx in [tuple(rng.integers(0, s) for s in X.shape) for _ in range(6)]:
        Xp = X.copy(); Xp[idx] += eps
        Xm = X.copy(); Xm[idx] -= eps
        fd = (learned.loss_and_grads(Xp, E, M, Ws)[0] - learned.loss_and_grads(Xm, E, M, Ws)[0]) / (2 * eps)
        assert abs(fd - dX[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_network_is_positively_homogeneous():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((3, 3, 3, 7))
    Ws = learned.init_weights(rng)
    Y1, _ = learned.forward(X, Ws)
    Y2, _ = learned.forward(2.5 * X, Ws)
    assert np.allclose(Y2, 2.5 * Y1)
