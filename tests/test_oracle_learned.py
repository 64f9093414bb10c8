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
    X = rng.standard_normal((3, 3, 3, 8))
    Ws = learned.init_weights(rng)
    Y1, _ = learned.forward(X, Ws)
    Y2, _ = learned.forward(2.5 * X, Ws)
    assert np.allclose(Y2, 2.5 * Y1)


def _placement(shape):
    """An injective placement of node outputs (nodes, 3) on a 'face' vector and
    its adjoint (the same ravel order both ways)."""
    def faces_of(Y):
        return Y.reshape(-1)

    def nodes_of(v):
        return v.reshape(shape + (3,))
    return faces_of, nodes_of


def _residual_problem(rng, shape=(3, 4, 5)):
    X = rng.standard_normal(shape + (8,))
    Ws = learned.init_weights(rng, 8, 4, 3)
    Ws[2] = Ws[2] * 10
    n = int(np.prod(shape)) * 3
    B = rng.standard_normal((n, n)) / np.sqrt(n)
    K = B + B.T + 2.0 * np.eye(n)            # symmetric, like K - sigma A
    m = (rng.random(n) > 0.25).astype(float)
    s = m * rng.standard_normal(n)
    return X, Ws, K, m, s


def test_residual_objective_gradients_match_finite_differences():
    rng = np.random.default_rng(4)
    X, Ws, K, m, s = _residual_problem(rng)
    fo, no = _placement(X.shape[:3])
    h2 = 0.3
    loss, Gs, dX = learned.residual_loss_and_grads(X, s, Ws, K, h2, fo, no, m)
    eps = 1e-6
    for li in range(3):
        for idx in [tuple(rng.integers(0, d) for d in Ws[li].shape) for _ in range(6)]:
            Wp = [w.copy() for w in Ws]; Wp[li][idx] += eps
            Wm = [w.copy() for w in Ws]; Wm[li][idx] -= eps
            fd = (learned.residual_loss_and_grads(X, s, Wp, K, h2, fo, no, m)[0]
                  - learned.residual_loss_and_grads(X, s, Wm, K, h2, fo, no, m)[0]) / (2 * eps)
            assert abs(fd - Gs[li][idx]) <= 1e-6 * max(1.0, abs(fd)), (li, idx, fd, Gs[li][idx])


def test_residual_objective_with_scaled_identity_is_the_mse_objective():
    """K = h^-2 I: the correction's residual is s - y, so the objective is the
    masked MSE against the target s placed on the nodes."""
    rng = np.random.default_rng(5)
    X, Ws, _, m, s = _residual_problem(rng)
    fo, no = _placement(X.shape[:3])
    h2 = 0.25
    K = np.eye(s.size) / h2
    lr, Gr, _ = learned.residual_loss_and_grads(X, s, Ws, K, h2, fo, no, m)
    lm, Gm, _ = learned.loss_and_grads(X, no(s), no(m), Ws)
    assert lr == pytest.approx(lm, rel=1e-12)
    for a, b in zip(Gr, Gm):
        assert np.allclose(a, b, rtol=1e-10, atol=1e-14)


def test_adam_first_step_moves_by_lr_against_the_gradient_sign():
    rng = np.random.default_rng(6)
    Ws = [rng.standard_normal((4, 3)), rng.standard_normal(5)]
    Gs = [rng.standard_normal((4, 3)), rng.standard_normal(5) * 1e-3]
    state = {"t": 0, "m": [np.zeros_like(w) for w in Ws], "v": [np.zeros_like(w) for w in Ws]}
    lr = 0.01
    out = learned.adam_step(Ws, Gs, state, lr=lr)
    for w0, w1, g in zip(Ws, out, Gs):
        # bias correction makes m_hat = g and v_hat = g^2 after one step
        assert np.allclose(w1 - w0, -lr * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
        assert np.allclose(np.abs(w1 - w0), lr, rtol=1e-4)


def test_adam_constant_gradient_keeps_the_step_length():
    rng = np.random.default_rng(7)
    W = [rng.standard_normal(6)]
    g = [rng.standard_normal(6)]
    state = {"t": 0, "m": [np.zeros(6)], "v": [np.zeros(6)]}
    lr = 0.05
    for t in range(1, 6):
        W1 = learned.adam_step(W, g, state, lr=lr)
        # with a constant gradient both bias-corrected moments equal g and g^2 at every step
        assert np.allclose(W1[0] - W[0], -lr * g[0] / (np.abs(g[0]) + 1e-8), rtol=1e-10), t
        W = W1
