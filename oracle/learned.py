"""Oracle: the learned smoother's 3-layer convolutional network (plain FP64 numpy).

The network is the library's own design for the learned smoother that sits inside
flexible GMRES next to the V-cycle preconditioner of the inner solve (the paper
itself has no learned part).  On the node grid of a level (shape (nz+1, ny+1,
nx+1)), with channel-last arrays X[k, j, i, c]:

    H1 = relu(conv(X, W1)),  H2 = relu(conv(H1, W2)),  Y = conv(H2, W3)

conv is a 3x3x3 cross-correlation with zero padding and no bias:

    conv(X, W)[k, j, i, o] = sum_{a, b, c in {0,1,2}} sum_q W[a, b, c, q, o] X[k+a-1, j+b-1, i+c-1, q]

Input channels (8): the residual on the x, y, z faces of each node (the faces
whose lower corner is the node), divided by its RMS over the open faces, then
the face fractions A_x, A_y, A_z, the cell fraction V of the node's cell, and a
zero channel.  Output channels (3): the predicted error on those faces, in
units of (RMS of r) * h^2.  Without biases, relu networks are positively
homogeneous, and the scaling above makes the prediction independent of the
residual's magnitude.

Two training objectives:
* ``loss_and_grads``: the masked mean squared error against a target error E;
* ``residual_loss_and_grads``: the residual the correction leaves, the one the
  library trains on:  0.5 |m (s - K (h^2 y))|^2 / n_open, where s = r / RMS(r)
  on the open faces, y = the network output placed on the faces, K the shifted
  operator K - sigma A (symmetric), m the open-face mask.  Its gradient with
  respect to y is -h^2 K m (s - K h^2 y) / n_open (K = K^T), which enters the
  same backward pass as the MSE gradient.
The optimiser is Adam (Kingma & Ba 2015), ``adam_step``.

Pins (tests/test_oracle_learned.py): single-channel conv equals
scipy.ndimage.correlate with zero padding (a library routine); a delta kernel
shifts; the analytic gradients of every weight and of the input match central
finite differences, for both objectives; with K = h^-2 I the residual objective
is the MSE objective with target s; Adam's first step moves every weight by lr
against its gradient's sign, and a constant gradient keeps moving it by lr.
"""
from __future__ import annotations

import numpy as np

OFFSETS = [(a, b, c) for a in range(3) for b in range(3) for c in range(3)]


def conv(X, W):
    """3x3x3 zero-padded cross-correlation. X: (nz, ny, nx, Cin), W: (3, 3, 3, Cin, Cout)."""
    nz, ny, nx, _ = X.shape
    P = np.pad(X, ((1, 1), (1, 1), (1, 1), (0, 0)))
    Y = np.zeros((nz, ny, nx, W.shape[4]))
    for a, b, c in OFFSETS:
        Y += P[a:a + nz, b:b + ny, c:c + nx, :] @ W[a, b, c]
    return Y


def conv_grad_input(dY, W):
    """d/dX of sum(dY * conv(X, W)): correlation of dY with the flipped,
    transposed kernel."""
    nz, ny, nx, _ = dY.shape
    P = np.pad(dY, ((1, 1), (1, 1), (1, 1), (0, 0)))
    dX = np.zeros((nz, ny, nx, W.shape[3]))
    for a, b, c in OFFSETS:
        # X[p + d] feeds Y[p] with W[d]; so dX[q] += dY[q - d] W[d]^T
        dX += P[2 - a:2 - a + nz, 2 - b:2 - b + ny, 2 - c:2 - c + nx, :] @ W[a, b, c].T
    return dX


def conv_grad_weight(X, dY):
    """d/dW of sum(dY * conv(X, W)): dW[a, b, c] = sum_p X[p + d]^T dY[p]."""
    nz, ny, nx, cin = X.shape
    P = np.pad(X, ((1, 1), (1, 1), (1, 1), (0, 0)))
    dW = np.zeros((3, 3, 3, cin, dY.shape[3]))
    for a, b, c in OFFSETS:
        Xs = P[a:a + nz, b:b + ny, c:c + nx, :].reshape(-1, cin)
        dW[a, b, c] = Xs.T @ dY.reshape(-1, dY.shape[3])
    return dW


def forward(X, Ws):
    W1, W2, W3 = Ws
    Z1 = conv(X, W1)
    H1 = np.maximum(Z1, 0.0)
    Z2 = conv(H1, W2)
    H2 = np.maximum(Z2, 0.0)
    Y = conv(H2, W3)
    return Y, (X, Z1, H1, Z2, H2)


def loss_and_grads(X, E, M, Ws):
    """Masked MSE 0.5 * sum(M (Y - E)^2) / sum(M) and its gradients."""
    Y, cache = forward(X, Ws)
    msum = max(float(M.sum()), 1.0)
    R = M * (Y - E)
    loss = 0.5 * float((R * (Y - E)).sum()) / msum
    dY = R / msum
    grads, dX = _backward(cache, dY, Ws)
    return loss, grads, dX


def _backward(cache, dY, Ws):
    """Weight gradients (and the input's) of a forward pass given dloss/dY."""
    X0, Z1, H1, Z2, H2 = cache
    W1, W2, W3 = Ws
    dW3 = conv_grad_weight(H2, dY)
    dH2 = conv_grad_input(dY, W3) * (Z2 > 0)
    dW2 = conv_grad_weight(H1, dH2)
    dH1 = conv_grad_input(dH2, W2) * (Z1 > 0)
    dW1 = conv_grad_weight(X0, dH1)
    dX = conv_grad_input(dH1, W1)
    return (dW1, dW2, dW3), dX


def residual_loss_and_grads(X, s_faces, Ws, K, h2, faces_of, nodes_of, open_mask):
    """The residual objective 0.5 |m (s - K h2 y)|^2 / n_open and its gradients.

    X: network input (nodes, 8 channels); s_faces: r / RMS(r) on the faces
    (natural face vector, zero on closed faces); K: the shifted operator as a
    (faces x faces) matrix; faces_of(Y) maps the network output (nodes, 3) to
    a face vector, nodes_of(v) the reverse (the adjoint placement);
    open_mask: 1 on open faces.  Returns (loss, (dW1, dW2, dW3), dX)."""
    Y, cache = forward(X, Ws)
    y = open_mask * faces_of(Y)
    res = open_mask * (s_faces - K @ (h2 * y))
    n = max(float(open_mask.sum()), 1.0)
    loss = 0.5 * float(res @ res) / n
    gy = -h2 * open_mask * (K.T @ res) / n          # dloss/dy on the faces
    dY = nodes_of(gy)
    grads, dX = _backward(cache, dY, Ws)
    return loss, grads, dX


def init_weights(rng, cin=8, hidden=16, cout=3):
    """He-normal initialisation (fan-in 27 * Cin)."""
    def he(ci, co):
        return rng.standard_normal((3, 3, 3, ci, co)) * np.sqrt(2.0 / (27 * ci))
    return [he(cin, hidden), he(hidden, hidden), he(hidden, cout) * 0.1]


def adam_step(Ws, Gs, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015), state = dict(t, m list, v list)."""
    state["t"] += 1
    t = state["t"]
    out = []
    for i, (W, G) in enumerate(zip(Ws, Gs)):
        state["m"][i] = b1 * state["m"][i] + (1 - b1) * G
        state["v"][i] = b2 * state["v"][i] + (1 - b2) * G * G
        mh = state["m"][i] / (1 - b1 ** t)
        vh = state["v"][i] / (1 - b2 ** t)
        out.append(W - lr * mh / (np.sqrt(vh) + eps))
    return out
