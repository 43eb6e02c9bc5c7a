"""FP64 reference of the learned first-layer correction network (test
infrastructure; only the tests, the smoke check and the benchmark's baseline
leg may import it).

The network maps the 9 column features (u_x, |S| and leaf-area density at the
three cells above the ground) to 4 outputs (du_x, du_z, dtau_x, dtau_z):

    z  = (x - x_mean) / x_std
    h1 = tanh(W1 z + b1)          W1: 64 x 9
    h2 = tanh(W2 h1 + b2)         W2: 64 x 64
    h3 = tanh(W3 h2 + b3)         W3: 64 x 64
    o  = W4 h3 + b4               W4: 4 x 64
    y  = y_mean + y_std * o

trained on the mean squared error of o against the standardised targets,
L = mean over samples and outputs of (o - (y - y_mean) / y_std)^2, with Adam
(Kingma & Ba 2015).  The correction is applied as an extra acceleration of
the cells at y = 0: a = (lam * du_x - dtau_x, lam * du_z - dtau_z).

Pins: the forward pass, the gradient, Adam and the BF16 rounding are pinned
against closed forms, central differences and known values; the correction
rule (correction_accel: how the four outputs become an acceleration) is
pinned on hand-set outputs, one output at a time, with a planted swap of the
two stress outputs caught.  The rule has no definition outside this project
(the paper has no learned part); whether it helps is measured by the gain
test against the coarsened finer run.

Parameters travel as one flat FP32/FP64 vector in this order:
W1, b1, W2, b2, W3, b3, W4, b4 (row-major, rows = outputs), then
x_mean, x_std, y_mean, y_std.  The matrix products use numpy's matmul as a
library primitive; everything else is written out.
"""
from __future__ import annotations

import numpy as np

SIZES = [(64, 9), (64, 64), (64, 64), (4, 64)]
N_IN, N_OUT = 9, 4
N_WEIGHTS = sum(o * i + o for o, i in SIZES)       # trainable parameters
N_PARAMS = N_WEIGHTS + 2 * N_IN + 2 * N_OUT        # plus the normalisation


def unpack(theta):
    """Flat vector -> list of (W, b) and the normalisation (x_mean, x_std, y_mean, y_std)."""
    theta = np.asarray(theta, dtype=np.float64)
    layers, k = [], 0
    for o, i in SIZES:
        W = theta[k:k + o * i].reshape(o, i)
        k += o * i
        b = theta[k:k + o]
        k += o
        layers.append((W, b))
    xm, xs = theta[k:k + N_IN], theta[k + N_IN:k + 2 * N_IN]
    k += 2 * N_IN
    ym, ys = theta[k:k + N_OUT], theta[k + N_OUT:k + 2 * N_OUT]
    return layers, (xm, xs, ym, ys)


def pack(layers, norm):
    parts = []
    for W, b in layers:
        parts += [np.ravel(W), np.ravel(b)]
    parts += [np.ravel(v) for v in norm]
    return np.concatenate(parts).astype(np.float64)


def forward(theta, X, keep=False):
    """Outputs y (n x 4) for features X (n x 9); with keep, also the layer
    activations (z, h1, h2, h3, o) for the backward pass."""
    layers, (xm, xs, ym, ys) = unpack(theta)
    z = (np.asarray(X, dtype=np.float64) - xm) / xs
    acts = [z]
    h = z
    for l, (W, b) in enumerate(layers):
        a = h @ W.T + b
        h = np.tanh(a) if l < 3 else a
        acts.append(h)
    y = ym + ys * h
    return (y, acts) if keep else y


def loss(theta, X, Y):
    """Mean squared error of the network output against standardised targets."""
    layers, (xm, xs, ym, ys) = unpack(theta)
    _, acts = forward(theta, X, keep=True)
    t = (np.asarray(Y, dtype=np.float64) - ym) / ys
    return float(np.mean((acts[-1] - t) ** 2))


def gradient(theta, X, Y):
    """dL/dtheta for the trainable parameters (N_WEIGHTS values, same order as
    the flat vector), by the chain rule through the layers in reverse."""
    layers, (xm, xs, ym, ys) = unpack(theta)
    _, acts = forward(theta, X, keep=True)
    n = acts[0].shape[0]
    t = (np.asarray(Y, dtype=np.float64) - ym) / ys
    delta = 2.0 * (acts[-1] - t) / (n * N_OUT)       # dL/do
    grads = [None] * 4
    for l in range(3, -1, -1):
        W, _ = layers[l]
        h_in = acts[l]
        grads[l] = (delta.T @ h_in, delta.sum(axis=0))  # dL/dW_l, dL/db_l
        if l > 0:
            back = delta @ W                            # dL/dh_{l}
            delta = back * (1.0 - acts[l] ** 2)         # through tanh
    out = []
    for gW, gb in grads:
        out += [np.ravel(gW), np.ravel(gb)]
    return np.concatenate(out)


def adam_update(w, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015, Algorithm 1) at step number t >= 1;
    returns the new (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v


def correction_accel(theta, X, lam):
    """Layer-0 acceleration (n x 2: x and z components) from the outputs."""
    y = forward(theta, X)
    return np.stack([lam * y[:, 0] - y[:, 2], lam * y[:, 1] - y[:, 3]], axis=1)


def round_bf16(a):
    """Round FP32 values to the nearest BF16 (ties to even), returned as FP64:
    the values a BF16 tensor holds."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
