"""FP64 oracle of the per-face warm-start MLP (test infrastructure only).

The network is x (nin) -> tanh(W1 x + b1) -> tanh(W2 h1 + b2) -> W3 h2 + b3 (nout), the
loss the mean over the batch and the outputs of the squared error. Parameters are one
flat vector in the order W1 (row-major [nh][nin]), b1, W2 [nh][nh], b2, W3 [nout][nh], b3.
The backward pass is the chain rule written out; `numerical_gradient` is its pin.
"""
from __future__ import annotations

import numpy as np


def unpack(theta, nin, nh, nout):
    o = 0
    W1 = theta[o:o + nh * nin].reshape(nh, nin); o += nh * nin
    b1 = theta[o:o + nh]; o += nh
    W2 = theta[o:o + nh * nh].reshape(nh, nh); o += nh * nh
    b2 = theta[o:o + nh]; o += nh
    W3 = theta[o:o + nout * nh].reshape(nout, nh); o += nout * nh
    b3 = theta[o:o + nout]; o += nout
    assert o == theta.size
    return W1, b1, W2, b2, W3, b3


def forward(theta, x, nin, nh, nout):
    W1, b1, W2, b2, W3, b3 = unpack(theta, nin, nh, nout)
    h1 = np.tanh(x @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ W3.T + b3, (h1, h2)


def loss(theta, x, t, nin, nh, nout):
    y, _ = forward(theta, x, nin, nh, nout)
    return float(np.mean((y - t) ** 2))


def gradient(theta, x, t, nin, nh, nout):
    """d loss / d theta by the chain rule."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, nin, nh, nout)
    y, (h1, h2) = forward(theta, x, nin, nh, nout)
    B = x.shape[0]
    dy = 2.0 * (y - t) / (B * nout)
    gW3 = dy.T @ h2
    gb3 = dy.sum(0)
    dz2 = (dy @ W3) * (1.0 - h2 ** 2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * (1.0 - h1 ** 2)
    gW1 = dz1.T @ x
    gb1 = dz1.sum(0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


def numerical_gradient(theta, x, t, nin, nh, nout, idx, h=1e-6):
    """Central differences of the loss for the parameters listed in idx."""
    out = np.zeros(len(idx))
    for n, i in enumerate(idx):
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        out[n] = (loss(tp, x, t, nin, nh, nout) - loss(tm, x, t, nin, nh, nout)) / (2 * h)
    return out
