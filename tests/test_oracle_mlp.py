"""Pins of the oracle MLP: its chain-rule gradient equals central differences, and the
network reduces to its output bias when the last layer's weights vanish."""
import numpy as np

from oracle import mlp


def _setup(seed=0, nin=12, nh=8, nout=4, B=20):
    rng = np.random.default_rng(seed)
    P = nh * nin + nh + nh * nh + nh + nout * nh + nout
    theta = rng.normal(scale=0.4, size=P)
    x = rng.normal(size=(B, nin))
    t = rng.normal(size=(B, nout))
    return theta, x, t, nin, nh, nout


def test_gradient_matches_central_differences():
    theta, x, t, nin, nh, nout = _setup()
    g = mlp.gradient(theta, x, t, nin, nh, nout)
    idx = np.arange(theta.size)
    fd = mlp.numerical_gradient(theta, x, t, nin, nh, nout, idx)
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-9)


def test_zero_output_weights_give_bias():
    theta, x, t, nin, nh, nout = _setup(seed=1)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(theta, nin, nh, nout)
    W3[:] = 0.0
    y, _ = mlp.forward(theta, x, nin, nh, nout)
    assert np.allclose(y, np.broadcast_to(b3, y.shape))
    # and the loss is then the mean of (b3 - t)^2
    assert abs(mlp.loss(theta, x, t, nin, nh, nout) - np.mean((b3 - t) ** 2)) < 1e-14
