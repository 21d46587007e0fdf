"""Pins of the neural-operator oracle: convolution against numpy.correlate,
backpropagated gradients against central finite differences, and an Adam step
computed by hand."""
import numpy as np
import pytest

from oracle import nop_oracle as N


def test_single_channel_conv_is_correlation():
    rng = np.random.default_rng(0)
    m, K = 17, 5
    x = rng.standard_normal((1, 1, m))
    shapes = [(1, 1, K)]
    W = rng.standard_normal(K)
    theta = np.concatenate([W, [0.3]])
    y = N.forward(theta, shapes, x)
    ref = np.correlate(np.pad(x[0, 0], 2), W, mode="valid") + 0.3
    np.testing.assert_allclose(y[0, 0], ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("layers,K", [(2, 3), (3, 5)])
def test_gradient_matches_finite_differences(layers, K):
    rng = np.random.default_rng(layers)
    shapes = N.layer_shapes(cin=4, cout=3, width=5, layers=layers, K=K)
    P = N.num_params(shapes)
    theta = rng.standard_normal(P) * 0.4
    x = rng.standard_normal((2, 4, 11))
    t = rng.standard_normal((2, 3, 11))
    loss, g = N.loss_and_grad(theta, shapes, x, t)
    eps = 1e-6
    for i in rng.choice(P, 25, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (N.loss_and_grad(tp, shapes, x, t)[0] - N.loss_and_grad(tm, shapes, x, t)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_adam_step_by_hand():
    theta = np.array([1.0, -2.0])
    g = np.array([0.5, -0.25])
    th, m1, m2 = N.adam_step(theta, g, np.zeros(2), np.zeros(2), t=1, lr=0.1)
    # first step: mhat = g, vhat = g^2 -> theta - lr * sign(g) (up to eps)
    np.testing.assert_allclose(th, theta - 0.1 * np.sign(g), rtol=1e-6)
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(m2, 0.001 * g * g)
