"""Pins of the FP64 MLP oracle: finite differences, closed forms (CPU only)."""
import numpy as np

from oracle import mlp


def test_gradient_against_central_differences():
    rng = np.random.default_rng(0)
    shapes = mlp.layer_shapes(5, 7, 3)
    theta = mlp.init_params(5, 7, 3, seed=1) + rng.normal(0, 0.05, mlp.n_params(5, 7, 3))
    x = rng.normal(size=(6, 5))
    y = rng.normal(size=(6, 3))
    loss, g = mlp.loss_and_grad(theta, x, y, shapes)
    fd = np.zeros_like(theta)
    h = 1e-6
    for i in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd[i] = (mlp.loss_and_grad(tp, x, y, shapes)[0] - mlp.loss_and_grad(tm, x, y, shapes)[0]) / (2 * h)
    assert np.linalg.norm(g - fd) <= 1e-6 * np.linalg.norm(fd)
    big = np.abs(fd) > 1e-3 * np.abs(fd).max()
    assert np.max(np.abs(g - fd)[big] / np.abs(fd)[big]) < 1e-5


def test_forward_reduces_to_a_linear_map_for_single_layer():
    """With no hidden layers the network is x W + b exactly."""
    rng = np.random.default_rng(1)
    shapes = mlp.layer_shapes(4, 0, 2, n_layers=0)
    theta = rng.normal(size=mlp.n_params(4, 0, 2, n_layers=0))
    x = rng.normal(size=(3, 4))
    W, b = mlp.unpack(theta, shapes)[0]
    out, _ = mlp.forward(theta, x, shapes)
    np.testing.assert_allclose(out, x @ W + b, rtol=1e-15)
    assert mlp.n_params(13, 256, 12) == 13 * 256 + 256 + 2 * (256 * 256 + 256) + 256 * 12 + 12


def test_silu_derivative_closed_form():
    z = np.linspace(-8, 8, 101)
    s = 1 / (1 + np.exp(-z))
    d = s * (1 + z * (1 - s))
    fd = ((z + 1e-6) / (1 + np.exp(-(z + 1e-6))) - (z - 1e-6) / (1 + np.exp(-(z - 1e-6)))) / 2e-6
    np.testing.assert_allclose(d, fd, rtol=1e-7, atol=1e-9)


def test_adam_first_step_is_signed_learning_rate():
    """With bias correction the first Adam step is lr * g / (|g| + eps): lr * sign(g)
    up to eps."""
    theta = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -1e-3, 2.0])
    new, m, v = mlp.adam_step(theta, g, np.zeros(3), np.zeros(3), 1, 0.01)
    np.testing.assert_allclose(new - theta, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
