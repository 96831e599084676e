"""Pins of the warm-start network oracle: gradients against central finite
differences, the SiLU derivative against its difference quotient, and Adam's
first step (which moves every parameter by lr against its gradient sign)."""
import numpy as np
import pytest

from oracle import mlp


def test_silu_derivative():
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    assert np.allclose(mlp.silu_grad(z), fd, atol=1e-9)
    assert mlp.silu(0.0) == 0.0 and mlp.silu(50.0) == pytest.approx(50.0)


@pytest.mark.parametrize("seed", [0, 1])
def test_gradients_match_finite_differences(seed):
    rng = np.random.default_rng(seed)
    shapes = mlp.layer_shapes(6, 7, 3, 5)
    theta = rng.standard_normal(mlp.n_params(shapes)) * 0.4
    x = rng.standard_normal((9, 6))
    t = rng.standard_normal((9, 5))
    L, g = mlp.loss_and_grad(theta, shapes, x, t)
    h = 1e-6
    idx = rng.choice(theta.size, 60, replace=False)
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (mlp.loss_and_grad(theta + e, shapes, x, t)[0] - mlp.loss_and_grad(theta - e, shapes, x, t)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_adam_first_step_and_descent():
    rng = np.random.default_rng(3)
    shapes = mlp.layer_shapes(6, 16, 2, 4)
    theta = rng.standard_normal(mlp.n_params(shapes)) * 0.3
    x = rng.standard_normal((32, 6))
    t = np.tanh(x[:, :4])
    L0, g = mlp.loss_and_grad(theta, shapes, x, t)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    th1, m, v = mlp.adam_step(theta, g, m, v, 1, 1e-3)
    moved = th1 - theta
    nz = np.abs(g) > 1e-6
    assert np.allclose(moved[nz], -1e-3 * np.sign(g[nz]), rtol=1e-3)
    th = theta
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    for k in range(1, 301):
        L, g = mlp.loss_and_grad(th, shapes, x, t)
        th, m, v = mlp.adam_step(th, g, m, v, k, 1e-2)
    assert L < 0.2 * L0
