"""GPU warm-start network (BF16 tensor cores, FP32 accumulation) against the
FP64 CPU oracle: forward pass, gradients, and training progress.

The oracle is given the same BF16-rounded weights and inputs, so the
remaining differences come from the BF16 activations and gradients of the
GPU path: a few 1e-3 relative on outputs, gradient cosine above 0.999.
"""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def bf16_round(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def MLP():
    from paper_2112_05258_gb300 import load
    from paper_2112_05258_gb300.mlp import MLP as M
    load()
    return M


def _setup(MLP, seed, n_in=6, hidden=64, n_hidden=3, n_out=16, batch=128):
    rng = np.random.default_rng(seed)
    shapes = omlp.layer_shapes(n_in, hidden, n_hidden, n_out)
    theta = np.concatenate([np.concatenate([rng.standard_normal(r * c) / np.sqrt(c), 0.1 * rng.standard_normal(r)])
                            for r, c in shapes]).astype(np.float32)
    net = MLP(n_in, hidden, n_hidden, n_out, max_batch=(batch + 63) // 64 * 64)
    net.set_params(theta)
    theta_b = theta.astype(np.float64).copy()
    # weights are rounded to BF16 on the GPU, biases stay FP32
    o = 0
    for r, c in shapes:
        theta_b[o:o + r * c] = bf16_round(theta[o:o + r * c])
        o += r * c + r
    x = rng.standard_normal((batch, n_in)).astype(np.float32)
    return net, shapes, theta, theta_b, x, rng


def test_forward_matches_oracle(MLP):
    net, shapes, theta, theta_b, x, rng = _setup(MLP, 0)
    y = net.forward(x)
    yo, _ = omlp.forward(theta_b, shapes, bf16_round(x))
    assert np.abs(y - yo).max() < 2e-2 * np.abs(yo).max()
    assert np.allclose(net.params(), theta)


@pytest.mark.parametrize("hidden,batch", [(64, 128), (256, 256)])
def test_gradients_match_oracle(MLP, hidden, batch):
    net, shapes, theta, theta_b, x, rng = _setup(MLP, 1, hidden=hidden, n_out=64, batch=batch)
    dy = rng.standard_normal((batch, 64)).astype(np.float32) / batch
    g = net.grad(x, dy).astype(np.float64)
    go = omlp.grad_from_output(theta_b, shapes, bf16_round(x), bf16_round(dy))
    cos = g @ go / (np.linalg.norm(g) * np.linalg.norm(go))
    assert cos > 0.999, cos
    assert np.linalg.norm(g - go) / np.linalg.norm(go) < 3e-2
    # per layer as well (weights and biases of each layer point the same way)
    o = 0
    for r, c in shapes:
        for n in (r * c, r):
            a, b = g[o:o + n], go[o:o + n]
            o += n
            assert a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30) > 0.995


def test_training_reduces_loss(MLP):
    rng = np.random.default_rng(7)
    n_in, n_out, N = 6, 16, 2048
    X = rng.uniform(-1, 1, (N, n_in)).astype(np.float32)
    A = rng.standard_normal((n_in, n_out))
    T = np.tanh(X @ A).astype(np.float32)
    shapes = omlp.layer_shapes(n_in, 128, 3, n_out)
    theta = np.concatenate([np.concatenate([rng.standard_normal(r * c) / np.sqrt(c), np.zeros(r)])
                            for r, c in shapes]).astype(np.float32)
    net = MLP(n_in, 128, 3, n_out, max_batch=256)
    net.set_params(theta)
    net.set_data(X, T)
    order = np.concatenate([rng.permutation(N) for _ in range(40)])[:600 * 256]
    losses = net.train(order, 256, 2e-3)
    assert losses[-20:].mean() < 0.05 * losses[:5].mean()
    # the trained GPU network generalises like its own training loss
    y = net.forward(X[:256])
    assert np.mean((y - T[:256]) ** 2) < 2 * losses[-20:].mean() + 1e-4


@pytest.mark.parametrize("batch", [16, 80, 1040])
def test_ragged_batches_match_oracle(MLP, batch):
    # tiles of 128 rows with a ragged last tile (16, 80), several tiles and a
    # weight-gradient product over 1040 rows (a ragged last K chunk)
    net, shapes, theta, theta_b, x, rng = _setup(MLP, 3, hidden=256, n_out=64, batch=batch)
    y = net.forward(x)
    yo, _ = omlp.forward(theta_b, shapes, bf16_round(x))
    assert np.abs(y - yo).max() < 2e-2 * np.abs(yo).max()
    dy = rng.standard_normal((batch, 64)).astype(np.float32) / batch
    g = net.grad(x, dy).astype(np.float64)
    go = omlp.grad_from_output(theta_b, shapes, bf16_round(x), bf16_round(dy))
    assert g @ go / (np.linalg.norm(g) * np.linalg.norm(go)) > 0.999
