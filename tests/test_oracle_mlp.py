"""Pins of the FP64 reference network of the learned closure: its gradient
against central finite differences (brute force, every parameter of a small
draw), and special cases with a closed form."""
import numpy as np
import pytest

from oracle import mlp


@pytest.mark.parametrize("lattice,delta", [(9, 0.0), (19, 0.0), (9, 0.1)])
def test_gradient_matches_finite_differences(lattice, delta):
    nin, nout = mlp.dims(lattice)
    rng = np.random.default_rng(1)
    p = mlp.init_params(lattice, seed=2)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(scale=0.1, size=p[k].shape)
    x = rng.normal(size=(7, nin))
    t = rng.normal(size=(7, nout))
    _, g = mlp.loss_and_grad(p, x, t, delta)
    eps = 1e-6
    for name, arr in p.items():
        flat = arr.reshape(-1)
        idx = rng.choice(flat.size, size=min(flat.size, 25), replace=False)
        for j in idx:
            old = flat[j]
            flat[j] = old + eps
            lp, _ = mlp.loss_and_grad(p, x, t, delta)
            flat[j] = old - eps
            lm, _ = mlp.loss_and_grad(p, x, t, delta)
            flat[j] = old
            fd = (lp - lm) / (2 * eps)
            assert g[name].reshape(-1)[j] == pytest.approx(fd, rel=1e-6, abs=1e-10), (name, j)


def test_gelu_closed_forms():
    z = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert mlp.gelu_prime(np.array([0.0]))[0] == pytest.approx(0.5)
    # gelu(z) - gelu(-z) = z (the tanh form is odd-symmetric around z/2)
    assert np.allclose(mlp.gelu(z) - mlp.gelu(-z), z)
    h = 1e-6
    assert np.allclose(mlp.gelu_prime(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), atol=1e-8)


def test_zero_hidden_weights_give_bias():
    """With W3 = 0 the output is b3 and the loss gradient of b3 is the mean
    residual times 2 / OUT."""
    p = mlp.init_params(9, seed=3)
    p["W3"][:] = 0.0
    p["b3"] = np.array([0.1, -0.2, 0.3])
    x = np.random.default_rng(4).normal(size=(5, 8))
    t = np.zeros((5, 3))
    y, _ = mlp.forward(p, x)
    assert np.allclose(y, p["b3"])
    _, g = mlp.loss_and_grad(p, x, t)
    assert np.allclose(g["b3"], 2.0 * p["b3"] / 3)
