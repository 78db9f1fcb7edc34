"""FP64 reference of the learned stress closure's network (test
infrastructure only; see oracle/__init__.py).

The network maps the lambda-scaled local state of a node to its lambda-scaled
stress source:  x = (lambda d_a u_b [D x D, row-major], (A - I) [C compact],
dt / lambda [2D only])  ->  y = lambda chi [C compact], with
chi = -(A - I)/lambda + A.grad u + (grad u)^T.A (Sec. 2.3).  In these
variables the Oldroyd-B source does not depend on lambda.

Architecture: IN -> 64 -> 64 -> OUT, GELU in its tanh form
gelu(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))) (Hendrycks and
Gimpel), loss = mean over samples and outputs of (y - t)^2.  Parameters are
row-major weight matrices W[out][in] and bias vectors.  The backward pass is
written out by hand (chain rule, layer by layer); numpy's matmul is the only
library primitive used.
"""
from __future__ import annotations

import numpy as np

H = 64
C_GELU = np.sqrt(2.0 / np.pi)


def dims(lattice: int):
    """(inputs, outputs): D2Q9 8 -> 3, D3Q19 15 -> 6."""
    return (8, 3) if lattice == 9 else (15, 6)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(C_GELU * (z + 0.044715 * z ** 3)))


def gelu_prime(z):
    u = C_GELU * (z + 0.044715 * z ** 3)
    th = np.tanh(u)
    return 0.5 * (1.0 + th) + 0.5 * z * (1.0 - th * th) * C_GELU * (1.0 + 3 * 0.044715 * z * z)


def init_params(lattice: int, seed: int = 0):
    """He-style initialisation (for tests; the GPU library has its own)."""
    nin, nout = dims(lattice)
    rng = np.random.default_rng(seed)
    return dict(W1=rng.normal(scale=np.sqrt(2.0 / nin), size=(H, nin)), b1=np.zeros(H),
                W2=rng.normal(scale=np.sqrt(2.0 / H), size=(H, H)), b2=np.zeros(H),
                W3=rng.normal(scale=np.sqrt(1.0 / H), size=(nout, H)), b3=np.zeros(nout))


def forward(p, x):
    """x [n, IN] -> y [n, OUT] and the cache for backward."""
    z1 = x @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (x, z1, h1, z2, h2)


def loss_and_grad(p, x, t, delta=0.0):
    """Mean squared error over all outputs and its gradient.  With delta > 0
    each sample's error is weighted by 1 / (mean_o t_o^2 + delta^2), a
    relative error with a floor."""
    y, (x, z1, h1, z2, h2) = forward(p, x)
    n, nout = y.shape
    r = y - t
    w = np.ones((n, 1)) if delta <= 0 else 1.0 / ((t * t).mean(axis=1, keepdims=True) + delta * delta)
    loss = float((w * r * r).mean())
    dy = 2.0 * w * r / (n * nout)
    g = {}
    g["W3"] = dy.T @ h2
    g["b3"] = dy.sum(axis=0)
    dh2 = dy @ p["W3"]
    dz2 = dh2 * gelu_prime(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * gelu_prime(z1)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return loss, g
