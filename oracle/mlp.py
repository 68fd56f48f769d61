"""FP64 CPU oracle of the warm-start MLP (forward, masked loss, gradient).

TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module.  It shares no code with the CUDA
library.

Network (the learned warm start of the throughput system): features x ->
h1 = GELU(W1 x + b1) -> h2 = GELU(W2 h1 + b2) -> y = W3 h2 + b3, with
GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2.  Loss: masked mean squared
error sum M (y - t)^2 / sum M over a batch.  Parameters are one flat vector:
W1 [H x I], b1 [H], W2 [H x H], b2 [H], W3 [O x H], b3 [O] (row-major).
"""
import math

import numpy as np

_erf = np.vectorize(math.erf, otypes=[np.float64])


def param_count(I, H, O):
    return H * I + H + H * H + H + O * H + O


def unpack(p, I, H, O):
    p = np.asarray(p, dtype=np.float64)
    k = 0
    out = []
    for shape in ((H, I), (H,), (H, H), (H,), (O, H), (O,)):
        size = int(np.prod(shape))
        out.append(p[k:k + size].reshape(shape))
        k += size
    assert k == p.size
    return out


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_prime(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(p, X, I, H, O):
    W1, b1, W2, b2, W3, b3 = unpack(p, I, H, O)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2
    h2 = gelu(z2)
    y = h2 @ W3.T + b3
    return y, (X, z1, h1, z2, h2)


def loss(p, X, T, M, I, H, O):
    y, _ = forward(p, X, I, H, O)
    M = np.asarray(M, dtype=np.float64)
    return float(np.sum(M * (y - T) ** 2) / np.sum(M))


def grad(p, X, T, M, I, H, O):
    """Gradient of `loss` by back-propagation, as one flat vector."""
    W1, b1, W2, b2, W3, b3 = unpack(p, I, H, O)
    y, (X, z1, h1, z2, h2) = forward(p, X, I, H, O)
    M = np.asarray(M, dtype=np.float64)
    dy = 2.0 * M * (y - T) / np.sum(M)
    gW3 = dy.T @ h2
    gb3 = dy.sum(axis=0)
    dz2 = (dy @ W3) * gelu_prime(z2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * gelu_prime(z1)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    return np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3)])
