"""Pins of the warm-start MLP oracle: GELU values fixed by the normal CDF,
and the back-propagated gradient against central finite differences."""
import math

import numpy as np

from oracle import mlp


def test_gelu_values():
    z = np.array([0.0, 1.0, -1.0, 2.0, 8.0, -8.0])
    g = mlp.gelu(z)
    # GELU(z) = z Phi(z); Phi(1) = 0.8413447460685429, Phi(2) = 0.9772498680518208
    assert g[0] == 0.0
    assert abs(g[1] - 0.8413447460685429) < 1e-15
    assert abs(g[2] - (-1.0) * (1 - 0.8413447460685429)) < 1e-15
    assert abs(g[3] - 2 * 0.9772498680518208) < 1e-15
    assert abs(g[4] - 8.0) < 1e-12 and abs(g[5]) < 1e-12
    h = 1e-6
    assert np.allclose(mlp.gelu_prime(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), atol=1e-9)


def test_gradient_matches_finite_differences():
    I, H, O, B = 7, 9, 5, 6
    rng = np.random.default_rng(0)
    p = rng.normal(scale=0.5, size=mlp.param_count(I, H, O))
    X = rng.normal(size=(B, I))
    T = rng.normal(size=(B, O))
    M = (rng.random((B, O)) < 0.7).astype(float)
    g = mlp.grad(p, X, T, M, I, H, O)
    h = 1e-6
    for k in rng.choice(p.size, 60, replace=False):
        e = np.zeros_like(p)
        e[k] = h
        fd = (mlp.loss(p + e, X, T, M, I, H, O) - mlp.loss(p - e, X, T, M, I, H, O)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(fd))


def test_masked_entries_do_not_matter():
    I, H, O = 3, 4, 4
    rng = np.random.default_rng(1)
    p = rng.normal(size=mlp.param_count(I, H, O))
    X = rng.normal(size=(2, I))
    T = rng.normal(size=(2, O))
    M = np.array([[1, 1, 0, 0], [1, 0, 0, 0]], float)
    T2 = T.copy()
    T2[M == 0] += 100.0
    assert mlp.loss(p, X, T, M, I, H, O) == mlp.loss(p, X, T2, M, I, H, O)
