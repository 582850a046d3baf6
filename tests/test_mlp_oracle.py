"""Pins of the FP64 reference of the learned-proposal network: analytic
backpropagation against central finite differences, and the Adam update
against its textbook first step (|step| = lr per coordinate)."""
import numpy as np

from oracle import mlp


def _params(rng, scale=0.05):
    p = rng.normal(0, scale, mlp.N_PARAMS)
    d = mlp.unpack(p)
    d["W4"][mlp.OUT:] = 0
    d["b4"][mlp.OUT:] = 0
    return mlp.pack(d)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = _params(rng)
    X = rng.normal(0, 1, (7, mlp.IN))
    Y = rng.normal(0, 1, (7, 3))
    g = mlp.grad(p, X, Y)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    d = mlp.unpack(np.arange(mlp.N_PARAMS, dtype=float))
    pad = set(d["W4"][mlp.OUT:].astype(int).ravel()) | set(d["b4"][mlp.OUT:].astype(int).ravel())
    for i in idx:
        if i in pad:
            continue
        h = 1e-6
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(p + e, X, Y) - mlp.loss(p - e, X, Y)) / (2 * h)
        assert abs(fd - g[i]) < 1e-5 * max(1e-3, abs(fd)), (i, fd, g[i])


def test_adam_first_step():
    rng = np.random.default_rng(1)
    p = rng.normal(size=10)
    g = rng.normal(size=10)
    p1, m, v = mlp.adam_step(p, g, np.zeros(10), np.zeros(10), 1, 1e-3)
    assert np.allclose(np.abs(p1 - p), 1e-3, rtol=1e-4)


def test_gelu_closed_form():
    """tanh-form GELU: GELU(z) - GELU(-z) = z exactly in real arithmetic,
    GELU(0) = 0, GELU -> z and -> 0 in the tails, within 1e-3 of the exact
    z Phi(z) everywhere, and the derivative matches finite differences."""
    from scipy.stats import norm

    z = np.linspace(-6.0, 6.0, 2401)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert np.allclose(mlp.gelu(z) - mlp.gelu(-z), z, atol=1e-14)
    assert np.max(np.abs(mlp.gelu(z) - z * norm.cdf(z))) < 1e-3
    assert abs(mlp.gelu(np.array([12.0]))[0] - 12.0) < 1e-12 and abs(mlp.gelu(np.array([-12.0]))[0]) < 1e-12
    h = 1e-6
    zz = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    assert np.allclose(mlp.gelu_grad(zz), (mlp.gelu(zz + h) - mlp.gelu(zz - h)) / (2 * h), atol=1e-8)
