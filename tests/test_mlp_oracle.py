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


def test_round_bf16_definition():
    """BF16 rounding (8 significant bits, ties to even) against torch's own
    float32 -> bfloat16 conversion, plus hand-checked ties."""
    import torch

    rng = np.random.default_rng(2)
    x = np.concatenate([rng.normal(0, 1, 4000), rng.normal(0, 1e-3, 2000), rng.normal(0, 50, 2000)])
    x32 = x.astype(np.float32)
    want = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.round_bf16(x32.astype(np.float64)), want)
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties go to the even
    # significand (1); 1 + 3 * 2^-8 between 1 + 2^-7 and 1 + 2^-6 goes up
    assert mlp.round_bf16(np.array([1 + 2.0 ** -8]))[0] == 1.0
    assert mlp.round_bf16(np.array([1 + 3 * 2.0 ** -8]))[0] == 1 + 2.0 ** -6
    assert mlp.round_bf16(np.array([-(1 + 3 * 2.0 ** -8)]))[0] == -(1 + 2.0 ** -6)
    assert mlp.round_bf16(np.array([0.0, 1.5, -0.375]))[:].tolist() == [0.0, 1.5, -0.375]


def test_bf16_operand_mode():
    """BF16-operand mode: the forward pass stays within the BF16 bound of the
    FP64 one, every gradient entry is bounded by its magnitude sum
    (|sum a b| <= sum |a| |b|), and the mode changes nothing when every
    operand is already BF16 and the hidden activations are rounded away
    (a network of zero hidden weights)."""
    rng = np.random.default_rng(3)
    p = _params(rng, 0.1)
    X = rng.normal(0, 1, (33, mlp.IN))
    Y = rng.normal(0, 1, (33, 3))
    o64, _ = mlp.forward(p, X)
    o16, _ = mlp.forward(p, X, bf16_operands=True)
    assert np.linalg.norm(o16 - o64) < 2.0 ** -6 * np.linalg.norm(o64)
    g, mag = mlp.grad(p, X, Y, bf16_operands=True, magnitudes=True)
    assert np.all(np.abs(g) <= mag * (1 + 1e-12) + 1e-300)
    g64 = mlp.grad(p, X, Y)
    assert np.linalg.norm(g - g64) < 2.0 ** -5 * np.linalg.norm(g64)
    # zero hidden and output weights: every output is the output bias, for
    # either mode; the first-layer gradient is then 0 in both
    d = mlp.unpack(p)
    for k in ("W2", "W3", "W4"):
        d[k][:] = 0.0
    d["b4"][: mlp.OUT] = mlp.round_bf16(rng.normal(0, 1, mlp.OUT))
    pz = mlp.pack(d)
    a, _ = mlp.forward(pz, X, bf16_operands=True)
    assert np.array_equal(a, np.broadcast_to(d["b4"][: mlp.OUT], a.shape))
    assert not np.any(mlp.unpack(mlp.grad(pz, X, Y, bf16_operands=True))["W1"])
