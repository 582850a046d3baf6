"""Plain FP64 reference of the learned-proposal network (test infrastructure).

Network: x [256] -> Linear(256,128) -> GELU -> Linear(128,128) -> GELU ->
Linear(128,128) -> GELU -> Linear(128,6) -> (mean [3], log-variance [3]).
GELU in its tanh form (Hendrycks & Gimpel, "Gaussian Error Linear Units"):
GELU(z) = 0.5 z (1 + tanh(c (z + a z^3))), c = sqrt(2 / pi), a = 0.044715,
which stays within 1e-3 of z * Phi(z).
Loss (Gaussian negative log-likelihood, constant dropped, mean over rows):
L = 1/B sum_rows sum_d 0.5 ((y_d - mu_d)^2 exp(-s_d) + s_d).
Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).

Parameters are held in the flat layout the CUDA library uses:
[W1 (128x256), b1 (128), W2 (128x128), b2, W3 (128x128), b3, W4 (16x128), b4 (16)],
weights as [out][in]; rows 6..15 of W4 and b4[6:] are padding and stay 0.
"""
import math

import numpy as np

IN, HID, OUTP, OUT = 256, 128, 16, 6
SHAPES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (HID, HID)),
          ("b3", (HID,)), ("W4", (OUTP, HID)), ("b4", (OUTP,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)

_C = math.sqrt(2.0 / math.pi)
_A = 0.044715


def unpack(flat):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + n], np.float64).reshape(shp)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SHAPES])


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(_C * (z + _A * z ** 3)))


def gelu_grad(z):
    t = np.tanh(_C * (z + _A * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * _C * (1.0 + 3.0 * _A * z * z)


def forward(params, X):
    p = unpack(params)
    X = np.asarray(X, np.float64)
    Z1 = X @ p["W1"].T + p["b1"]
    H1 = gelu(Z1)
    Z2 = H1 @ p["W2"].T + p["b2"]
    H2 = gelu(Z2)
    Z3 = H2 @ p["W3"].T + p["b3"]
    H3 = gelu(Z3)
    Z4 = H3 @ p["W4"].T + p["b4"]
    return Z4[:, :OUT], dict(X=X, Z1=Z1, H1=H1, Z2=Z2, H2=H2, Z3=Z3, H3=H3)


def loss(params, X, Y):
    out, _ = forward(params, X)
    mu, s = out[:, :3], out[:, 3:6]
    return float(np.mean(np.sum(0.5 * ((Y - mu) ** 2 * np.exp(-s) + s), axis=1)))


def grad(params, X, Y):
    """Analytic gradient of ``loss`` (backpropagation through the 4 layers)."""
    p = unpack(params)
    out, c = forward(params, X)
    B = X.shape[0]
    mu, s = out[:, :3], out[:, 3:6]
    r = Y - mu
    e = np.exp(-s)
    dZ4 = np.zeros((B, OUTP))
    dZ4[:, :3] = -r * e / B
    dZ4[:, 3:6] = 0.5 * (1.0 - r * r * e) / B
    g = {}
    g["W4"] = dZ4.T @ c["H3"]
    g["b4"] = dZ4.sum(axis=0)
    dH3 = dZ4 @ p["W4"]
    dZ3 = dH3 * gelu_grad(c["Z3"])
    g["W3"] = dZ3.T @ c["H2"]
    g["b3"] = dZ3.sum(axis=0)
    dH2 = dZ3 @ p["W3"]
    dZ2 = dH2 * gelu_grad(c["Z2"])
    g["W2"] = dZ2.T @ c["H1"]
    g["b2"] = dZ2.sum(axis=0)
    dH1 = dZ2 @ p["W2"]
    dZ1 = dH1 * gelu_grad(c["Z1"])
    g["W1"] = dZ1.T @ c["X"]
    g["b1"] = dZ1.sum(axis=0)
    g["W4"][OUT:] = 0.0
    g["b4"][OUT:] = 0.0
    return pack(g)


def adam_step(params, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
