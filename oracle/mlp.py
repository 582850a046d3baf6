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

Precision.  The network is specified with BF16 weights and FP32 accumulation.
A BF16 x BF16 tensor-core product takes both operands in BF16, so with
``bf16_operands=True`` every matrix-product operand is rounded to BF16 (8
significant bits, round to nearest, ties to even) before an exact FP64
product: the weights, each hidden activation H_l, and in the backward pass
each back-propagated error dZ_l where it enters a product (dW_l = dZ_l^T in,
dH_{l-1} = dZ_l W_l).  Biases, pre-activations, GELU, the loss and the bias
gradients (column sums of dZ_l) stay unrounded.  With the default
``bf16_operands=False`` everything is plain FP64.

Test infrastructure only: the CUDA library never imports this module.
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


def round_bf16(x):
    """Round to the nearest BF16 value (8 significant bits, ties to even),
    from the definition: x = m 2^e with 0.5 <= |m| < 1, keep m to 2^-8."""
    x = np.asarray(x, np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0), e - 8)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(_C * (z + _A * z ** 3)))


def gelu_grad(z):
    t = np.tanh(_C * (z + _A * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * _C * (1.0 + 3.0 * _A * z * z)


def forward(params, X, bf16_operands=False):
    p = unpack(params)
    q = round_bf16 if bf16_operands else (lambda a: a)
    X = q(np.asarray(X, np.float64))
    W = [q(p["W1"]), q(p["W2"]), q(p["W3"]), q(p["W4"])]
    Z1 = X @ W[0].T + p["b1"]
    H1 = q(gelu(Z1))
    Z2 = H1 @ W[1].T + p["b2"]
    H2 = q(gelu(Z2))
    Z3 = H2 @ W[2].T + p["b3"]
    H3 = q(gelu(Z3))
    Z4 = H3 @ W[3].T + p["b4"]
    return Z4[:, :OUT], dict(X=X, Z1=Z1, H1=H1, Z2=Z2, H2=H2, Z3=Z3, H3=H3, W=W)


def loss(params, X, Y, bf16_operands=False):
    out, _ = forward(params, X, bf16_operands)
    mu, s = out[:, :3], out[:, 3:6]
    return float(np.mean(np.sum(0.5 * ((Y - mu) ** 2 * np.exp(-s) + s), axis=1)))


def grad(params, X, Y, bf16_operands=False, magnitudes=False):
    """Analytic gradient of ``loss`` (backpropagation through the 4 layers).

    With ``magnitudes=True`` also returns, in the same flat layout, the sum of
    absolute products that forms each entry (sum over rows of |dZ| |input| for
    a weight, of |dZ| for a bias): the scale at which operand rounding in the
    product acts on that entry."""
    q = round_bf16 if bf16_operands else (lambda a: a)
    out, c = forward(params, X, bf16_operands)
    W = c["W"]
    B = X.shape[0]
    mu, s = out[:, :3], out[:, 3:6]
    r = Y - mu
    e = np.exp(-s)
    dZ4 = np.zeros((B, OUTP))
    dZ4[:, :3] = -r * e / B
    dZ4[:, 3:6] = 0.5 * (1.0 - r * r * e) / B
    g, mag = {}, {}
    ins = {1: c["X"], 2: c["H1"], 3: c["H2"], 4: c["H3"]}
    zs = {1: c["Z1"], 2: c["Z2"], 3: c["Z3"]}
    dZ = dZ4
    for layer in (4, 3, 2, 1):
        dZq = q(dZ)
        g["W%d" % layer] = dZq.T @ ins[layer]
        g["b%d" % layer] = dZ.sum(axis=0)
        mag["W%d" % layer] = np.abs(dZq).T @ np.abs(ins[layer])
        mag["b%d" % layer] = np.abs(dZ).sum(axis=0)
        if layer > 1:
            dH = dZq @ W[layer - 1]
            dZ = dH * gelu_grad(zs[layer - 1])
    for d in (g, mag):
        d["W4"][OUT:] = 0.0
        d["b4"][OUT:] = 0.0
    return (pack(g), pack(mag)) if magnitudes else pack(g)


def adam_step(params, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
