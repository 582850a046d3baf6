"""The learned-proposal network on the tensor cores (tcgen05) against the FP64
reference, element by element.

The reference runs in its BF16-operand mode: every matrix-product operand
(weights, hidden activations, back-propagated errors) rounded to BF16 as the
BF16 x BF16 tensor-core product takes it, products and sums exact.  What is
left between the two is the kernel's FP32 accumulation and its hardware tanh
(relative error about 2^-11) inside GELU; where that moves a value across a
BF16 rounding boundary, the rounded operand changes by one BF16 unit.  Each
entry y = sum_k a_k b_k is therefore checked as

    |y_gpu - y_ref| <= 1e-2 |y_ref| + 2^-8 S,   S = sum_k |a_k| |b_k|,

1e-2 relative (the bound asked of the BF16 backward) plus one BF16 unit of
the entry's magnitude sum, the scale at which a changed operand acts (the
same S gives the usual dot-product rounding bound).  For the outputs S is
formed from the last layer's weights and activations plus the bias, for a
weight gradient from |dZ|^T |input| over the rows, for a bias gradient from
the column sum of |dZ|."""
import numpy as np
import pytest

from oracle import mlp as ref
from paper_2202_11001_gb300 import dmr, synth

pytestmark = pytest.mark.gpu

RTOL = 1e-2
ATOL_UNITS = 2.0 ** -8


def _bf16(a):
    import torch

    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _check(name, got, want, mag):
    got, want, mag = (np.asarray(v, np.float64) for v in (got, want, mag))
    assert got.shape == want.shape, (name, got.shape, want.shape)
    err = np.abs(got - want)
    bound = RTOL * np.abs(want) + ATOL_UNITS * mag
    bad = np.flatnonzero(err > bound)
    worst = float(np.max(err / np.maximum(bound, 1e-300)))
    assert bad.size == 0, "%s: %d of %d entries outside the bound (worst at %.3g of it; first %s: got %r want %r)" % (
        name, bad.size, err.size, worst, np.unravel_index(bad[0], err.shape), got.flat[bad[0]], want.flat[bad[0]])
    return worst


def _output_magnitude(pb, X):
    """S of each output entry: sum_j |W4_ij| |H3_j| + |b4_i|."""
    _, c = ref.forward(pb, X, bf16_operands=True)
    p = ref.unpack(pb)
    return (np.abs(c["H3"]) @ np.abs(c["W"][3]).T + np.abs(p["b4"]))[:, :ref.OUT]


@pytest.mark.parametrize("n", [1, 127, 300, 1000, 4096])
def test_forward_matches_reference(n):
    import torch

    net = dmr.MLP(seed=3)
    p = net.params().astype(np.float64)
    rng = np.random.default_rng(n)
    X = _bf16(rng.normal(0, 1, (n, ref.IN)))
    got = net.forward(torch.from_numpy(X).to(torch.bfloat16).cuda()).cpu().numpy()
    want, _ = ref.forward(p, X, bf16_operands=True)
    assert got.shape == (n, 6)
    _check("outputs (n=%d)" % n, got, want, _output_magnitude(p, X))


@pytest.mark.parametrize("n", [1, 300, 4096])
def test_gradients_match_reference(n):
    import torch

    net = dmr.MLP(seed=4)
    p = net.params().astype(np.float64)
    rng = np.random.default_rng(5 + n)
    X = _bf16(rng.normal(0, 1, (n, ref.IN)))
    Y = rng.normal(0, 0.5, (n, 3))
    loss, g = net.train_step(torch.from_numpy(X).to(torch.bfloat16).cuda(), torch.from_numpy(Y).float().cuda(), 0.0,
                             want_grad=True)
    want_loss = ref.loss(p, X, Y, bf16_operands=True)
    assert abs(loss - want_loss) <= RTOL * abs(want_loss), (loss, want_loss)
    want, mag = ref.grad(p, X, Y, bf16_operands=True, magnitudes=True)
    gd, wd, md = ref.unpack(g.astype(np.float64)), ref.unpack(want), ref.unpack(mag)
    for k in wd:
        _check("%s (n=%d)" % (k, n), gd[k], wd[k], md[k])


def test_training_reduces_loss():
    import torch

    net = dmr.MLP(seed=6)
    rng = np.random.default_rng(7)
    n = 2048
    X = rng.normal(0, 1, (n, ref.IN)).astype(np.float32)
    w = rng.normal(0, 0.1, (ref.IN, 3))
    Y = (X @ w).astype(np.float32)
    Xd = torch.from_numpy(X).to(torch.bfloat16).cuda()
    Yd = torch.from_numpy(Y).cuda()
    first = net.train_step(Xd, Yd, 1e-3)
    for _ in range(150):
        last = net.train_step(Xd, Yd, 1e-3)
    assert last < first - 0.3, (first, last)


def test_adam_step_matches_reference():
    """One Adam step on the GPU against the reference update applied to the
    GPU's own gradient (FP32 parameters and moments; 1e-5 relative)."""
    import torch

    net = dmr.MLP(seed=9)
    p0 = net.params().astype(np.float64)
    rng = np.random.default_rng(10)
    n = 512
    X = _bf16(rng.normal(0, 1, (n, ref.IN)))
    Y = rng.normal(0, 0.5, (n, 3))
    Xd = torch.from_numpy(X).to(torch.bfloat16).cuda()
    Yd = torch.from_numpy(Y).float().cuda()
    _, g = net.train_step(Xd, Yd, 0.0, want_grad=True)
    net.train_step(Xd, Yd, 1e-3)
    p1 = net.params().astype(np.float64)
    want, _, _ = ref.adam_step(p0, g.astype(np.float64), np.zeros_like(p0), np.zeros_like(p0), 1, 1e-3)
    d = ref.unpack(np.arange(ref.N_PARAMS))
    pad = np.concatenate([d["W4"][ref.OUT:].ravel(), d["b4"][ref.OUT:]]).astype(np.int64)
    live = np.setdiff1d(np.arange(ref.N_PARAMS), pad)
    assert np.all(p1[pad] == 0.0)
    assert np.allclose(p1[live], want[live], rtol=1e-5, atol=1e-7)


def test_features_match_scipy_patches():
    import torch
    from scipy import ndimage

    pr = synth.sphere_pair(seed=8, C=2)
    g = dmr.Problem(pr["img"][0], pr["img"][1], *pr["spacing"], pr["mesh"], max_candidates=2)
    X = dmr.MLP.features(g, torch.from_numpy(pr["coords"]).cuda()).float().cpu().numpy()
    P = g.P
    for row in (0, 5, P + 13):
        c, p = divmod(row, P)
        want = []
        for mesh in range(2):
            pt = pr["coords"][c, mesh, :, p]
            img = pr["img"][mesh].astype(np.float64)
            for dz in range(-2, 3):
                for dy in range(-2, 3):
                    for dx in range(-2, 3):
                        q = pt + np.array([dx, dy, dz])
                        want.append(ndimage.map_coordinates(img, [[q[2]], [q[1]], [q[0]]], order=1, mode="nearest")[0])
        want = np.array(want)
        assert np.allclose(X[row, :250], want, atol=1e-2, rtol=1e-2)


def test_forward_rejects_unaligned_input():
    """The input is read by TMA, whose base address must be 16-byte aligned:
    a view starting 2 bytes into a buffer is refused on the host (no launch)."""
    import torch

    m = dmr.MLP(seed=3)
    flat = torch.zeros(1 + 4 * 256, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(dmr.DmrError):
        m.forward(flat[1:].view(4, 256))
    ok = m.forward(flat[:4 * 256].view(4, 256))  # the aligned view still runs
    assert tuple(ok.shape) == (4, 6)
    m.close()
