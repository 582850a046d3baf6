"""The learned-proposal network on the tensor cores (tcgen05) against the FP64
reference: forward on ragged row counts, backpropagated gradients, and
training progress.  BF16 weights and activations bound the agreement to
about 1e-2 relative."""
import numpy as np
import pytest

from oracle import mlp as ref
from paper_2202_11001_gb300 import dmr, synth

pytestmark = pytest.mark.gpu


def _bf16(a):
    import torch

    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("n", [1, 128, 300, 1000])
def test_forward_matches_reference(n):
    import torch

    net = dmr.MLP(seed=3)
    p = net.params().astype(np.float64)
    pb = ref.pack({k: (_bf16(v) if k.startswith("W") else v) for k, v in ref.unpack(p).items()})
    rng = np.random.default_rng(n)
    X = _bf16(rng.normal(0, 1, (n, ref.IN)))
    got = net.forward(torch.from_numpy(X).to(torch.bfloat16).cuda()).cpu().numpy()
    want, _ = ref.forward(pb, X)
    assert got.shape == (n, 6)
    assert _rel(got, want) < 2e-2


def test_gradients_match_reference():
    import torch

    net = dmr.MLP(seed=4)
    p = net.params().astype(np.float64)
    pb = ref.pack({k: (_bf16(v) if k.startswith("W") else v) for k, v in ref.unpack(p).items()})
    rng = np.random.default_rng(5)
    n = 384
    X = _bf16(rng.normal(0, 1, (n, ref.IN)))
    Y = rng.normal(0, 0.5, (n, 3))
    loss, g = net.train_step(torch.from_numpy(X).to(torch.bfloat16).cuda(), torch.from_numpy(Y).float().cuda(), 0.0,
                             want_grad=True)
    want = ref.grad(pb, X, Y)
    assert abs(loss - ref.loss(pb, X, Y)) < 2e-2 * abs(ref.loss(pb, X, Y)) + 1e-3
    gd, wd = ref.unpack(g.astype(np.float64)), ref.unpack(want)
    for k in wd:
        assert _rel(gd[k], wd[k]) < 5e-2, (k, _rel(gd[k], wd[k]))


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
