"""Shared helpers of the GPU parity tests: build the same problem on the CUDA
library and on the FP64 oracle from one seeded synthetic workload."""
import numpy as np

from oracle import oracle as orc
from paper_2202_11001_gb300 import synth

RTOL = 1e-5  # objective tolerance vs the FP64 oracle (values), Sec. 2.3


def quantize(img, storage):
    """Round an FP32 image to the storage type on the host (round to nearest
    even, as torch does); returns (bits for the library, FP64 values for the
    oracle)."""
    import torch

    t = torch.from_numpy(np.ascontiguousarray(img, np.float32))
    if storage == "f32":
        return np.ascontiguousarray(img, np.float32), img.astype(np.float64)
    dt = torch.bfloat16 if storage == "bf16" else torch.float16
    q = t.to(dt)
    return q.view(torch.int16).numpy().view(np.uint16).copy(), q.to(torch.float64).numpy()


def make_pair(pr, storage="f32", model=orc.SPRING, black=True, lam=1.0, mu=1.0, guide=True, cap=None):
    from paper_2202_11001_gb300 import dmr

    src, tgt = pr["img"]
    (bs, fs), (bt, ft) = quantize(src, storage), quantize(tgt, storage)
    spS, spT = pr["spacing"]
    gd = pr["guide"] if guide else None
    cap = cap or pr["coords"].shape[0]
    g = dmr.Problem(bs, bt, spS, spT, pr["mesh"], guide=gd, black_rule=black, model=model, lam=lam, mu=mu,
                    storage=storage, img_dtype=storage, max_candidates=cap)
    o = orc.Oracle(fs, ft, spS, spT, pr["mesh"], guide=gd, black_rule=black, model=model, lam=lam, mu=mu)
    return g, o


def assert_obj_close(got, want, rtol=RTOL, what="objectives"):
    got = np.asarray(got)
    want = np.asarray(want)
    assert got.shape == want.shape
    # c_fold is an integer count: exact
    assert np.array_equal(got[..., 3], want[..., 3]), (what, got[..., 3], want[..., 3])
    assert np.array_equal(np.isnan(got), np.isnan(want)), (what, "NaN pattern differs", got, want)
    got = np.where(np.isnan(got), 0.0, got)
    want = np.where(np.isnan(want), 0.0, want)
    for j in range(3):
        err = np.abs(got[..., j] - want[..., j])
        tol = rtol * np.maximum(np.abs(want[..., j]), 1e-300) + 1e-300
        bad = err > tol
        assert not bad.any(), "%s[%d]: max rel err %.3e at %s (got %r want %r)" % (
            what, j, float(np.max(err / np.maximum(np.abs(want[..., j]), 1e-300))), np.argwhere(bad)[:3].tolist(),
            got[..., j][bad][:3], want[..., j][bad][:3])


def assert_terms_match(g, o, c, rtol=RTOL):
    tg, to = g.terms(c), o.terms(c)
    assert np.array_equal(tg["cov"], to["cov"]), "coverage mismatch cand %d: %s" % (
        c, np.argwhere(tg["cov"] != to["cov"])[:5].tolist())
    assert np.array_equal(tg["fold"], to["fold"])
    assert np.allclose(tg["ssd"], to["ssd"], rtol=rtol, atol=1e-7)
    assert np.allclose(tg["def"], to["def"], rtol=rtol, atol=1e-9, equal_nan=True)
