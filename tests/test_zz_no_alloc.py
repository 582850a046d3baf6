"""The no-allocation single-candidate evaluation (dmr_eval_one_noalloc).

Some callers cannot allocate device memory at evaluation time: optimiser
loops that cannot afford the device synchronisation of cudaMalloc/cudaFree,
and processes whose device memory belongs to another allocator or a pool
sized up front.  They evaluate one candidate through this entry point, whose
scratch is a fixed device array inside the library.  The test calls it
through the C-ABI twice in a row, on different candidates, and checks each
result against dmr_eval_full and against the FP64 oracle with the tolerance
of the other parity tests; sizes beyond the fixed scratch and arguments the
binding would have to convert are rejected.  It lives in its own file,
collected last.
"""
import numpy as np
import pytest

from _harness import assert_obj_close
from oracle import oracle as orc
from paper_2202_11001_gb300 import dmr, synth

pytestmark = pytest.mark.gpu


def test_eval_one_noalloc_matches_eval_full_twice():
    import torch

    pr = synth.ellipsoid_pair(seed=3, C=3)
    src, tgt = pr["img"]
    g = dmr.Problem(src, tgt, *pr["spacing"], pr["mesh"], guide=pr["guide"], model=dmr.LINEAR,
                    max_candidates=3)
    ref = g.eval_full(pr["coords"])
    want = orc.Oracle(src, tgt, *pr["spacing"], pr["mesh"], guide=pr["guide"], model=orc.LINEAR).eval_full(
        pr["coords"])
    coords = torch.from_numpy(pr["coords"]).cuda()
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    for c in (2, 0):  # two calls in a row; the second reuses the shared scratch
        g.eval_one_noalloc(coords[c], out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()[None]
        assert_obj_close(got, ref[c][None], what="noalloc vs eval_full, cand %d" % c)
        assert_obj_close(got, np.asarray(want)[c][None], what="noalloc vs oracle, cand %d" % c)
    # sizes beyond the fixed scratch are rejected with a clear error
    big = synth.sphere_pair(seed=0, n=24, mesh=12, C=1)  # 11^3 cubes = 7986 tets
    gb = dmr.Problem(big["img"][0], big["img"][1], *big["spacing"], big["mesh"], max_candidates=1)
    cb = torch.from_numpy(big["coords"][0]).cuda()
    with pytest.raises(dmr.DmrError, match="limit"):
        gb.eval_one_noalloc(cb, out)
    # arguments the binding would have to convert (an allocation) are refused
    with pytest.raises(dmr.DmrError, match="float64"):
        g.eval_one_noalloc(coords[0].float(), out)
    with pytest.raises(dmr.DmrError, match="needs"):
        g.eval_one_noalloc(coords[0], out[:2])
    with pytest.raises(dmr.DmrError, match="float64"):
        g.eval_one_noalloc(coords[0].cpu(), out)
