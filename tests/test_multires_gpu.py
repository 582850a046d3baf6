"""Grid multi-resolution run on the GPU (Sec. 2.4) on a small version of the
paper's cube problem: the finer level starts from refined approximation-set
members, which stay feasible; hypervolume never decreases within a level
(elitist archive)."""
import numpy as np
import pytest

from paper_2202_11001_gb300 import synth

pytestmark = pytest.mark.gpu


def test_multi_resolution_cube_small():
    from paper_2202_11001_gb300 import dmr, gomea

    pr = synth.cube_pair(seed=2, n=24, half=7.0, depth=3.0, r_src=4.0, r_tgt=2.5, n_guide=6, mesh=3, C=12)
    src, tgt = pr["img"]

    def build(mesh, C):
        return dmr.Problem(src, tgt, *pr["spacing"], mesh, guide=pr["guide"], model=dmr.LINEAR, max_candidates=C)

    p0 = build(pr["mesh"], 12)
    o0 = np.asarray(p0.eval_full(pr["coords"]))
    ref = 1.1 * np.max(o0[o0[:, 3] == 0, :3], axis=0)
    levels = [{"mesh": (3, 3, 3), "C": 12, "generations": 4, "sigma0": 0.8},
              {"mesh": (5, 5, 5), "C": 16, "generations": 3, "sigma0": 0.4}]
    res = gomea.multi_resolution(build, pr["coords"], levels, ref, np.random.default_rng(0))
    assert len(res) == 2
    assert res[1]["seeded_feasible"] == 1.0
    for r in res:
        hv = [h for _, h in r["curve"]]
        assert all(b >= a for a, b in zip(hv, hv[1:]))
        assert r["archive_size"] > 0
        r["gomea"].prob.close()
    fine = res[1]["gomea"]
    assert fine.coords.shape == (16, 2, 3, 125)
