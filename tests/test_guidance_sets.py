"""Guidance in the paper's set form (Sec. 2.3.3): each point of a guidance set
contributes the smallest squared distance from its mapped position to the
points of the partner set, symmetrically, normalised by the total number of
points.

Oracle pins (CPU): one set per pair equals the point-pair form exactly;
identical meshes give the brute-force minimum distances; partial evaluation
equals a full evaluation of the trial state.  GPU: full, partial and plan
evaluation against the oracle with sets."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2202_11001_gb300 import synth


def _sets_problem(seed=31, C=4):
    pr = synth.sphere_pair(seed=seed, n=16, n_guide=8, C=C)
    # scramble partners inside two sets of four so that the set minimum differs
    g = pr["guide"].copy()
    g[:4, 1] = g[[2, 3, 0, 1], 1]
    g[4:, 1] = g[[5, 4, 7, 6], 1]
    pr["guide"] = g
    pr["sets"] = np.array([7, 7, 7, 7, 3, 3, 3, 3])
    return pr


def test_singleton_sets_equal_point_pairs():
    pr = synth.sphere_pair(seed=3, C=3)
    src, tgt = pr["img"]
    o1 = orc.Oracle(src, tgt, *pr["spacing"], pr["mesh"], guide=pr["guide"])
    o2 = orc.Oracle(src, tgt, *pr["spacing"], pr["mesh"], guide=pr["guide"], guide_sets=np.arange(5) * 3 + 1)
    assert np.array_equal(o1.eval_full(pr["coords"]), o2.eval_full(pr["coords"]))


def test_identical_meshes_give_minimum_distances():
    n, m = (12, 12, 12), (3, 3, 3)
    img = np.zeros((12, 12, 12))
    rng = np.random.default_rng(9)
    p = rng.uniform(0.5, 10.5, (6, 3))
    q = rng.uniform(0.5, 10.5, (6, 3))
    sets = np.array([0, 0, 0, 1, 1, 2])
    sp = (1.0, 1.5, 2.0)
    w = np.array(sp)
    o = orc.Oracle(img, img, sp, sp, m, guide=np.stack([p, q], axis=1), guide_sets=sets)
    r = synth.rest_lattice(n, m)
    obj = o.eval_full(np.stack([r, r])[None])
    tot = 0.0
    for i in range(6):
        mates = np.nonzero(sets == sets[i])[0]
        tot += min(np.sum(((p[i] - q[j]) * w) ** 2) for j in mates)
        tot += min(np.sum(((q[i] - p[j]) * w) ** 2) for j in mates)
    assert abs(obj[0, 2] - tot / 12.0) < 1e-12


def test_partial_equals_full_with_sets():
    pr = _sets_problem()
    src, tgt = pr["img"]
    o = orc.Oracle(src, tgt, *pr["spacing"], pr["mesh"], guide=pr["guide"], guide_sets=pr["sets"])
    o.eval_full(pr["coords"])
    groups = synth.single_point_fos(pr["mesh"])
    rng = np.random.default_rng(5)
    gids, cands = [4, 13, 22, 9], [0, 1, 2, 3]
    cur = np.stack([o.coords(c) for c in cands])
    tc = synth.trial_coords(cur, groups, gids, cands, 0.4, pr["mesh"], rng)
    obj = o.eval_partial(groups, gids, cands, tc)
    for k, (g, c) in enumerate(zip(gids, cands)):
        full = cur[k].copy()
        full[:, :, groups[g]] = tc[k][:, :, : len(groups[g])]
        o2 = orc.Oracle(src, tgt, *pr["spacing"], pr["mesh"], guide=pr["guide"], guide_sets=pr["sets"])
        assert np.allclose(obj[k], o2.eval_full(full[None])[0], rtol=1e-12, atol=1e-15)


@pytest.mark.gpu
def test_gpu_sets_full_partial_and_plan():
    from _harness import assert_obj_close
    from paper_2202_11001_gb300 import dmr

    C = 6
    pr = _sets_problem(seed=32, C=C)
    src, tgt = pr["img"]
    g = dmr.Problem(src, tgt, *pr["spacing"], pr["mesh"], guide=pr["guide"], guide_sets=pr["sets"], max_candidates=C)
    o = orc.Oracle(src.astype(np.float64), tgt.astype(np.float64), *pr["spacing"], pr["mesh"], guide=pr["guide"],
                   guide_sets=pr["sets"])
    assert_obj_close(g.eval_full(pr["coords"]), o.eval_full(pr["coords"]))
    groups = synth.single_point_fos(pr["mesh"])
    g.set_fos(groups)
    w = g.waves()[0]
    gids = np.tile(w, C).astype(np.int32)
    cids = np.repeat(np.arange(C), len(w)).astype(np.int32)
    tc = synth.trial_coords(pr["coords"], groups, gids, cids, 0.4, pr["mesh"], np.random.default_rng(6))
    assert_obj_close(g.eval_partial(gids, cids, tc), o.eval_partial(groups, gids, cids, tc), what="trial objectives")
    rng = np.random.default_rng(7)
    deltas = rng.normal(0, 0.3, size=(len(groups), C, 2, 3, 1))
    fix = synth.fixed_axes(pr["mesh"])
    for gi, grp in enumerate(groups):
        for ax in range(3):
            if (fix[grp[0]] >> ax) & 1:
                deltas[gi, :, :, ax, 0] = 0.0
    plan = g.plan_generation(np.arange(C, dtype=np.int32), deltas)
    plan.run()
    final = np.stack([g.coords(c) for c in range(C)])
    o2 = orc.Oracle(src.astype(np.float64), tgt.astype(np.float64), *pr["spacing"], pr["mesh"], guide=pr["guide"],
                    guide_sets=pr["sets"])
    assert_obj_close(g.objectives(), o2.eval_full(final))
