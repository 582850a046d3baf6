"""GPU-vs-oracle parity through the C-ABI (Sec. 2.2, 2.3).

Per-tet voxel coverage and fold counts match bit-exactly; objective values
match the FP64 oracle within 1e-5 relative, with the oracle fed the same
(quantised) images.  Sizes span several tiles and ragged tails.
"""
import numpy as np
import pytest

from _harness import RTOL, assert_obj_close, assert_terms_match, make_pair
from oracle import oracle as orc
from paper_2202_11001_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("model", [orc.SPRING, orc.LINEAR])
def test_full_sphere16(model):
    pr = synth.sphere_pair(seed=0)
    g, o = make_pair(pr, model=model)
    og = g.eval_full(pr["coords"])
    oo = o.eval_full(pr["coords"])
    assert_obj_close(og, oo)
    for c in range(pr["coords"].shape[0]):
        assert_terms_match(g, o, c)
        lg, tg = g.landmarks(c)
        lo, to = o.landmarks(c)
        assert np.array_equal(lg, lo)
        assert np.allclose(tg, to, rtol=RTOL, atol=1e-12)


def test_regular_mesh_ties_bit_exact():
    """Unjittered lattice: many voxel centres lie exactly on faces, so every
    such voxel goes through the exact FP64 tie rule."""
    pr = synth.sphere_pair(seed=1, C=2, amp=0.0)
    g, o = make_pair(pr)
    assert_obj_close(g.eval_full(pr["coords"]), o.eval_full(pr["coords"]))
    for c in range(2):
        assert_terms_match(g, o, c)
        assert g.terms(c)["cov"].sum(axis=0).tolist() == [16 ** 3, 16 ** 3]


def test_partial_all_groups_sphere16():
    """All 27 single-point groups x 10 candidates: trial objectives, trial
    coverage, then commit of random accepts and a fresh full evaluation."""
    pr = synth.sphere_pair(seed=2)
    g, o = make_pair(pr)
    C = pr["coords"].shape[0]
    g.eval_full(pr["coords"])
    o.eval_full(pr["coords"])
    groups = synth.single_point_fos(pr["mesh"])
    g.set_fos(groups)
    rng = np.random.default_rng(3)
    for w in g.waves():
        gids = np.repeat(w, C).astype(np.int32)
        cids = np.tile(np.arange(C), len(w)).astype(np.int32)
        cur = np.stack([o.coords(c) for c in range(C)])
        tc = synth.trial_coords(cur, groups, gids, cids, 0.4, pr["mesh"], rng)
        pg = g.eval_partial(gids, cids, tc)
        po = o.eval_partial(groups, gids, cids, tc)
        assert_obj_close(pg, po, what="trial objectives")
        for k in range(0, len(gids), 7):
            tg, to = g.trial(k), o.trial(k)
            assert np.array_equal(tg["tets"], to["tets"])
            assert np.array_equal(tg["cov"], to["cov"])
            assert np.array_equal(tg["fold"], to["fold"])
            assert np.allclose(tg["ssd"], to["ssd"], rtol=RTOL, atol=1e-7)
        acc = (rng.uniform(size=len(gids)) < 0.5).astype(np.uint8)
        g.commit(acc)
        o.commit(acc)
    assert_obj_close(g.objectives(), o.objectives())
    for c in range(C):
        assert np.array_equal(g.coords(c), o.coords(c))
        assert_terms_match(g, o, c)
        lg, _ = g.landmarks(c)
        lo, _ = o.landmarks(c)
        assert np.array_equal(lg, lo)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_reduced_precision_storage(storage):
    pr = synth.sphere_pair(seed=4, C=6)
    g, o = make_pair(pr, storage=storage)
    assert_obj_close(g.eval_full(pr["coords"]), o.eval_full(pr["coords"]))
    for c in range(6):
        assert_terms_match(g, o, c)


def test_ellipsoid64_full_and_partial_black_rule():
    """64^3 ellipsoids on an exactly-black background (black rule active at
    every boundary), 5^3 meshes: full evaluation and one wave of partial
    evaluations on 8 candidates."""
    pr = synth.ellipsoid_pair(seed=1, C=8)
    g, o = make_pair(pr, model=orc.LINEAR)
    assert_obj_close(g.eval_full(pr["coords"]), o.eval_full(pr["coords"]))
    for c in range(8):
        assert_terms_match(g, o, c)
    groups = synth.single_point_fos(pr["mesh"])
    g.set_fos(groups)
    rng = np.random.default_rng(5)
    w = g.waves()[0]
    gids = np.repeat(w, 8).astype(np.int32)
    cids = np.tile(np.arange(8), len(w)).astype(np.int32)
    tc = synth.trial_coords(pr["coords"], groups, gids, cids, 1.5, pr["mesh"], rng)
    assert_obj_close(g.eval_partial(gids, cids, tc), o.eval_partial(groups, gids, cids, tc), what="trial objectives")


def test_ellipsoid64_black_rule_off():
    """The same ellipsoids with the black rule off: tets whose partner region
    is all background (every reachable partner voxel 0) contribute the own
    image's squares; per-tet terms and objectives against the oracle."""
    pr = synth.ellipsoid_pair(seed=2, C=4)
    g, o = make_pair(pr, model=orc.LINEAR, black=False)
    assert_obj_close(g.eval_full(pr["coords"]), o.eval_full(pr["coords"]))
    for c in range(4):
        assert_terms_match(g, o, c)


@pytest.mark.parametrize("which", ["both", "source", "target"])
@pytest.mark.parametrize("black", [True, False])
def test_zero_images_empty_space_paths(which, black):
    """Images that are all 0 on one or both sides: every item takes an
    empty-space path (partner region all 0, with or without the own box all 0)
    or its complement; coverage exact, objectives against the oracle, then one
    wave of partial evaluations."""
    pr = synth.sphere_pair(seed=7, C=4)
    src, tgt = pr["img"]
    if which in ("both", "source"):
        src = np.zeros_like(src)
    if which in ("both", "target"):
        tgt = np.zeros_like(tgt)
    pr = dict(pr, img=(src, tgt))
    g, o = make_pair(pr, black=black)
    assert_obj_close(g.eval_full(pr["coords"]), o.eval_full(pr["coords"]))
    for c in range(4):
        assert_terms_match(g, o, c)
    groups = synth.single_point_fos(pr["mesh"])
    g.set_fos(groups)
    w = g.waves()[0]
    gids = np.repeat(w, 4).astype(np.int32)
    cids = np.tile(np.arange(4), len(w)).astype(np.int32)
    tc = synth.trial_coords(pr["coords"], groups, gids, cids, 0.4, pr["mesh"], np.random.default_rng(9))
    assert_obj_close(g.eval_partial(gids, cids, tc), o.eval_partial(groups, gids, cids, tc), what="trial objectives")


def test_plan_generation_matches_sequential_and_oracle():
    """The CUDA-graph generation plan (propose, partial evaluation,
    accept-if-improves, commit for every wave) equals the same steps through
    eval_partial + commit_improving, and its committed state equals a fresh
    oracle evaluation of the final coordinates (telescoping, Sec. 2.2)."""
    pr = synth.sphere_pair(seed=6, C=6)
    C = 6
    g1, o = make_pair(pr)
    g2, _ = make_pair(pr)
    for g in (g1, g2):
        g.eval_full(pr["coords"])
    groups = synth.single_point_fos(pr["mesh"])
    g1.set_fos(groups)
    g2.set_fos(groups)
    waves = g1.waves()
    rng = np.random.default_rng(7)
    deltas = rng.normal(0, 0.3, size=(len(groups), C, 2, 3, 1))
    fix = synth.fixed_axes(pr["mesh"])
    for gi, grp in enumerate(groups):
        for ax in range(3):
            if (fix[grp[0]] >> ax) & 1:
                deltas[gi, :, :, ax, 0] = 0.0
    plan = g1.plan_generation(np.arange(C, dtype=np.int32), deltas)
    n_acc = 0
    for _ in range(2):
        plan.run()
        for w in waves:
            cids = np.repeat(np.arange(C), len(w)).astype(np.int32)
            gids = np.tile(w, C).astype(np.int32)
            cur = np.stack([g2.coords(c) for c in range(C)])
            tc = np.stack([cur[c][:, :, groups[gg]] + deltas[gg, c] for gg, c in zip(gids, cids)])
            g2.eval_partial(gids, cids, tc)
            n_acc += int(g2.commit_improving().sum())
    assert n_acc > 0
    assert np.array_equal(g1.objectives(), g2.objectives())
    final = np.stack([g1.coords(c) for c in range(C)])
    for c in range(C):
        assert np.array_equal(final[c], g2.coords(c))
    fresh = o.eval_full(final)
    assert_obj_close(g1.objectives(), fresh)
    for c in range(C):
        assert_terms_match(g1, o, c)


def test_folds_nan_and_border_violations():
    pr = synth.sphere_pair(seed=8, C=4)
    c = pr["coords"].copy()
    ctr = 1 + 3 * (1 + 3 * 1)
    c[0, 1, :, ctr] += np.array([9.0, 8.0, 7.5])   # fold the target mesh
    c[1, 0, 0, 1 + 3 * 0] += 0.25                   # border point off its plane (y=0 face keeps y)
    c[1, 0, 1, 1 + 3 * 0] += 0.25
    c[2, 0, 2, ctr] = np.nan                        # non-finite coordinate
    g, o = make_pair(pr)
    og, oo = g.eval_full(c), o.eval_full(c)
    assert_obj_close(og, oo)
    assert og[0, 3] > 0 and og[1, 3] > 0 and og[2, 3] > 0 and og[3, 3] == 0
    for k in range(4):
        assert_terms_match(g, o, k)


def test_tile_shapes_same_result_and_autotune():
    """Every tile shape (warps per CTA x voxels per warp iteration) gives
    bit-identical results; the autotuner picks one of them."""
    pr = synth.ellipsoid_pair(seed=9, C=3)
    g, o = make_pair(pr)
    ref = g.eval_full(pr["coords"])
    assert_obj_close(ref, o.eval_full(pr["coords"]))
    for w in (4, 8, 16):
        for v in (32, 64, 128):
            g.set_tile(w, v)
            out = g.eval_full(pr["coords"])
            assert np.array_equal(out, ref), (w, v)
    bw, bv, table = g.autotune()
    assert (bw, bv) in table and all(t > 0 for t in table.values())
    assert g.tile() == (bw, bv)
    assert np.array_equal(g.eval_full(pr["coords"]), ref)


def _deltas(pr, groups, C, sigma, seed):
    rng = np.random.default_rng(seed)
    d = rng.normal(0, sigma, size=(len(groups), C, 2, 3, 1))
    fix = synth.fixed_axes(pr["mesh"])
    for gi, grp in enumerate(groups):
        for ax in range(3):
            if (fix[grp[0]] >> ax) & 1:
                d[gi, :, :, ax, 0] = 0.0
    return d


def test_batched_problems_equal_single_plans_and_oracle():
    """Batching (uneven images, meshes and populations in one launch per
    kernel and wave) gives exactly the single-problem results."""
    from paper_2202_11001_gb300 import dmr

    specs = [synth.sphere_pair(seed=20, C=5), synth.ellipsoid_pair(seed=21, n=24, mesh=4, C=7, n_guide=4),
             synth.sphere_pair(seed=22, n=20, mesh=5, C=3), synth.ellipsoid_pair(seed=23, n=32, mesh=3, C=4, n_guide=0)]
    for pr in specs:
        if pr["guide"] is not None and len(pr["guide"]) == 0:
            pr["guide"] = None
    single, batched, oracles, plans_in = [], [], [], []
    for i, pr in enumerate(specs):
        C = pr["coords"].shape[0]
        gs, o = make_pair(pr)
        gb, _ = make_pair(pr)
        groups = synth.single_point_fos(pr["mesh"])
        for g in (gs, gb):
            g.eval_full(pr["coords"])
            g.set_fos(groups)
        d = _deltas(pr, groups, C, 0.3 if pr["mesh"][0] <= 3 else 0.8, 30 + i)
        single.append((gs, gs.plan_generation(np.arange(C, dtype=np.int32), d)))
        batched.append(gb)
        plans_in.append((np.arange(C, dtype=np.int32), d))
        oracles.append(o)
    bt = dmr.Batch(batched)
    plan = bt.plan_generation([c for c, _ in plans_in], [d for _, d in plans_in])
    for _ in range(2):
        plan.run()
        for g, pl in single:
            pl.run()
    for (gs, _), gb, o, pr in zip(single, batched, oracles, specs):
        assert np.array_equal(gs.objectives(), gb.objectives())
        C = pr["coords"].shape[0]
        final = np.stack([gb.coords(c) for c in range(C)])
        for c in range(C):
            assert np.array_equal(final[c], gs.coords(c))
        assert_obj_close(gb.objectives(), o.eval_full(final))


def test_plan_update_equals_new_plan():
    """dmr_plan_update: a plan fed new proposal offsets (host or device) runs
    exactly like a plan built with them."""
    import torch

    pr = synth.sphere_pair(seed=40, C=5)
    C = 5
    g1, _ = make_pair(pr)
    g2, _ = make_pair(pr)
    groups = synth.single_point_fos(pr["mesh"])
    for g in (g1, g2):
        g.eval_full(pr["coords"])
        g.set_fos(groups)
    d0 = _deltas(pr, groups, C, 0.3, 41)
    d1 = _deltas(pr, groups, C, 0.3, 42)
    d2 = _deltas(pr, groups, C, 0.3, 43)
    p1 = g1.plan_generation(np.arange(C, dtype=np.int32), d0)
    p2 = g2.plan_generation(np.arange(C, dtype=np.int32), d1)
    p1.update(d1)
    p1.run()
    p2.run()
    assert np.array_equal(g1.objectives(), g2.objectives())
    p1.update(torch.from_numpy(d2).cuda())
    p3 = g2.plan_generation(np.arange(C, dtype=np.int32), d2)
    p1.run()
    p3.run()
    assert np.array_equal(g1.objectives(), g2.objectives())
    for c in range(C):
        assert np.array_equal(g1.coords(c), g2.coords(c))
