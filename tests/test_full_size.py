"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times, for every image storage type (FP32, BF16, FP16), against the FP64
oracle fed the same (quantised) images:

* per trial: one wave of partial evaluations (Sec. 2.2) of sampled
  candidates through dmr_eval_partial -- every trial's objective vector
  within 1e-5 relative (fold counts exact), and for sampled trials the
  per-tet terms (coverage bit-exact, SSD and deformation within 1e-5);
* committed state: one CUDA-graph generation of partial evaluations with
  accept-if-improves and commit (autotuned tile), after which the committed
  objectives and per-tet terms of sampled candidates equal a fresh oracle
  evaluation of their final coordinates (telescoping).

Workloads: the 64^3 ellipsoid pair (population 128, 5^3 meshes), the
256x256x96 CT phantom (population 512, 10^3 meshes) and the 64-problem batch
(edge 32..128, meshes 4^3..9^3, populations 64..512; four problems sampled)."""
import numpy as np
import pytest

from _harness import RTOL, assert_obj_close, quantize
from oracle import oracle as orc
from paper_2202_11001_gb300 import synth

pytestmark = pytest.mark.gpu

STORAGES = ["f32", "bf16", "f16"]


def _gpu_problem(pr, C, storage):
    """The library problem on the quantised images, its FOS, and the FP64
    values of those images for the oracle."""
    import torch

    from paper_2202_11001_gb300 import dmr

    (bs, fs), (bt, ft) = quantize(pr["img"][0], storage), quantize(pr["img"][1], storage)
    g = dmr.Problem(bs, bt, *pr["spacing"], pr["mesh"], guide=pr["guide"], model=dmr.LINEAR, storage=storage,
                    img_dtype=storage, max_candidates=C)
    g.eval_full(torch.from_numpy(pr["coords"]).cuda())
    groups = synth.single_point_fos(pr["mesh"])
    g.set_fos(groups)
    return g, groups, (fs, ft)


def _oracle(pr, vals):
    return orc.Oracle(vals[0], vals[1], *pr["spacing"], pr["mesh"], guide=pr["guide"], model=orc.LINEAR)


def _check_terms(tg, to, what):
    assert np.array_equal(tg["cov"], to["cov"]), (what, "coverage", np.argwhere(tg["cov"] != to["cov"])[:5].tolist())
    assert np.array_equal(tg["fold"], to["fold"]), (what, "fold")
    assert np.allclose(tg["ssd"], to["ssd"], rtol=RTOL, atol=1e-7), what
    assert np.allclose(tg["def"], to["def"], rtol=RTOL, atol=1e-9), what


def _check_trials(g, groups, vals, pr, cands, seed, n_terms=6):
    """One wave of partial evaluations of candidates `cands` (their committed
    state) on the GPU and on the oracle: every trial's objectives, and the
    per-tet terms of n_terms trials spread over the wave."""
    cur = np.stack([g.coords(c) for c in cands])
    o = _oracle(pr, vals)
    o.eval_full(cur)
    wave = g.waves()[0]
    gids = np.repeat(wave, len(cands)).astype(np.int32)
    local = np.tile(np.arange(len(cands)), len(wave)).astype(np.int32)
    tc = synth.trial_coords(cur, groups, gids, local, pr["sigma"], pr["mesh"], np.random.default_rng(seed))
    got = g.eval_partial(gids, np.asarray(cands, np.int32)[local], tc)
    want = o.eval_partial(groups, gids, local, tc)
    assert_obj_close(got, want, what="trial objectives")
    for k in np.linspace(0, len(gids) - 1, n_terms).astype(int):
        tg, to = g.trial(int(k)), o.trial(int(k))
        assert np.array_equal(tg["tets"], to["tets"]), ("touched tets", k)
        _check_terms(tg, to, "trial %d" % k)
    return len(gids)


def _check_committed(g, pr, vals, sample):
    final = np.stack([g.coords(c) for c in sample])
    o = _oracle(pr, vals)
    want = o.eval_full(final)
    assert_obj_close(g.objectives()[sample], want, what="committed objectives")
    for j, c in enumerate(sample):
        _check_terms(g.terms(c), o.terms(j), "cand %d" % c)


def _one_generation(g, groups, pr, C, seed):
    import bench

    g.autotune()
    plan = g.plan_generation(np.arange(C, dtype=np.int32), bench.deltas_for(pr, groups, C, np.random.default_rng(seed)))
    before = g.objectives().copy()
    plan.run()
    plan.close()
    after = g.objectives()
    assert (after[:, 3] <= before[:, 3]).all()
    return int(np.sum(np.any(after != before, axis=1)))


@pytest.mark.parametrize("storage", STORAGES)
def test_ellipsoid64_full_size(storage):
    import bench

    pr = bench.workload("ellipsoid64", 0)
    C = pr["coords"].shape[0]
    g, groups, vals = _gpu_problem(pr, C, storage)
    assert _check_trials(g, groups, vals, pr, [0, 77, C - 1], 31) > 0
    changed = _one_generation(g, groups, pr, C, 100)
    assert changed > C // 2
    _check_committed(g, pr, vals, [0, 41, 86, C - 1])
    g.close()


@pytest.mark.parametrize("storage", STORAGES)
def test_ct256_full_size(storage):
    import bench

    pr = bench.workload("ct", 0)
    C = pr["coords"].shape[0]
    g, groups, vals = _gpu_problem(pr, C, storage)
    assert _check_trials(g, groups, vals, pr, [0, 300, C - 1], 32) > 0
    changed = _one_generation(g, groups, pr, C, 101)
    assert changed > C // 2
    _check_committed(g, pr, vals, [0, 255, C - 1])
    g.close()


@pytest.mark.parametrize("storage", STORAGES)
def test_batch64_full_size(storage):
    """The whole 64-problem batch in one plan, as bench.py builds and runs it;
    four problems spread over the batch sampled."""
    import bench
    from paper_2202_11001_gb300 import dmr

    probs, groups, dels = bench.batch_inputs(2)
    gs, vals, cands = [], [], []
    for pr in probs:
        C = pr["coords"].shape[0]
        g, _, v = _gpu_problem(pr, C, storage)
        gs.append(g)
        vals.append(v)
        cands.append(np.arange(C, dtype=np.int32))
    sample = (0, 21, 42, 63)
    for q in sample:
        C = probs[q]["coords"].shape[0]
        _check_trials(gs[q], groups[q], vals[q], probs[q], [0, C - 1], 40 + q, n_terms=3)
    bench.batch_tile(gs, probs, "")
    bt = dmr.Batch(gs)
    plan = bt.plan_generation(cands, dels)
    plan.run()
    plan.close()
    bt.close()
    for q in sample:
        C = probs[q]["coords"].shape[0]
        _check_committed(gs[q], probs[q], vals[q], [0, C // 2, C - 1])
    for g in gs:
        g.close()
