"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (autotuned tile, one CUDA-graph generation of partial evaluations with
accept-if-improves and commit), on sampled outputs the oracle computes one by
one: after the generation, the committed objectives and per-tet terms of
sampled candidates equal a fresh FP64 oracle evaluation of their final
coordinates (telescoping, Sec. 2.2): coverage and folds bit-exact, objectives
within 1e-5 relative.

Workloads: the 64^3 ellipsoid pair (population 128, 5^3 meshes), the
256x256x96 CT phantom (population 512, 10^3 meshes) and the 64-problem batch
(edge 32..128, meshes 4^3..9^3, populations 64..512)."""
import numpy as np
import pytest

from _harness import RTOL, assert_obj_close
from oracle import oracle as orc
from paper_2202_11001_gb300 import synth

pytestmark = pytest.mark.gpu


def _gpu_problem(pr, C):
    import torch

    from paper_2202_11001_gb300 import dmr

    g = dmr.Problem(pr["img"][0], pr["img"][1], *pr["spacing"], pr["mesh"], guide=pr["guide"], model=dmr.LINEAR,
                    storage="f32", max_candidates=C)
    g.eval_full(torch.from_numpy(pr["coords"]).cuda())
    groups = synth.single_point_fos(pr["mesh"])
    g.set_fos(groups)
    return g, groups


def _check_sampled(g, pr, sample):
    final = np.stack([g.coords(c) for c in sample])
    o = orc.Oracle(pr["img"][0].astype(np.float64), pr["img"][1].astype(np.float64), *pr["spacing"], pr["mesh"],
                   guide=pr["guide"], model=orc.LINEAR)
    want = o.eval_full(final)
    assert_obj_close(g.objectives()[sample], want, what="committed objectives")
    for j, c in enumerate(sample):
        tg, to = g.terms(c), o.terms(j)
        assert np.array_equal(tg["cov"], to["cov"]), ("coverage", c, np.argwhere(tg["cov"] != to["cov"])[:5].tolist())
        assert np.array_equal(tg["fold"], to["fold"])
        assert np.allclose(tg["ssd"], to["ssd"], rtol=RTOL, atol=1e-7)
        assert np.allclose(tg["def"], to["def"], rtol=RTOL, atol=1e-9)



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


def test_ellipsoid64_generation_full_size():
    import bench

    pr = bench.workload("ellipsoid64", 0)
    C = pr["coords"].shape[0]
    g, groups = _gpu_problem(pr, C)
    changed = _one_generation(g, groups, pr, C, 100)
    assert changed > C // 2
    _check_sampled(g, pr, [0, 41, 86, C - 1])
    g.close()


def test_ct256_generation_full_size():
    import bench

    pr = bench.workload("ct", 0)
    C = pr["coords"].shape[0]
    g, groups = _gpu_problem(pr, C)
    changed = _one_generation(g, groups, pr, C, 101)
    assert changed > C // 2
    _check_sampled(g, pr, [0, 255, C - 1])
    g.close()


def test_batch64_generation_full_size():
    import bench
    from paper_2202_11001_gb300 import dmr

    probs = synth.batch_problems(seed=2)
    gs, cands, dels = [], [], []
    for i, pr in enumerate(probs):
        C = pr["coords"].shape[0]
        pr["sigma"] = 0.1 * pr["img"][0].shape[0] / (pr["mesh"][0] - 1)
        g, groups = _gpu_problem(pr, C)
        gs.append(g)
        cands.append(np.arange(C, dtype=np.int32))
        dels.append(bench.deltas_for(pr, groups, C, np.random.default_rng(500 + i)))
    big = max(range(len(gs)), key=lambda i: probs[i]["coords"].shape[0] * gs[i].ntet)
    w, v, _ = gs[big].autotune()
    gs[0].set_tile(w, v)
    plan = dmr.Batch(gs).plan_generation(cands, dels)
    plan.run()
    plan.close()
    for q in (0, 21, 42, 63):
        C = probs[q]["coords"].shape[0]
        _check_sampled(gs[q], probs[q], [0, C - 1])
    for g in gs:
        g.close()
