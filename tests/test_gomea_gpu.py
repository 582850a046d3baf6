"""The minimal MO-GOMEA scaffold over the GPU evaluator: the archive stays
feasible and mutually non-dominated, its hypervolume never decreases, the
evaluation budget follows the partial-evaluation convention, and the
committed objectives equal a fresh oracle evaluation (Sec. 2.2, 2.4)."""
import numpy as np
import pytest

from _harness import assert_obj_close, make_pair
from paper_2202_11001_gb300 import gomea, synth

pytestmark = pytest.mark.gpu


def test_gomea_generations_archive_and_budget():
    pr = synth.sphere_pair(seed=40, C=8)
    g, o = make_pair(pr)
    groups = synth.single_point_fos(pr["mesh"])
    opt = gomea.Gomea(g, pr["coords"], groups, pr["mesh"], 0.4, np.random.default_rng(1))
    ref = 1.1 * np.max(opt.obj[:, :3], axis=0)
    hv = opt.run(4, ref)
    vals = [h for _, h in hv]
    assert all(b >= a - 1e-15 for a, b in zip(vals, vals[1:]))
    assert vals[-1] > 0
    A = opt.archive.objs
    assert gomea.nondominated(A).all()
    # budget: full evaluation of C candidates + 4 generations of all groups
    star = opt.touched
    assert abs(opt.evals - (8 + 4 * 8 * star.sum() / g.ntet)) < 1e-9
    assert abs(star.sum() - 4 * g.ntet) < 1e-9  # every tet has 4 vertices
    assert_obj_close(g.objectives(), o.eval_full(opt.coords))
