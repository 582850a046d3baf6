"""Small and degenerate configurations through the C-ABI against the FP64
oracle (Sec. 2.2, 2.3): a single lattice cube (2 x 2 x 2 points, 6 tets) on
tiny images of unequal, non-cubic sizes with anisotropic spacing; a
non-cubic mesh (2 x 3 x 5 points); a population of one candidate.  Full
evaluation (objectives, per-tet coverage bit-exact) and every single-point
group partially re-evaluated (trial objectives); then the host-side
refusals of empty and out-of-range trial lists."""
import numpy as np
import pytest

from _harness import assert_obj_close, assert_terms_match, make_pair
from paper_2202_11001_gb300 import synth

pytestmark = pytest.mark.gpu

CONFIGS = {
    # name: (source dims (nx, ny, nz), target dims, mesh points, population)
    "one_cube": ((5, 4, 3), (6, 5, 4), (2, 2, 2), 3),
    "noncubic_mesh": ((9, 7, 11), (8, 8, 10), (2, 3, 5), 4),
    "one_candidate": ((6, 6, 6), (6, 6, 6), (3, 3, 3), 1),
}


def _tiny(seed, dims_s, dims_t, m, C):
    rng = np.random.default_rng(seed)

    def img(d):
        a = rng.uniform(0.1, 1.0, size=(d[2], d[1], d[0])).astype(np.float32)
        a[rng.uniform(size=a.shape) < 0.3] = 0.0  # black voxels for the black-vs-grey rule
        return a

    src, tgt = img(dims_s), img(dims_t)
    coords = synth.population(dims_s, dims_t, m, C, 0.4, rng)
    gs = rng.uniform(0.0, 1.0, (3, 3)) * (np.array(dims_s) - 1)
    gt = rng.uniform(0.0, 1.0, (3, 3)) * (np.array(dims_t) - 1)
    return dict(img=(src, tgt), spacing=((1.0, 1.5, 2.0), (1.2, 1.0, 0.8)), mesh=m,
                guide=np.stack([gs, gt], axis=1), coords=coords), rng


@pytest.mark.parametrize("name", sorted(CONFIGS))
def test_small_configurations_full_and_partial(name):
    dims_s, dims_t, m, C = CONFIGS[name]
    pr, rng = _tiny(11, dims_s, dims_t, m, C)
    g, o = make_pair(pr)
    assert_obj_close(g.eval_full(pr["coords"]), o.eval_full(pr["coords"]), what=name + " full")
    for c in range(C):
        assert_terms_match(g, o, c)
    groups = synth.single_point_fos(m)
    g.set_fos(groups)
    for w in g.waves():
        gids = np.repeat(w, C).astype(np.int32)
        cids = np.tile(np.arange(C), len(w)).astype(np.int32)
        cur = np.stack([o.coords(c) for c in range(C)])
        tc = synth.trial_coords(cur, groups, gids, cids, 0.3, m, rng)
        assert_obj_close(g.eval_partial(gids, cids, tc), o.eval_partial(groups, gids, cids, tc),
                         what=name + " partial")
    g.close()


def test_trial_lists_refused_on_the_host():
    from paper_2202_11001_gb300 import dmr

    pr, rng = _tiny(12, *CONFIGS["one_cube"])
    g, _ = make_pair(pr)
    g.eval_full(pr["coords"])
    groups = synth.single_point_fos(pr["mesh"])
    g.set_fos(groups)
    C = pr["coords"].shape[0]
    cur = pr["coords"]
    ok_g, ok_c = np.array([0], np.int32), np.array([0], np.int32)
    tc = synth.trial_coords(cur, groups, ok_g, ok_c, 0.3, pr["mesh"], rng)
    with pytest.raises(dmr.DmrError):
        g.eval_partial(np.zeros(0, np.int32), np.zeros(0, np.int32), tc[:0])
    with pytest.raises(dmr.DmrError):
        g.eval_partial(ok_g, np.array([C], np.int32), tc)
    with pytest.raises(dmr.DmrError):
        g.eval_partial(np.array([len(groups)], np.int32), ok_c, tc)
    # the problem is still usable afterwards
    assert np.isfinite(g.eval_partial(ok_g, ok_c, tc)).all()
    g.close()
