"""Grid refinement of the multi-resolution scheme (Sec. 2.4): edge, face and
cube midpoints, m -> 2m - 1 points per axis.

Oracle pins (CPU): the rest lattice refines to the finer rest lattice
exactly; coarse points are kept bit-exactly; refinement commutes with affine
maps; a face point is the mean of its 4 corners and a cube point the mean of
its 8; the paper's 6^3 -> 11^3 parameter counts; refining feasible jittered
meshes keeps every tet positive and border coordinates on their planes
(c_fold = 0 on the finer problem).  GPU: bit-exact against the oracle."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2202_11001_gb300 import synth


def _idx(m, a, b, c):
    return a + m[0] * (b + m[1] * c)


def test_rest_lattice_refines_to_finer_rest_lattice():
    n, m = (16, 16, 8), (5, 5, 3)
    M = tuple(2 * a - 1 for a in m)
    coarse = np.broadcast_to(synth.rest_lattice(n, m), (1, 2, 3, np.prod(m))).copy()
    fine = orc.refine(coarse, m)
    want = synth.rest_lattice(n, M)
    assert np.array_equal(fine[0, 0], want) and np.array_equal(fine[0, 1], want)


def test_paper_parameter_counts():
    m = (6, 6, 6)
    coarse = np.zeros((1, 2, 3, 216))
    fine = orc.refine(coarse, m)
    assert coarse[0].size == 1296 and fine[0].size == 7986  # Sec. 2.5: 1296 and 7986 parameters


def test_coarse_points_kept_and_midpoints_are_means():
    rng = np.random.default_rng(3)
    m = (4, 3, 5)
    M = tuple(2 * a - 1 for a in m)
    coarse = rng.normal(size=(2, 2, 3, np.prod(m)))
    fine = orc.refine(coarse, m)
    for c in range(m[2]):
        for b in range(m[1]):
            for a in range(m[0]):
                assert np.array_equal(fine[..., _idx(M, 2 * a, 2 * b, 2 * c)], coarse[..., _idx(m, a, b, c)])
    # an edge point, a face point and a cube centre against numpy means
    e = fine[..., _idx(M, 3, 2, 4)]
    assert np.allclose(e, 0.5 * (coarse[..., _idx(m, 1, 1, 2)] + coarse[..., _idx(m, 2, 1, 2)]), rtol=0, atol=1e-15)
    f = fine[..., _idx(M, 1, 2, 3)]
    want = np.mean([coarse[..., _idx(m, a, 1, c)] for a in (0, 1) for c in (1, 2)], axis=0)
    assert np.allclose(f, want, rtol=0, atol=4e-16 * 4)
    k = fine[..., _idx(M, 5, 3, 7)]
    want = np.mean([coarse[..., _idx(m, a, b, c)] for a in (2, 3) for b in (1, 2) for c in (3, 4)], axis=0)
    assert np.allclose(k, want, rtol=0, atol=1e-14)


def test_refinement_commutes_with_affine_maps():
    rng = np.random.default_rng(4)
    m = (4, 4, 4)
    coarse = rng.normal(size=(3, 2, 3, 64)) * 5
    A = rng.normal(size=(3, 3))
    t = rng.normal(size=3)
    lhs = orc.refine(np.einsum("ij,cmjp->cmip", A, coarse) + t[None, None, :, None], m)
    rhs = np.einsum("ij,cmjp->cmip", A, orc.refine(coarse, m)) + t[None, None, :, None]
    assert np.allclose(lhs, rhs, rtol=0, atol=1e-12)


def test_refined_feasible_meshes_stay_feasible():
    pr = synth.sphere_pair(seed=3, C=6)
    m = pr["mesh"]
    M = tuple(2 * a - 1 for a in m)
    src, tgt = pr["img"]
    oc = orc.Oracle(src.astype(np.float64), tgt.astype(np.float64), *pr["spacing"], m, guide=pr["guide"])
    assert (oc.eval_full(pr["coords"])[:, 3] == 0).all()
    fine = orc.refine(pr["coords"], m)
    of = orc.Oracle(src.astype(np.float64), tgt.astype(np.float64), *pr["spacing"], M, guide=pr["guide"])
    obj = of.eval_full(fine)
    assert (obj[:, 3] == 0).all(), obj[:, 3]
    fix = synth.fixed_axes(M)
    for ax in range(3):
        free = ((fix >> ax) & 1) == 0
        assert np.array_equal(fine[:, :, ax, ~free], np.broadcast_to(synth.rest_lattice(src.shape[::-1], M)[ax, ~free],
                                                                      fine[:, :, ax, ~free].shape))


@pytest.mark.gpu
def test_gpu_refinement_bit_exact():
    import torch

    from paper_2202_11001_gb300 import dmr

    rng = np.random.default_rng(5)
    for m, C in (((3, 3, 3), 4), ((6, 6, 6), 33), ((5, 4, 7), 9)):
        coarse = rng.normal(size=(C, 2, 3, int(np.prod(m)))) * 10
        want = orc.refine(coarse, m)
        assert np.array_equal(dmr.refine(coarse, m), want)
        got = dmr.refine(torch.from_numpy(coarse).cuda(), m).cpu().numpy()
        assert np.array_equal(got, want)
