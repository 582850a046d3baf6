"""Hypervolume of the approximation set (the scaffold's quality metric):
the library's exact slicing algorithm against the plain definition
(inclusion-exclusion over boxes) on small sets, and the 2-D staircase."""
import numpy as np
import pytest

from oracle.oracle import hypervolume_bruteforce
from paper_2202_11001_gb300 import dmr


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2202_11001_gb300.build import build_library

    build_library()


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_hv_matches_inclusion_exclusion(d):
    rng = np.random.default_rng(d)
    for trial in range(30):
        n = int(rng.integers(0, 9))
        pts = rng.uniform(0, 1, size=(n, d))
        if trial % 3 == 0 and n > 1:
            pts[1] = pts[0]  # duplicates
        if trial % 4 == 0 and n > 2:
            pts[2, 0] = pts[0, 0]  # ties in one coordinate
        ref = np.full(d, 1.05)
        ref[0] = 0.9  # some points outside the reference box
        got = dmr.hypervolume(pts, ref)
        want = hypervolume_bruteforce(pts, ref)
        assert abs(got - want) < 1e-12, (d, n, got, want)


def test_hv_2d_staircase_closed_form():
    """Points on an anti-diagonal: the union, counted column by column."""
    pts = np.array([[0.0, 3.0], [1.0, 2.0], [2.0, 1.0], [3.0, 0.0]])
    area = 0.0
    for k in range(4):  # column [k, k+1) is covered from min{y_i : x_i <= k} up to 4
        area += 4.0 - min(pts[i, 1] for i in range(4) if pts[i, 0] <= k)
    assert area == 10.0
    assert abs(dmr.hypervolume(pts, [4.0, 4.0]) - area) < 1e-12


def test_hv_dominated_points_add_nothing():
    rng = np.random.default_rng(9)
    base = rng.uniform(0, 0.5, size=(5, 3))
    worse = base + rng.uniform(0.01, 0.2, size=base.shape)
    ref = np.ones(3)
    assert abs(dmr.hypervolume(np.vstack([base, worse]), ref) - dmr.hypervolume(base, ref)) < 1e-12
