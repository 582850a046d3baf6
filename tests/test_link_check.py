"""The paper's folding check (Sec. 2.3.4): a point lying outside its link
(the faces of its star's tets that do not contain it), by ray-crossing
parity; border points in 2-D in their plane, border-edge points in 1-D.

Oracle pins (CPU): rest and mildly jittered meshes have no violation; a
single moved interior point is inside its link exactly when its generalised
winding number (sum of signed solid angles, Van Oosterom & Strackee) is
non-zero; border-face and border-edge points leaving their polygon or
interval are caught; every violation comes with a non-positive signed volume
(the stronger check c_fold uses).  GPU: counts equal the oracle's."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2202_11001_gb300 import synth


def _problem(n=20, m=(4, 4, 4)):
    img = np.zeros((n, n, n))
    o = orc.Oracle(img, img, (1, 1, 1), (1, 1, 1), m)
    r = synth.rest_lattice((n, n, n), m)
    return o, np.stack([r, r])


def _solid_angle_winding(p, tris):
    tot = 0.0
    for a, b, c in tris:
        A, B, C = a - p, b - p, c - p
        la, lb, lc = np.linalg.norm(A), np.linalg.norm(B), np.linalg.norm(C)
        num = np.dot(A, np.cross(B, C))
        den = la * lb * lc + np.dot(A, B) * lc + np.dot(A, C) * lb + np.dot(B, C) * la
        tot += 2.0 * np.arctan2(num, den)
    return tot / (4 * np.pi)


def test_rest_and_jittered_meshes_have_no_violation():
    o, c = _problem()
    assert list(o.link_violations(c)) == [0, 0]
    pr = synth.sphere_pair(seed=5, n=16, mesh=5, C=6)
    src, tgt = pr["img"]
    o2 = orc.Oracle(src, tgt, *pr["spacing"], pr["mesh"])
    for cc in pr["coords"]:
        assert list(o2.link_violations(cc)) == [0, 0]


def test_interior_point_matches_winding_number():
    o, c0 = _problem()
    m = (4, 4, 4)
    tets = orc.build_tets(m)
    v = 1 + 4 * (1 + 4 * 2)  # interior point (1, 1, 2)
    star = [t for t in range(len(tets)) if v in tets[t]]
    # link triangles ordered so that (v, a, b, c) is positively oriented at
    # rest: the signed solid angles then add up to +-1 inside, 0 outside
    links = []
    for t in star:
        a, b, cc = [w for w in tets[t] if w != v]
        P = c0[0]
        if np.linalg.det(np.stack([P[:, a] - P[:, v], P[:, b] - P[:, v], P[:, cc] - P[:, v]])) < 0:
            b, cc = cc, b
        links.append((a, b, cc))
    rng = np.random.default_rng(3)
    seen = {0: 0, 1: 0}
    for _ in range(200):
        c = c0.copy()
        c[0, :, v] += rng.normal(0, 4.0, 3)
        tris = [np.array([c[0][:, w] for w in tri]) for tri in links]
        wn = _solid_angle_winding(c[0][:, v], tris)
        inside = abs(wn) > 0.5
        got = o.link_point(c, 0, v)
        assert got == (0 if inside else 1), (wn, got)
        if got:
            assert o.link_violations(c)[0] >= 1
        seen[got] += 1
    assert seen[0] > 20 and seen[1] > 20  # both outcomes exercised


def test_border_face_and_edge_points():
    o, c0 = _problem()
    v_face = 0 + 4 * (1 + 4 * 2)  # x = border, y = 1, z = 2: moves in its x plane
    c = c0.copy()
    c[1, 1, v_face] += 2.0  # inside its in-plane polygon (neighbours 6.67 apart)
    assert list(o.link_violations(c)) == [0, 0]
    c[1, 1, v_face] += 6.0  # past its y-neighbour (which then leaves its own polygon too)
    viol = o.link_violations(c)
    assert viol[0] == 0 and o.link_point(c, 1, v_face) == 1
    v_edge = 1 + 4 * (0 + 4 * 0)  # y, z borders; free along x
    c = c0.copy()
    c[0, 0, v_edge] += 5.0  # still between x-neighbours (6.67 apart)
    assert list(o.link_violations(c)) == [0, 0]
    c[0, 0, v_edge] += 3.0
    viol = o.link_violations(c)
    assert o.link_point(c, 0, v_edge) == 1 and viol[1] == 0


def test_violation_implies_non_positive_volume():
    o, c0 = _problem()
    rng = np.random.default_rng(4)
    for _ in range(100):
        c = c0 + np.where(synth.fixed_axes((4, 4, 4))[None, None, :] >> np.arange(3)[None, :, None] & 1, 0.0,
                          rng.normal(0, 3.0, c0.shape))
        viol = o.link_violations(c)
        if viol.sum():
            assert o.eval_full(c[None])[0, 3] > 0


@pytest.mark.gpu
def test_gpu_link_counts_equal_oracle():
    from paper_2202_11001_gb300 import dmr

    n, m, C = 20, (4, 5, 4), 24
    img = np.zeros((n, n, n), np.float32)
    r = synth.rest_lattice((n, n, n), m)
    rng = np.random.default_rng(8)
    fix = synth.fixed_axes(m)
    free = ~((fix[None, :] >> np.arange(3)[:, None]) & 1).astype(bool)
    coords = np.stack([np.stack([r, r])] * C)
    for k in range(C):
        coords[k] += np.where(free[None], rng.normal(0, 0.5 + 0.25 * k, (2, 3, r.shape[1])), 0.0)
    g = dmr.Problem(img, img, (1, 1, 1), (1, 1, 1), m, max_candidates=C)
    g.eval_full(coords)
    o = orc.Oracle(img.astype(np.float64), img.astype(np.float64), (1, 1, 1), (1, 1, 1), m)
    got = g.link_check()
    want = np.stack([o.link_violations(coords[k]) for k in range(C)])
    assert np.array_equal(got, want)
    assert want.sum() > 0 and (want == 0).any()
