"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: counts the
paper prints, closed forms of homogeneous deformations, a library routine
(scipy's linear interpolation, numpy's determinant and linear solve),
brute-force enumeration, and invariants of the decomposition (Sec. 2.2,
2.3).  A dropped term, a wrong sign, a transposed operand or a wrong index in
the oracle fails at least one of them.
"""
import itertools
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2202_11001_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _regular(n, m):
    r = synth.rest_lattice(n, m)
    return np.stack([r, r])  # [2, 3, P]


def _mk(img_s, img_t, m, guide=None, black=True, model=orc.SPRING, lam=1.0, mu=1.0, sp=(1, 1, 1)):
    return orc.Oracle(img_s, img_t, sp, sp, m, guide=guide, black_rule=black, model=model, lam=lam, mu=mu)


def _tet_vertices(coords1, tets, mesh, t):
    return coords1[mesh][:, tets[t]].T  # [4, 3]


# ----------------------------------------------------------------- topology
def test_paper_counts_golden():
    """Sec. 2.5: 6^3 / 11^3 grids -> 1296 / 7986 parameters; Sec. 2.1: 6 tets
    per cube.  Values read from tests/golden/paper_counts.txt."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_counts.txt")) if l.strip() and l[0] != "#"]
    for pts, cubes, params in rows:
        pts, cubes, params = int(pts), int(cubes), int(params)
        m = (pts, pts, pts)
        assert pts ** 3 * 3 * 2 == params
        tets = orc.build_tets(m)
        assert len(tets) == 6 * cubes ** 3
        assert len(np.unique(tets)) == pts ** 3


@pytest.mark.parametrize("m,nt", [((3, 3, 3), 48), ((5, 5, 5), 384), ((10, 10, 10), 4374), ((4, 6, 5), 360)])
def test_tet_counts_and_conformity(m, nt):
    tets = orc.build_tets(m)
    assert tets.shape == (nt, 4)
    # every face is shared by at most 2 tets; faces used once lie on the box
    faces = {}
    for t, v in enumerate(tets):
        for f in range(4):
            key = tuple(sorted(int(x) for i, x in enumerate(v) if i != f))
            faces.setdefault(key, []).append(t)
    assert max(len(x) for x in faces.values()) == 2
    P = int(np.prod(m))
    idx = np.stack(np.unravel_index(np.arange(P), (m[2], m[1], m[0]))[::-1], axis=1)  # (a,b,c)
    for key, ts in faces.items():
        if len(ts) == 1:
            pts = idx[list(key)]
            on = [(np.all(pts[:, ax] == 0) or np.all(pts[:, ax] == m[ax] - 1)) for ax in range(3)]
            assert any(on), "interior face used by one tet only"
    # rest volumes: each tet is 1/6 of a cube and orientation is positive
    r = synth.rest_lattice((2 * (m[0] - 1), 2 * (m[1] - 1), 2 * (m[2] - 1)), m)
    for v in tets[:: max(1, nt // 97)]:
        X = r[:, v].T
        d = np.linalg.det(np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]]))
        assert d > 0
        assert abs(d / 6.0 - 8.0 / 6.0) < 1e-12


def test_star_sizes_mirrored():
    """Mirrored 2x2x2 groups (Fig. 1B): interior vertices whose lattice
    coordinates are all even or all odd are the diagonal end of all 8 cubes
    around them (48 tets); every other interior vertex has 16."""
    m = (7, 6, 5)
    img = np.zeros((4, 4, 4))
    o = _mk(img, img, m)
    ptr, idx = o.star()
    sizes = np.diff(ptr)
    assert sizes.sum() == 4 * o.ntet
    for c in range(1, m[2] - 1):
        for b in range(1, m[1] - 1):
            for a in range(1, m[0] - 1):
                p = a + m[0] * (b + m[1] * c)
                par = {a & 1, b & 1, c & 1}
                assert sizes[p] == (48 if len(par) == 1 else 16)
    tets = o.tets()
    for p in range(o.P):
        for t in idx[ptr[p]:ptr[p + 1]]:
            assert p in tets[t]


def test_face_sign_is_inward():
    """The per-face sign is combinatorial; the two tets sharing a face get
    opposite signs, and the opposite vertex lies on the positive side."""
    m = (4, 4, 4)
    img = np.zeros((6, 6, 6))
    o = _mk(img, img, m)
    tets, fp = o.tets(), o.face_perm()
    r = synth.rest_lattice((6, 6, 6), m)
    seen = {}
    for t in range(o.ntet):
        X = r[:, tets[t]].T
        for f in range(4):
            ia, ib, ic, s = fp[t, f]
            key = tuple(sorted(tets[t][[ia, ib, ic]]))
            assert list(key) == list(tets[t][[ia, ib, ic]])
            n = np.cross(X[ib] - X[ia], X[ic] - X[ia])
            assert s * np.dot(n, X[f] - X[ia]) > 0
            seen.setdefault(key, []).append(int(s))
    for key, ss in seen.items():
        if len(ss) == 2:
            assert ss[0] == -ss[1]


# ------------------------------------------------------- inside / coverage
def _bary(X, p):
    A = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
    l123 = np.linalg.solve(A, p - X[0])
    return np.concatenate([[1 - l123.sum()], l123])


@pytest.mark.parametrize("jit", [0.0, 0.45])
def test_coverage_partition_bruteforce(jit):
    """Every voxel centre belongs to exactly one tet (tie rule, Sec. 2.3.1
    footnote read in 3-D); the bbox-clipped count equals brute force over
    the whole image; clear-cut voxels agree with numpy barycentrics."""
    n = (9, 8, 7)
    m = (4, 3, 3)
    rng = np.random.default_rng(5)
    img = np.zeros(n[::-1])
    o = _mk(img, img, m)
    c1 = _regular(n, m)
    if jit:
        c1[0] = synth.jitter(c1[0], m, jit, rng)
        c1[1] = synth.jitter(c1[1], m, jit, rng)
    tets = o.tets()
    for mesh in range(2):
        total = np.zeros(n[::-1], np.int32)
        for t in range(o.ntet):
            mask = o.coverage_mask(mesh, c1, t)
            total += mask
            tt = o.tet_terms(c1, t)
            assert tt["cov"][mesh] == int(mask.sum())
            X = _tet_vertices(c1, tets, mesh, t)
            zz, yy, xx = np.nonzero(np.ones(n[::-1]))
            for z, y, x in list(zip(zz, yy, xx))[:: 7]:
                lam = _bary(X, np.array([x, y, z], float))
                if lam.min() > 1e-9:
                    assert mask[z, y, x] == 1
                elif lam.min() < -1e-9:
                    assert mask[z, y, x] == 0
        assert total.min() == 1 and total.max() == 1


def test_tie_rule_equals_symbolic_perturbation():
    """On a regular lattice many voxel centres lie exactly on faces.  The tie
    rule must give the tet that contains p + (e^3, e^2, e) for small e."""
    n = (8, 8, 8)
    m = (3, 3, 3)
    img = np.zeros(n)
    o = _mk(img, img, m)
    c1 = _regular(n, m)
    tets = o.tets()
    masks = np.stack([o.coverage_mask(0, c1, t) for t in range(o.ntet)])
    eps = 1e-3
    d = np.array([eps ** 3, eps ** 2, eps])
    checked = 0
    for z, y, x in itertools.product(range(8), repeat=3):
        p = np.array([x, y, z], float)
        owners = np.nonzero(masks[:, z, y, x])[0]
        assert len(owners) == 1
        lams = [_bary(_tet_vertices(c1, tets, 0, t), p) for t in range(o.ntet)]
        on_face = sum(1 for l in lams if l.min() > -1e-12) > 1
        if not on_face:
            continue
        pp = p + d
        inside = [t for t in range(o.ntet) if _bary(_tet_vertices(c1, tets, 0, t), pp).min() > 0]
        assert inside == [owners[0]]
        checked += 1
    assert checked > 50


def test_star_invariance():
    """Moving one interior point inside its star (no fold) keeps the star's
    total coverage (the star region does not change)."""
    n = (16, 16, 16)
    m = (3, 3, 3)
    img = np.zeros(n)
    o = _mk(img, img, m)
    c1 = _regular(n, m)
    ptr, idx = o.star()
    p = 1 + 3 * (1 + 3 * 1)
    star = idx[ptr[p]:ptr[p + 1]]
    base = sum(o.tet_terms(c1, t)["cov"][0] for t in star)
    rng = np.random.default_rng(1)
    for _ in range(5):
        c2 = c1.copy()
        c2[0, :, p] += rng.uniform(-2.5, 2.5, 3)
        assert all(o.six_vol(0, c2, t) > 0 for t in star)
        assert sum(o.tet_terms(c2, t)["cov"][0] for t in star) == base


# ------------------------------------------------------------ map / sample
def test_map_matches_linear_solve():
    n = (12, 12, 12)
    m = (3, 3, 3)
    img = np.zeros(n)
    o = _mk(img, img, m)
    rng = np.random.default_rng(2)
    c1 = _regular(n, m)
    c1[0] = synth.jitter(c1[0], m, 1.0, rng)
    c1[1] = synth.jitter(c1[1], m, 1.0, rng)
    tets = o.tets()
    for t in range(0, o.ntet, 5):
        for d in range(2):
            own = _tet_vertices(c1, tets, d, t)
            par = _tet_vertices(c1, tets, 1 - d, t)
            v = own.mean(axis=0) + rng.uniform(-0.5, 0.5, 3)
            lam = _bary(own, v)
            want = lam @ par
            got = o.map_point(d, c1, t, v)
            assert np.allclose(got, want, atol=1e-11)
            assert abs(o.six_vol(d, c1, t) - np.linalg.det(np.stack([own[1] - own[0], own[2] - own[0], own[3] - own[0]]))) < 1e-10


def test_trilinear_matches_scipy():
    from scipy import ndimage

    rng = np.random.default_rng(3)
    n = (7, 6, 5)
    img = rng.uniform(0, 1, n[::-1])
    o = _mk(img, img, (2, 2, 2))
    for _ in range(300):
        p = rng.uniform(-2.0, np.array(n) + 1.0)
        s, _ = o.sample(0, p)
        want = ndimage.map_coordinates(img, [[p[2]], [p[1]], [p[0]]], order=1, mode="nearest")[0]
        assert abs(s - want) < 1e-12


def test_black_support_rule():
    img = np.zeros((4, 4, 4))
    img[1, 1, 2] = 0.5  # voxel (x=2, y=1, z=1)
    o = _mk(img, img, (2, 2, 2))
    assert o.sample(0, np.array([1.0, 1.0, 1.0]))[1] is True  # weight only on (1,1,1)
    assert o.sample(0, np.array([1.5, 1.0, 1.0]))[1] is False  # (2,1,1) in support
    assert o.sample(0, np.array([1.0 + 1e-9, 1.0, 1.0]))[1] is False
    assert o.sample(0, np.array([3.0, 3.0, 3.0]))[1] is True


# ------------------------------------------------------------ objectives
def test_identical_meshes_and_images_give_zero():
    """P1/P3: identical meshes -> zero deformation (both models); identical
    images and meshes -> zero dissimilarity even with the black rule on."""
    pr = synth.sphere_pair(seed=7)
    src = pr["img"][0].astype(np.float64)
    src[src < 0.02] = 0.0  # make a black region so the rule is exercised
    for model in (orc.SPRING, orc.LINEAR):
        o = _mk(src, src, pr["mesh"], guide=None, model=model)
        c = pr["coords"][:3].copy()
        c[:, 1] = c[:, 0]
        obj = o.eval_full(c)
        assert np.all(obj[:, 0] == 0.0)
        assert np.all(obj[:, 1] == 0.0)
        assert np.all(obj[:, 3] == 0.0)


def test_rigid_motion_spring_zero():
    n = (20, 20, 20)
    m = (3, 3, 3)
    img = np.zeros(n)
    o = _mk(img, img, m)
    rng = np.random.default_rng(4)
    c1 = _regular(n, m)
    c1[0] = synth.jitter(c1[0], m, 1.5, rng)
    ang = 0.3
    R = np.array([[np.cos(ang), -np.sin(ang), 0], [np.sin(ang), np.cos(ang), 0], [0, 0, 1]])
    c1[1] = R @ c1[0] + np.array([[1.25], [-0.5], [0.75]])
    e = sum(o.tet_terms(c1, t)["def"] for t in range(o.ntet))
    assert e < 1e-18


def test_uniform_scaling_spring_closed_form():
    """Cubic lattice with cell h scaled by s: per Kuhn tet the 6 edges give
    3h^2 + 2(2h^2) + 3h^2 = 10h^2 and the 4 spokes 40/9 h^2, so
    f_def = (s-1)^2 (130/9) h^2 / 10."""
    h, m = 4.0, (4, 4, 4)
    n = (12, 12, 12)
    img = np.zeros(n)
    o = _mk(img, img, m)
    c1 = _regular(n, m)
    s = 1.15
    ctr = np.array([[5.5], [5.5], [5.5]])
    c1[1] = ctr + s * (c1[0] - ctr)
    obj = o.eval_full(c1[None])
    assert abs(obj[0, 1] - (s - 1) ** 2 * (130.0 / 9.0) * h * h / 10.0) < 1e-12


@pytest.mark.parametrize("lam,mu", [(1.0, 1.0), (0.7, 1.3)])
def test_linear_elastic_homogeneous(lam, mu):
    """P11: a homogeneous affine target (x -> A x + b) gives every tet the same
    energy density psi(A) = mu eps:eps + lam/2 tr(eps)^2, eps = sym(A) - I;
    with A = diag(1+d,1,1) this is (mu + lam/2) d^2."""
    m = (3, 3, 3)
    n = (10, 10, 10)
    img = np.zeros(n)
    o = _mk(img, img, m, model=orc.LINEAR, lam=lam, mu=mu)
    rng = np.random.default_rng(6)
    c1 = _regular(n, m)
    c1[0] = synth.jitter(c1[0], m, 0.8, rng)
    for A in (np.diag([1.07, 1.0, 1.0]), np.array([[1.05, 0.08, -0.02], [0.01, 0.97, 0.05], [0.03, -0.04, 1.02]])):
        c2 = c1.copy()
        c2[1] = A @ c1[0] + np.array([[0.3], [-0.2], [0.1]])
        eps = 0.5 * (A + A.T) - np.eye(3)
        psi = mu * np.sum(eps * eps) + 0.5 * lam * np.trace(eps) ** 2
        obj = o.eval_full(c2[None])
        assert abs(obj[0, 1] - psi) < 1e-12 * max(1.0, psi)
    d = 0.07
    assert abs((mu + lam / 2) * d * d - (mu * d * d + 0.5 * lam * d * d)) < 1e-15


def test_affine_warp_recovered():
    """P4: target mesh = A * source mesh + b; every voxel maps to A v + b; with
    a linear-ramp target image and the source image equal to the warped ramp
    plus kappa, forward SSD is kappa^2 per voxel (trilinear is exact on
    linear fields away from the clamp)."""
    n = (14, 13, 12)
    m = (3, 3, 3)
    A = np.array([[0.86, 0.05, 0.02], [-0.03, 0.9, 0.04], [0.01, -0.02, 0.88]])
    ctr = (np.array(n) - 1) / 2.0
    b = ctr - A @ ctr
    for corner in itertools.product(*[(0, k - 1) for k in n]):
        q = A @ np.array(corner, float) + b
        assert np.all(q >= 0) and np.all(q <= np.array(n) - 1)
    g = np.array([0.031, -0.017, 0.023])
    zz, yy, xx = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    P = np.stack([xx, yy, zz], axis=-1).astype(float)
    ramp_t = 0.4 + P @ g
    kappa = 0.125
    ramp_s = 0.4 + (P @ A.T + b) @ g + kappa
    o = _mk(ramp_s, ramp_t, m, black=False)
    c1 = _regular(n, m)
    c1[1] = A @ c1[0] + b[:, None]
    tets = o.tets()
    fwd, cov = 0.0, 0
    for t in range(o.ntet):
        tt = o.tet_terms(c1, t)
        fwd += tt["ssd"][0]
        cov += tt["cov"][0]
        v = _tet_vertices(c1, tets, 0, t).mean(axis=0)
        assert np.allclose(o.map_point(0, c1, t, v), A @ v + b, atol=1e-12)
    assert cov == np.prod(n)
    assert abs(fwd - kappa * kappa * cov) < 1e-9
    # the same warp with kappa = 0 is recovered exactly (dissimilarity ~ 0)
    o2 = _mk(ramp_s - kappa, ramp_t, m, black=False)
    f0 = sum(o2.tet_terms(c1, t)["ssd"][0] for t in range(o2.ntet))
    assert f0 < 1e-20


def test_black_rule_closed_form():
    """P9: all-zero source vs constant c>0 target: every voxel pair is a
    black/grey mismatch, so f_sim = 1; without the rule f_sim = c^2."""
    n = (9, 9, 9)
    m = (3, 3, 3)
    zero = np.zeros(n)
    c = 0.37
    const = np.full(n, c)
    c1 = _regular(n, m)[None]
    assert _mk(zero, const, m, black=True).eval_full(c1)[0, 0] == 1.0
    assert abs(_mk(zero, const, m, black=False).eval_full(c1)[0, 0] - c * c) < 1e-15


def test_guidance_closed_forms():
    """P10: identity meshes carry every landmark unchanged; an affine target
    mesh carries p to A p + b (and q back through the inverse)."""
    n = (12, 12, 12)
    m = (3, 3, 3)
    img = np.zeros(n)
    rng = np.random.default_rng(8)
    p = rng.uniform(0.5, 10.5, (6, 3))
    q = p + rng.normal(0, 1.0, (6, 3))
    q = np.clip(q, 0.2, 10.8)
    guide = np.stack([p, q], axis=1)
    sp = (1.0, 1.5, 2.0)
    o = orc.Oracle(img, img, sp, sp, m, guide=guide)
    c1 = _regular(n, m)
    obj = o.eval_full(c1[None])
    w = np.array(sp)
    want = np.mean(np.sum(((p - q) * w) ** 2, axis=1))
    assert abs(obj[0, 2] - want) < 1e-12
    A = np.array([[0.95, 0.03, 0.0], [0.02, 1.0, -0.04], [0.0, 0.01, 0.97]])
    ctr = np.full(3, 5.5)
    b = ctr - A @ ctr
    c2 = c1.copy()
    c2[1] = A @ c1[0] + b[:, None]
    obj = o.eval_full(c2[None])
    fw = np.sum(((p @ A.T + b - q) * w) ** 2, axis=1)
    Ai = np.linalg.inv(A)
    bw = np.sum((((q - b) @ Ai.T - p) * w) ** 2, axis=1)
    assert abs(obj[0, 2] - (fw.sum() + bw.sum()) / 12.0) < 1e-10


def test_fold_and_border_counts():
    n = (12, 12, 12)
    m = (3, 3, 3)
    img = np.zeros(n)
    o = _mk(img, img, m)
    c1 = _regular(n, m)
    assert o.eval_full(c1[None])[0, 3] == 0
    ptr, idx = o.star()
    # a border point (a=0, b=1, c=1) leaves its plane: every tet of its star
    # counts it once
    p = 0 + 3 * (1 + 3 * 1)
    c2 = c1.copy()
    c2[0, 0, p] += 0.25
    assert o.eval_full(c2[None])[0, 3] == ptr[p + 1] - ptr[p]
    # the centre point pushed far through its star folds some tets
    pc = 1 + 3 * (1 + 3 * 1)
    c3 = c1.copy()
    c3[1, :, pc] += np.array([9.0, 8.0, 7.5])
    folded = sum(1 for t in idx[ptr[pc]:ptr[pc + 1]] if o.six_vol(1, c3, t) <= 0)
    assert folded > 0
    assert o.eval_full(c3[None])[0, 3] >= folded
    c4 = c1.copy()
    c4[0, 1, pc] = np.nan
    assert o.eval_full(c4[None])[0, 3] >= 1


# ------------------------------------------------------------ partial eval
def _small_problem(seed=11, model=orc.SPRING):
    pr = synth.sphere_pair(seed=seed, C=4)
    o = orc.Oracle(pr["img"][0], pr["img"][1], *pr["spacing"], pr["mesh"], guide=pr["guide"], model=model)
    return pr, o


@pytest.mark.parametrize("model", [orc.SPRING, orc.LINEAR])
def test_telescoping(model):
    """Sec. 2.2 + 2.3 decomposability: applying accepted partial changes one
    group at a time keeps the objectives equal to a fresh full evaluation."""
    pr, o = _small_problem(model=model)
    rng = np.random.default_rng(12)
    coords = pr["coords"].copy()
    o.eval_full(coords)
    groups = synth.single_point_fos(pr["mesh"])
    for rnd in range(3):
        gids = rng.permutation(len(groups))[:9]
        for g in gids:
            cands = np.arange(coords.shape[0])
            cur = np.stack([o.coords(c) for c in cands])
            tc = synth.trial_coords(cur, groups, [g] * len(cands), cands, 0.3, pr["mesh"], rng)
            obj = o.eval_partial(groups, [g] * len(cands), cands, tc)
            acc = rng.uniform(size=len(cands)) < 0.7
            o.commit(acc)
    final = np.stack([o.coords(c) for c in range(coords.shape[0])])
    cur = o.objectives()
    o2 = orc.Oracle(pr["img"][0], pr["img"][1], *pr["spacing"], pr["mesh"], guide=pr["guide"], model=model)
    fresh = o2.eval_full(final)
    assert np.allclose(cur, fresh, rtol=1e-12, atol=1e-15)


def test_partial_sum_over_single_point_groups_is_four_times_full():
    """Each tet has 4 vertices: over all single-point groups (no move) every
    tet is counted 4 times, bit-exactly on coverage counts."""
    pr, o = _small_problem()
    o.eval_full(pr["coords"])
    groups = synth.single_point_fos(pr["mesh"])
    c = 1
    cur = o.coords(c)
    tot = np.zeros(2, np.int64)
    for g in range(len(groups)):
        tc = cur[:, :, groups[g]][None]
        obj = o.eval_partial(groups, [g], [c], tc)
        assert np.allclose(obj[0], o.objectives([c])[0], rtol=1e-13, atol=1e-16)
        tot += o.trial(0)["cov"].sum(axis=0)
    full = o.terms(c)["cov"].sum(axis=0)
    assert np.array_equal(tot, 4 * full)
    assert np.array_equal(full, [16 ** 3, 16 ** 3])


def test_partial_equals_full_on_trial_state():
    pr, o = _small_problem(seed=13)
    rng = np.random.default_rng(14)
    o.eval_full(pr["coords"])
    groups = synth.tet_fos(pr["mesh"], rng)
    gids = [0, 3, 5, 7]
    cands = [0, 1, 2, 3]
    cur = np.stack([o.coords(c) for c in cands])
    tc = synth.trial_coords(cur, groups, gids, cands, 0.4, pr["mesh"], rng)
    obj = o.eval_partial(groups, gids, cands, tc)
    for k, (g, c) in enumerate(zip(gids, cands)):
        full = cur[k].copy()
        full[:, :, groups[g]] = tc[k][:, :, : len(groups[g])]
        o2 = orc.Oracle(pr["img"][0], pr["img"][1], *pr["spacing"], pr["mesh"], guide=pr["guide"])
        want = o2.eval_full(full[None])[0]
        assert np.allclose(obj[k], want, rtol=1e-12, atol=1e-15)


def test_commit_rejects_overlapping_accepts():
    pr, o = _small_problem()
    o.eval_full(pr["coords"])
    groups = synth.single_point_fos(pr["mesh"])
    cur = o.coords(0)
    tc = np.stack([cur[:, :, groups[13]], cur[:, :, groups[14]]])
    o.eval_partial(groups, [13, 14], [0, 0], tc)
    with pytest.raises(ValueError):
        o.commit([1, 1])
    o.commit([1, 0])
