"""Seeded synthetic inputs for the registration workloads.

This module produces input data only: image pairs, initial mesh lattices,
jittered candidate populations, guidance point pairs, FOS point groups and
trial (proposal) coordinates.  It holds none of the objective arithmetic;
both the CUDA library's tests and the FP64 oracle consume what it returns.

Workloads (all seeded with ``numpy.random.default_rng(seed)``):

* ``sphere_pair``     16^3 float32, sphere r=5 at the centre (1 on 0) vs the
                      same sphere stretched 1.2x in x, both + N(0, 0.01);
                      3^3-point meshes jittered U(-0.5, 0.5); 5 guidance
                      pairs on the sphere surface; population 10.
* ``ellipsoid_pair``  64^3 float32, three overlapping ellipsoids 0.3/0.6/1.0
                      on 0, target = source warped by a sum of 4 Gaussian
                      displacement bumps (amplitude <= 6 voxels); 5^3-point
                      meshes; 20 guidance pairs; population 128.
* ``batch_problems``  64 problems built like ``ellipsoid_pair`` with edge
                      length ~ U{32..128}, mesh points ~ U{4..9} per axis and
                      population ~ U{64..512}.
* ``ct_phantom``      256x256x96 int16-valued CT-like phantom (air -1000,
                      fat -100 body, six 40 HU organs, 700 HU spine, N(0,10)
                      noise), spacing 1x1x3 mm; target with organs displaced
                      5-25 mm and one organ removed; mapped to [0, 1] with the
                      window [-950, 1000] HU so air is exactly 0 (black);
                      10^3-point meshes, 200 guidance pairs, population 512;
                      a 4x mean-pooled 64x64x24 coarse level.
"""
from __future__ import annotations

import numpy as np

try:  # scipy is only needed for the warped and pooled phantoms
    from scipy import ndimage as _ndi
except Exception:  # pragma: no cover
    _ndi = None


# --------------------------------------------------------------- meshes
def fixed_axes(m):
    """uint8 [P]: bit a set when the point lies on the image border along
    axis a (that coordinate is fixed, Sec. 2.3.4 border rule)."""
    mx, my, mz = (int(v) for v in m)
    a = np.arange(mx)[None, None, :]
    b = np.arange(my)[None, :, None]
    c = np.arange(mz)[:, None, None]
    fx = ((a == 0) | (a == mx - 1)).astype(np.uint8)
    fy = ((b == 0) | (b == my - 1)).astype(np.uint8)
    fz = ((c == 0) | (c == mz - 1)).astype(np.uint8)
    mask = fx * 1 + fy * 2 + fz * 4
    return np.broadcast_to(mask, (mz, my, mx)).reshape(-1).astype(np.uint8)


def rest_lattice(n, m):
    """[3, P] initial point positions on an image of size n=(nx,ny,nz):
    point (a,b,c) at -0.5 + a*n/(m-1) per axis, so border points lie on the
    outer voxel faces."""
    out = []
    grids = np.meshgrid(np.arange(m[2]), np.arange(m[1]), np.arange(m[0]), indexing="ij")
    idx = [grids[2].reshape(-1), grids[1].reshape(-1), grids[0].reshape(-1)]
    for ax in range(3):
        out.append(idx[ax].astype(np.float64) * float(n[ax]) / float(m[ax] - 1) - 0.5)
    return np.stack(out)


def jitter(rest, m, amp, rng):
    """Add U(-amp, amp) to every free coordinate (border axes stay exact)."""
    fix = fixed_axes(m)
    out = rest.copy()
    for ax in range(3):
        free = ((fix >> ax) & 1) == 0
        out[ax, free] += rng.uniform(-amp, amp, size=int(free.sum()))
    return out


def population(n_s, n_t, m, C, amp, rng):
    """[C, 2, 3, P] candidates: both meshes jittered around their lattices."""
    rs, rt = rest_lattice(n_s, m), rest_lattice(n_t, m)
    out = np.empty((C, 2, 3, rs.shape[1]), np.float64)
    for c in range(C):
        out[c, 0] = jitter(rs, m, amp, rng)
        out[c, 1] = jitter(rt, m, amp, rng)
    return out


def single_point_fos(m):
    """One FOS group per mesh point."""
    P = int(np.prod(m))
    return [np.array([p], np.int32) for p in range(P)]


def tet_fos(m, rng):
    """Sec. 2.2: per cube, the points of one of its six tetrahedra (picked at
    random) form a group.  Returned as sorted point ids."""
    groups = []
    mx, my, mz = (int(v) for v in m)
    for cz in range(mz - 1):
        for cy in range(my - 1):
            for cx in range(mx - 1):
                par = (cx & 1, cy & 1, cz & 1)
                start = [cx + par[0], cy + par[1], cz + par[2]]
                d = [-1 if p else 1 for p in par]
                order = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)][rng.integers(6)]
                v = [list(start)]
                for ax in order:
                    nxt = list(v[-1])
                    nxt[ax] += d[ax]
                    v.append(nxt)
                ids = sorted(a + mx * (b + my * c) for a, b, c in v)
                groups.append(np.array(ids, np.int32))
    return groups


def trial_coords(coords, groups, group_ids, cand_ids, sigma, m, rng):
    """[ntr, 2, 3, Gmax] proposals: the candidate's current group coordinates
    plus N(0, sigma) on free axes (border axes are left exact)."""
    fix = fixed_axes(m)
    gmax = max(len(groups[g]) for g in group_ids) if len(group_ids) else 1
    out = np.zeros((len(group_ids), 2, 3, gmax), np.float64)
    for k, (g, c) in enumerate(zip(group_ids, cand_ids)):
        pts = groups[g]
        cur = coords[c][:, :, pts]
        noise = rng.normal(0.0, sigma, size=cur.shape)
        for ax in range(3):
            noise[:, ax, ((fix[pts] >> ax) & 1) == 1] = 0.0
        out[k, :, :, : len(pts)] = cur + noise
    return out


# --------------------------------------------------------------- images
def _noise(shape, sd, rng):
    return rng.normal(0.0, sd, size=shape).astype(np.float32)


def sphere_pair(seed=0, n=16, radius=5.0, stretch=1.2, n_guide=5, mesh=3, C=10, amp=0.5):
    rng = np.random.default_rng(seed)
    c = (n - 1) / 2.0
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    src = (((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2) <= radius ** 2).astype(np.float32)
    tgt = ((((x - c) / stretch) ** 2 + (y - c) ** 2 + (z - c) ** 2) <= radius ** 2).astype(np.float32)
    src = src + _noise(src.shape, 0.01, rng)
    tgt = tgt + _noise(tgt.shape, 0.01, rng)
    d = rng.normal(size=(n_guide, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    p = c + radius * d
    q = p.copy()
    q[:, 0] = c + stretch * (p[:, 0] - c)
    guide = np.stack([p, q], axis=1)
    m = (mesh, mesh, mesh)
    dims = (n, n, n)
    coords = population(dims, dims, m, C, amp, rng)
    return dict(name="sphere16", img=(src, tgt), spacing=((1.0, 1.0, 1.0), (1.0, 1.0, 1.0)),
                mesh=m, guide=guide, coords=coords, rng=rng)


def cube_pair(seed=0, n=50, half=15.0, depth=6.0, r_src=8.0, r_tgt=5.0, v_cube=0.5, v_sphere=1.0, n_guide=20,
              mesh=6, C=250, amp=0.5):
    """The paper's synthetic problem (Sec. 2.5): a cube deformed non-affinely
    with a shrinking sphere at its centre; each side of the cube bends inward
    as a parabola orthogonal to it; guidance points on the sphere surface.
    The paper gives no sizes or values; the reading here: an n^3 image, a
    cube of half-width `half` (value v_cube) on black, a sphere of radius
    r_src (value v_sphere) at the centre.  In the target every face is pushed
    towards the centre by depth * (1 - u^2)(1 - w^2) (u, w in-face coordinates
    scaled to [-1, 1] over the face) and the sphere has radius r_tgt.
    Guidance: n_guide points on the source sphere and their radial images on
    the target sphere."""
    rng = np.random.default_rng(seed)
    c = (n - 1) / 2.0
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    P = [x - c, y - c, z - c]

    def cube(bend):
        inside = np.ones((n, n, n), bool)
        for ax in range(3):
            u, w = P[(ax + 1) % 3] / half, P[(ax + 2) % 3] / half
            push = bend * np.clip(1.0 - u * u, 0.0, None) * np.clip(1.0 - w * w, 0.0, None)
            inside &= np.abs(P[ax]) <= half - push
        return inside

    def image(bend, r):
        img = np.zeros((n, n, n), np.float32)
        img[cube(bend)] = v_cube
        img[P[0] ** 2 + P[1] ** 2 + P[2] ** 2 <= r * r] = v_sphere
        return img

    src, tgt = image(0.0, r_src), image(depth, r_tgt)
    d = rng.normal(size=(n_guide, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    guide = np.stack([c + r_src * d, c + r_tgt * d], axis=1)
    m = (mesh, mesh, mesh)
    dims = (n, n, n)
    coords = population(dims, dims, m, C, amp, rng)
    return dict(name="cube%d" % n, img=(src, tgt), spacing=((1.0, 1.0, 1.0), (1.0, 1.0, 1.0)), mesh=m,
                guide=guide, coords=coords, rng=rng)


def _ellipsoids(n, rng, count=3, values=(0.3, 0.6, 1.0)):
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    img = np.zeros((n, n, n), np.float32)
    shapes = []
    for k in range(count):
        ctr = rng.uniform(0.3 * n, 0.7 * n, size=3)
        ax = rng.uniform(0.12 * n, 0.3 * n, size=3)
        inside = ((x - ctr[0]) / ax[0]) ** 2 + ((y - ctr[1]) / ax[1]) ** 2 + ((z - ctr[2]) / ax[2]) ** 2 <= 1.0
        img[inside] = values[k]
        shapes.append((ctr, ax))
    return img, shapes


def _bumps(n, rng, count=4, amp=6.0):
    bumps = []
    for _ in range(count):
        ctr = rng.uniform(0.25 * n, 0.75 * n, size=3)
        sig = rng.uniform(0.12 * n, 0.25 * n)
        a = rng.normal(size=3)
        a *= rng.uniform(0.3, 1.0) * amp / np.linalg.norm(a)
        bumps.append((ctr, sig, a))
    return bumps


def _disp(points, bumps):
    """Displacement u(x) at points [N, 3] (x, y, z order)."""
    u = np.zeros_like(points)
    for ctr, sig, a in bumps:
        w = np.exp(-np.sum((points - ctr) ** 2, axis=1) / (2 * sig * sig))
        u += w[:, None] * a[None, :]
    return u


def ellipsoid_pair(seed=1, n=64, mesh=5, C=128, n_guide=20, amp=None):
    if _ndi is None:
        raise RuntimeError("scipy is required for the warped ellipsoid phantom")
    rng = np.random.default_rng(seed)
    src, shapes = _ellipsoids(n, rng)
    bumps = _bumps(n, rng, amp=6.0 * n / 64.0)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    pts = np.stack([x.reshape(-1), y.reshape(-1), z.reshape(-1)], axis=1).astype(np.float64)
    u = _disp(pts, bumps)
    srcpos = pts - u  # T(x) = S(x - u(x))
    tgt = _ndi.map_coordinates(src.astype(np.float64), [srcpos[:, 2], srcpos[:, 1], srcpos[:, 0]],
                               order=1, mode="nearest").reshape(n, n, n).astype(np.float32)
    # guidance: points on the ellipsoid surfaces, carried to x = p + u(x)
    g = []
    for k in range(n_guide):
        ctr, ax = shapes[k % len(shapes)]
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        g.append(ctr + ax * d)
    p = np.array(g, dtype=np.float64).reshape(-1, 3)
    q = p.copy()
    for _ in range(8):
        q = p + _disp(q, bumps)
    guide = np.stack([p, q], axis=1)
    m = (mesh, mesh, mesh)
    dims = (n, n, n)
    cube = n / (mesh - 1)
    coords = population(dims, dims, m, C, 0.1 * cube if amp is None else amp, rng)
    return dict(name="ellipsoid%d" % n, img=(src, tgt), spacing=((1.0, 1.0, 1.0), (1.0, 1.0, 1.0)),
                mesh=m, guide=guide, coords=coords, rng=rng)


def batch_problems(seed=2, count=64, n_range=(32, 128), m_range=(4, 9), c_range=(64, 512)):
    rng = np.random.default_rng(seed)
    probs = []
    for k in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        mm = int(rng.integers(m_range[0], m_range[1] + 1))
        C = int(rng.integers(c_range[0], c_range[1] + 1))
        sub = int(rng.integers(0, 2 ** 31 - 1))
        pr = ellipsoid_pair(seed=sub, n=n, mesh=mm, C=C, n_guide=8)
        pr["name"] = "batch%02d_n%d_m%d_c%d" % (k, n, mm, C)
        probs.append(pr)
    return probs


def _hu_to_unit(hu):
    return np.clip((hu + 950.0) / 1950.0, 0.0, 1.0).astype(np.float32)


def ct_phantom(seed=3, dims=(256, 256, 96), spacing=(1.0, 1.0, 3.0), mesh=10, C=512,
               n_guide=200, level="full", amp=None):
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    X, Y, Z = x * spacing[0], y * spacing[1], z * spacing[2]
    cx, cy = nx * spacing[0] / 2.0, ny * spacing[1] / 2.0
    body = ((X - cx) / (0.43 * nx * spacing[0])) ** 2 + ((Y - cy) / (0.31 * ny * spacing[1])) ** 2 <= 1.0
    spine_c = (cx, cy + 0.18 * ny * spacing[1])
    spine = (X - spine_c[0]) ** 2 + (Y - spine_c[1]) ** 2 <= (0.045 * nx * spacing[0]) ** 2
    organs = []
    zext = nz * spacing[2]
    for k in range(6):
        ang = 2 * np.pi * k / 6 + rng.uniform(-0.3, 0.3)
        r = rng.uniform(0.12, 0.2) * nx * spacing[0]
        ctr = np.array([cx + r * np.cos(ang), cy - 0.04 * ny * spacing[1] + 0.7 * r * np.sin(ang),
                        rng.uniform(0.3, 0.7) * zext])
        ax = np.array([rng.uniform(12, 28), rng.uniform(12, 24), rng.uniform(20, 0.3 * zext)])
        organs.append((ctr, ax))
    removed = int(rng.integers(len(organs)))
    shifts = []
    for _ in organs:
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        shifts.append(d * rng.uniform(5.0, 25.0))

    def render(shifted):
        hu = np.full((nz, ny, nx), -1000.0, np.float64)
        hu[body] = -100.0
        for k, (ctr, ax) in enumerate(organs):
            if shifted and k == removed:
                continue
            c = ctr + (shifts[k] if shifted else 0.0)
            inside = ((X - c[0]) / ax[0]) ** 2 + ((Y - c[1]) / ax[1]) ** 2 + ((Z - c[2]) / ax[2]) ** 2 <= 1.0
            hu[inside & body] = 40.0
        hu[spine] = 700.0
        hu += rng.normal(0.0, 10.0, size=hu.shape)
        return np.round(hu).astype(np.int16)

    hs, ht = render(False), render(True)
    src, tgt = _hu_to_unit(hs.astype(np.float64)), _hu_to_unit(ht.astype(np.float64))
    sp = tuple(float(s) for s in spacing)
    g = []
    kept = [k for k in range(len(organs)) if k != removed]
    for i in range(n_guide):
        k = kept[i % len(kept)]
        ctr, ax = organs[k]
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        pm = ctr + ax * d
        qm = pm + shifts[k]
        g.append([pm / np.array(sp), qm / np.array(sp)])
    guide = np.clip(np.array(g), 0.0, np.array([nx - 1, ny - 1, nz - 1], np.float64))
    if level == "coarse":
        f = 4
        src = src.reshape(nz // f, f, ny // f, f, nx // f, f).mean(axis=(1, 3, 5)).astype(np.float32)
        tgt = tgt.reshape(nz // f, f, ny // f, f, nx // f, f).mean(axis=(1, 3, 5)).astype(np.float32)
        sp = tuple(s * f for s in sp)
        guide = (guide + 0.5) / f - 0.5
        dims = (nx // f, ny // f, nz // f)
    m = (mesh, mesh, mesh)
    cube = min(dims) / (mesh - 1)
    coords = population(dims, dims, m, C, 0.1 * cube if amp is None else amp, rng)
    return dict(name="ct%dx%dx%d" % dims, img=(src, tgt), spacing=(sp, sp), mesh=m, guide=guide,
                coords=coords, rng=rng, hu=(hs, ht) if level == "full" else None)
