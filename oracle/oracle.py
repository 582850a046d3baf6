"""ctypes wrapper of the plain FP64 CPU oracle (``dmr_oracle.c``).

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this module; the CUDA library and its
Python binding never do.  The oracle follows the paper's definitions
(Sec. 2.1 mesh model, Sec. 2.2 partial evaluation, Sec. 2.3.1-2.3.4
objectives and constraints) in FP64 with FMA contraction disabled.

Arrays use the same layouts as the C-ABI of the CUDA library:
images ``[nz, ny, nx]``; candidate coordinates ``[C, 2, 3, P]`` (mesh,
axis, point); guidance pairs ``[ng, 2, 3]`` (source point, target point).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dmr_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libdmr_oracle.so")
_lock = threading.Lock()
_lib = None

SPRING = 0
LINEAR = 1

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_i8p = np.ctypeslib.ndpointer(dtype=np.int8, flags="C_CONTIGUOUS")


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, FMA contraction off, OpenMP)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-fopenmp", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build_oracle())
        vp = ctypes.c_void_p
        lib.dmo_create.restype = vp
        lib.dmo_create.argtypes = [_i32p, _i32p, _f64p, _f64p, _f64p, _f64p, _i32p, _f64p,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_double]
        lib.dmo_destroy.argtypes = [vp]
        lib.dmo_set_guide_sets.argtypes = [vp, ctypes.c_void_p]
        lib.dmo_link_violations.argtypes = [vp, _f64p, _i32p]
        lib.dmo_link_point.argtypes = [vp, _f64p, ctypes.c_int, ctypes.c_int]
        lib.dmo_ntet.argtypes = [vp]
        lib.dmo_npoints.argtypes = [vp]
        lib.dmo_get_tets.argtypes = [vp, _i32p]
        lib.dmo_get_star.argtypes = [vp, _i32p, _i32p]
        lib.dmo_get_face_perm.argtypes = [vp, _i8p]
        lib.dmo_rest_coords.argtypes = [vp, ctypes.c_int, _f64p]
        lib.dmo_eval_full.argtypes = [vp, ctypes.c_int, _f64p, _f64p]
        lib.dmo_eval_partial.argtypes = [vp, ctypes.c_int, _i32p, _i32p, _i32p, _f64p, _f64p]
        lib.dmo_commit.argtypes = [vp, _u8p]
        lib.dmo_get_objectives.argtypes = [vp, ctypes.c_int, _i32p, _f64p]
        lib.dmo_get_raw.argtypes = [vp, ctypes.c_int, _f64p]
        lib.dmo_get_coords.argtypes = [vp, ctypes.c_int, _f64p]
        lib.dmo_get_terms.argtypes = [vp, ctypes.c_int, _f64p, _i32p, _f64p, _i32p]
        lib.dmo_get_landmarks.argtypes = [vp, ctypes.c_int, _i32p, _f64p]
        lib.dmo_get_trial.argtypes = [vp, ctypes.c_int, _i32p, _f64p, _i32p, _f64p, _i32p]
        lib.dmo_tet_terms.argtypes = [vp, _f64p, ctypes.c_int, _f64p, _i32p, _f64p, _i32p]
        lib.dmo_inside.argtypes = [vp, ctypes.c_int, _f64p, ctypes.c_int, _f64p]
        lib.dmo_coverage_mask.argtypes = [vp, ctypes.c_int, _f64p, ctypes.c_int, _u8p]
        lib.dmo_map_point.argtypes = [vp, ctypes.c_int, _f64p, ctypes.c_int, _f64p, _f64p]
        lib.dmo_sample.restype = ctypes.c_double
        lib.dmo_sample.argtypes = [vp, ctypes.c_int, _f64p, ctypes.POINTER(ctypes.c_int32)]
        lib.dmo_six_vol.restype = ctypes.c_double
        lib.dmo_six_vol.argtypes = [vp, ctypes.c_int, _f64p, ctypes.c_int]
        lib.dmo_refine.restype = ctypes.c_int
        lib.dmo_refine.argtypes = [_f64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _f64p]
        lib.dmo_num_tets.argtypes = [_i32p]
        lib.dmo_build_tets.argtypes = [_i32p, _i32p]
        lib.dmo_set_threads.argtypes = [ctypes.c_int]
        lib.dmo_max_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def set_threads(n: int) -> None:
    _load().dmo_set_threads(int(n))


def max_threads() -> int:
    return int(_load().dmo_max_threads())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def build_tets(mesh_pts):
    lib = _load()
    m = _i32(mesh_pts)
    nt = lib.dmo_num_tets(m)
    out = np.zeros((max(nt, 1), 4), np.int32)
    lib.dmo_build_tets(m, out)
    return out[:nt]


class Oracle:
    """One registration problem (image pair, mesh size, guidance) plus the
    population state used for partial evaluation."""

    def __init__(self, img_s, img_t, spacing_s, spacing_t, mesh_pts, guide=None,
                 black_rule=True, model=SPRING, lam=1.0, mu=1.0, guide_sets=None):
        self._lib = _load()
        img_s = _f64(img_s)
        img_t = _f64(img_t)
        self.n = [np.array(img_s.shape[::-1], np.int32), np.array(img_t.shape[::-1], np.int32)]
        self.sp = [_f64(spacing_s), _f64(spacing_t)]
        self.m = _i32(mesh_pts)
        g = np.zeros((0, 2, 3)) if guide is None else _f64(guide).reshape(-1, 2, 3)
        self.ng = g.shape[0]
        gbuf = _f64(g.reshape(-1)) if self.ng else np.zeros(6, np.float64)
        self.model = int(model)
        self.h = self._lib.dmo_create(self.n[0], self.n[1], self.sp[0], self.sp[1],
                                      img_s.reshape(-1), img_t.reshape(-1), self.m, gbuf,
                                      self.ng, int(bool(black_rule)), self.model,
                                      float(lam), float(mu))
        self.ntet = self._lib.dmo_ntet(self.h)
        self._gsets = None
        if guide_sets is not None and self.ng:
            self._gsets = _i32(guide_sets)
            assert self._gsets.shape == (self.ng,)
            self._lib.dmo_set_guide_sets(self.h, self._gsets.ctypes.data)
        self.P = self._lib.dmo_npoints(self.h)
        self.C = 0
        self._last_ntr = 0

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self._lib.dmo_destroy(h)
            self.h = None

    # -- topology -----------------------------------------------------
    def tets(self):
        out = np.zeros((self.ntet, 4), np.int32)
        self._lib.dmo_get_tets(self.h, out)
        return out

    def star(self):
        ptr = np.zeros(self.P + 1, np.int32)
        idx = np.zeros(4 * self.ntet, np.int32)
        self._lib.dmo_get_star(self.h, ptr, idx)
        return ptr, idx

    def face_perm(self):
        out = np.zeros((self.ntet, 4, 4), np.int8)
        self._lib.dmo_get_face_perm(self.h, out)
        return out

    def rest_coords(self, mesh):
        out = np.zeros((3, self.P), np.float64)
        self._lib.dmo_rest_coords(self.h, int(mesh), out)
        return out

    # -- population ---------------------------------------------------
    def eval_full(self, coords):
        c = _f64(coords).reshape(-1, 2, 3, self.P)
        C = c.shape[0]
        obj = np.zeros((C, 4), np.float64)
        self._lib.dmo_eval_full(self.h, C, c.reshape(-1), obj)
        self.C = C
        return obj

    def eval_partial(self, groups, group_ids, cand_ids, tcoords):
        """groups: list of point-id arrays; trial k moves groups[group_ids[k]]
        of candidate cand_ids[k] to tcoords[k] ([2, 3, >=len(group)])."""
        group_ids = np.asarray(group_ids, np.int64)
        cand = _i32(cand_ids)
        ntr = len(group_ids)
        gptr = np.zeros(ntr + 1, np.int32)
        pts, tc = [], []
        tco = np.asarray(tcoords, np.float64)
        for k, g in enumerate(group_ids):
            grp = np.asarray(groups[g], np.int32)
            gptr[k + 1] = gptr[k] + len(grp)
            pts.append(grp)
            tc.append(tco[k][:, :, : len(grp)].reshape(-1))
        gpts = _i32(np.concatenate(pts) if pts else np.zeros(1, np.int32))
        tcf = _f64(np.concatenate(tc) if tc else np.zeros(6, np.float64))
        obj = np.zeros((max(ntr, 1), 4), np.float64)
        rc = self._lib.dmo_eval_partial(self.h, ntr, cand if ntr else np.zeros(1, np.int32),
                                        gptr, gpts, tcf, obj)
        if rc != 0:
            raise ValueError("oracle eval_partial: bad candidate id")
        self._last_ntr = ntr
        return obj[:ntr]

    def commit(self, accept):
        a = np.ascontiguousarray(np.asarray(accept, np.uint8).reshape(-1))
        if a.shape[0] != self._last_ntr:
            raise ValueError("accept length != number of trials")
        rc = self._lib.dmo_commit(self.h, a if len(a) else np.zeros(1, np.uint8))
        if rc != 0:
            raise ValueError("oracle commit: accepted trials of one candidate overlap")

    def objectives(self, cands=None):
        cands = np.arange(self.C) if cands is None else np.asarray(cands)
        c = _i32(cands)
        out = np.zeros((len(c), 4), np.float64)
        self._lib.dmo_get_objectives(self.h, len(c), c, out)
        return out

    def raw(self, c):
        out = np.zeros(4, np.float64)
        self._lib.dmo_get_raw(self.h, int(c), out)
        return out

    def coords(self, c):
        out = np.zeros((2, 3, self.P), np.float64)
        self._lib.dmo_get_coords(self.h, int(c), out)
        return out

    def terms(self, c):
        ssd = np.zeros((self.ntet, 2), np.float64)
        cov = np.zeros((self.ntet, 2), np.int32)
        de = np.zeros(self.ntet, np.float64)
        fo = np.zeros(self.ntet, np.int32)
        self._lib.dmo_get_terms(self.h, int(c), ssd, cov, de, fo)
        return {"ssd": ssd, "cov": cov, "def": de, "fold": fo}

    def landmarks(self, c):
        n = max(self.ng, 1)
        loc = np.zeros((2, n), np.int32)
        gt = np.zeros((2, n), np.float64)
        self._lib.dmo_get_landmarks(self.h, int(c), loc, gt)
        return loc[:, : self.ng], gt[:, : self.ng]

    def trial(self, k, cap=4096):
        tets = np.zeros(cap, np.int32)
        ssd = np.zeros((cap, 2), np.float64)
        cov = np.zeros((cap, 2), np.int32)
        de = np.zeros(cap, np.float64)
        fo = np.zeros(cap, np.int32)
        nt = self._lib.dmo_get_trial(self.h, int(k), tets, ssd, cov, de, fo)
        return {"tets": tets[:nt], "ssd": ssd[:nt], "cov": cov[:nt], "def": de[:nt], "fold": fo[:nt]}

    # -- single items (pins) -----------------------------------------
    def tet_terms(self, coords1, t):
        c = _f64(coords1).reshape(-1)
        ssd = np.zeros(2, np.float64)
        cov = np.zeros(2, np.int32)
        de = np.zeros(1, np.float64)
        fo = np.zeros(1, np.int32)
        self._lib.dmo_tet_terms(self.h, c, int(t), ssd, cov, de, fo)
        return {"ssd": ssd, "cov": cov, "def": float(de[0]), "fold": int(fo[0])}

    def inside(self, mesh, coords1, t, p):
        return bool(self._lib.dmo_inside(self.h, int(mesh), _f64(coords1).reshape(-1), int(t), _f64(p)))

    def coverage_mask(self, mesh, coords1, t):
        n = self.n[mesh]
        out = np.zeros((int(n[2]), int(n[1]), int(n[0])), np.uint8)
        self._lib.dmo_coverage_mask(self.h, int(mesh), _f64(coords1).reshape(-1), int(t), out)
        return out

    def map_point(self, direction, coords1, t, v):
        out = np.zeros(3, np.float64)
        self._lib.dmo_map_point(self.h, int(direction), _f64(coords1).reshape(-1), int(t), _f64(v), out)
        return out

    def sample(self, img, p):
        b = ctypes.c_int32(0)
        s = self._lib.dmo_sample(self.h, int(img), _f64(p), ctypes.byref(b))
        return s, bool(b.value)

    def link_violations(self, coords1):
        """Points outside their link per mesh (Sec. 2.3.4 ray test), [2]."""
        out = np.zeros(2, np.int32)
        self._lib.dmo_link_violations(self.h, _f64(coords1).reshape(-1), out)
        return out

    def link_point(self, coords1, mesh, v):
        """1 when point v of `mesh` lies outside its link (Sec. 2.3.4)."""
        return int(self._lib.dmo_link_point(self.h, _f64(coords1).reshape(-1), int(mesh), int(v)))

    def six_vol(self, mesh, coords1, t):
        return float(self._lib.dmo_six_vol(self.h, int(mesh), _f64(coords1).reshape(-1), int(t)))


def refine(coarse, m):
    """Grid refinement (Sec. 2.4): coords [C][2][3][P] on m points per axis ->
    [C][2][3][P'] on 2m - 1 points per axis (edge, face and cube midpoints)."""
    coarse = np.ascontiguousarray(coarse, np.float64)
    C = coarse.shape[0]
    M = [2 * int(a) - 1 for a in m]
    fine = np.zeros((C, 2, 3, M[0] * M[1] * M[2]), np.float64)
    rc = _load().dmo_refine(coarse.reshape(-1), C, int(m[0]), int(m[1]), int(m[2]), fine.reshape(-1))
    if rc != 0:
        raise ValueError("refine: bad arguments")
    return fine


def hypervolume_bruteforce(points, ref):
    """Hypervolume as the plain definition: the measure of the union of the
    boxes [p_i, ref], by inclusion-exclusion over all non-empty subsets (the
    intersection of boxes [p_i, ref] is the box [max_i p_i, ref]).  Small n
    only (2^n subsets)."""
    import itertools

    pts = [np.asarray(p, np.float64) for p in points if np.all(np.asarray(p) < np.asarray(ref))]
    ref = np.asarray(ref, np.float64)
    total = 0.0
    for k in range(1, len(pts) + 1):
        for sub in itertools.combinations(pts, k):
            corner = np.max(np.stack(sub), axis=0)
            total += (-1) ** (k + 1) * float(np.prod(ref - corner))
    return total
