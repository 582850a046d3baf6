"""Thin Python binding of the C-ABI in ``include/dmr.h`` (libdmr.so).

Argument marshalling only: every step of the evaluation runs in the CUDA
library.  Arrays may be numpy arrays (host) or torch tensors (host or
device); device tensors are passed by pointer without copies.  There is no
CPU fallback: if the CUDA library is missing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdmr.so")

F32, BF16, F16 = 0, 1, 2
SPRING, LINEAR = 0, 1
_DT = {"f32": F32, "float32": F32, "bf16": BF16, "bfloat16": BF16, "f16": F16, "float16": F16}

_lib = None


class DmrError(RuntimeError):
    pass


class _Desc(ctypes.Structure):
    _fields_ = [
        ("img", ctypes.c_void_p * 2),
        ("img_dtype", ctypes.c_int),
        ("dims", (ctypes.c_int * 3) * 2),
        ("spacing", (ctypes.c_double * 3) * 2),
        ("storage_dtype", ctypes.c_int),
        ("mesh_pts", ctypes.c_int * 3),
        ("guide", ctypes.c_void_p),
        ("n_guide", ctypes.c_int),
        ("black_rule", ctypes.c_int),
        ("deform_model", ctypes.c_int),
        ("lam", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("max_candidates", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("guide_set", ctypes.c_void_p),
    ]


def load():
    """Load libdmr.so (built in-tree by ``build.build_library``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise DmrError("CUDA library %s is not built; run __graft_entry__.build()" % LIB_PATH)
    try:  # share one CUDA runtime with torch when it is present
        import torch  # noqa: F401
    except ImportError:
        pass
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, ip = ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p
    sig = {
        "dmr_problem_create": [ctypes.POINTER(_Desc), ctypes.POINTER(ctypes.c_void_p)],
        "dmr_problem_destroy": [vp],
        "dmr_set_stream": [vp, vp],
        "dmr_problem_info": [vp, ip, ip],
        "dmr_tets_out": [vp, ip],
        "dmr_set_fos": [vp, i, ip, ip],
        "dmr_fos_info": [vp, ip, ip, ip],
        "dmr_fos_waves": [vp, ip, ip],
        "dmr_eval_full": [vp, i, vp, vp],
        "dmr_eval_partial": [vp, i, vp, vp, vp, vp],
        "dmr_commit": [vp, vp],
        "dmr_commit_improving": [vp, vp],
        "dmr_objectives_out": [vp, i, vp, vp],
        "dmr_coords_out": [vp, i, vp],
        "dmr_terms_out": [vp, i, vp, vp, vp, vp],
        "dmr_landmarks_out": [vp, i, vp, vp],
        "dmr_trial_out": [vp, i, vp, vp, vp, vp, vp],
        "dmr_samples": [vp, ctypes.POINTER(ctypes.c_longlong), i],
        "dmr_plan_generation": [vp, i, vp, vp, ctypes.POINTER(ctypes.c_void_p)],
        "dmr_plan_run": [vp],
        "dmr_plan_update": [vp, vp],
        "dmr_plan_destroy": [vp],
        "dmr_plan_launches": [vp, ip],
        "dmr_plan_kernel_ms": [vp, ip, ip],
        "dmr_set_tile": [vp, i, i],
        "dmr_eval_one_noalloc": [vp, vp, vp],
        "dmr_sample_counts": [vp, vp, vp, i],
        "dmr_autotune": [vp, i, ip, ip, ip],
        "dmr_batch_create": [i, vp, ctypes.POINTER(ctypes.c_void_p)],
        "dmr_batch_destroy": [vp],
        "dmr_batch_plan_generation": [vp, vp, vp, vp, ctypes.POINTER(ctypes.c_void_p)],
        "dmr_hypervolume": [vp, i, i, vp, vp],
        "dmr_refine": [vp, i, vp, vp, vp],
        "dmr_link_check": [vp, i, vp, vp],
        "dmr_mlp_create": [ctypes.c_ulonglong, vp, ctypes.POINTER(ctypes.c_void_p)],
        "dmr_mlp_destroy": [vp],
        "dmr_mlp_n_params": [],
        "dmr_mlp_params": [vp, vp, vp],
        "dmr_mlp_features": [vp, vp, i, vp],
        "dmr_mlp_forward": [vp, vp, i, vp],
        "dmr_mlp_train_step": [vp, vp, vp, i, ctypes.c_float, vp, vp],
        "dmr_get_tile": [vp, ip, ip],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.dmr_last_error.restype = ctypes.c_char_p
    lib.dmr_last_error.argtypes = []
    _lib = lib
    return lib


def exported_symbols():
    return [
        "dmr_problem_create", "dmr_problem_destroy", "dmr_set_stream", "dmr_problem_info", "dmr_tets_out",
        "dmr_set_fos", "dmr_fos_info", "dmr_fos_waves", "dmr_eval_full", "dmr_eval_partial", "dmr_commit",
        "dmr_commit_improving", "dmr_objectives_out", "dmr_coords_out", "dmr_terms_out", "dmr_landmarks_out",
        "dmr_trial_out", "dmr_samples", "dmr_plan_generation", "dmr_plan_run", "dmr_plan_update", "dmr_plan_destroy",
        "dmr_plan_launches", "dmr_plan_kernel_ms", "dmr_set_tile", "dmr_get_tile", "dmr_autotune", "dmr_batch_create", "dmr_batch_destroy",
        "dmr_batch_plan_generation", "dmr_hypervolume", "dmr_refine", "dmr_link_check", "dmr_mlp_create", "dmr_mlp_destroy", "dmr_mlp_n_params",
        "dmr_mlp_params", "dmr_mlp_features", "dmr_mlp_forward", "dmr_mlp_train_step", "dmr_eval_one_noalloc", "dmr_sample_counts", "dmr_last_error",
    ]


def _check(rc):
    if rc < 0:
        raise DmrError("dmr error %d: %s" % (rc, _lib.dmr_last_error().decode()))
    return rc


class _Arg:
    """Pointer to an array argument: numpy (host) or torch (host/device)."""

    def __init__(self, a, dtype):
        self.keep = None
        if a is None:
            self.ptr = None
            return
        try:
            import torch

            if isinstance(a, torch.Tensor):
                want = {np.float64: torch.float64, np.int32: torch.int32, np.uint8: torch.uint8,
                        np.float32: torch.float32, np.uint16: torch.int16}[dtype]
                t = a.contiguous()
                if t.dtype != want and not (dtype == np.uint16 and t.dtype in (torch.bfloat16, torch.float16)):
                    t = t.to(want)
                self.keep = t
                self.ptr = t.data_ptr()
                return
        except ImportError:
            pass
        arr = np.ascontiguousarray(a, dtype=dtype)
        self.keep = arr
        self.ptr = arr.ctypes.data


def _ptr(a, dtype):
    return _Arg(a, dtype)


def _is_torch(a):
    try:
        import torch

        return isinstance(a, torch.Tensor)
    except ImportError:
        return False


def _out_like(ref, shape, dtype):
    """Output buffer on the same device as ``ref`` (torch) or numpy."""
    if _is_torch(ref):
        import torch

        tdt = {np.float64: torch.float64, np.int32: torch.int32, np.uint8: torch.uint8}[dtype]
        return torch.empty(shape, dtype=tdt, device=ref.device)
    return np.zeros(shape, dtype)


def _addr(buf):
    return buf.data_ptr() if _is_torch(buf) else buf.ctypes.data


def hypervolume(points, ref):
    """Exact hypervolume of ``points`` [n, d] (minimisation) w.r.t. ``ref``."""
    lib = load()
    pts = np.ascontiguousarray(np.asarray(points, np.float64).reshape(-1, len(ref)))
    r = np.ascontiguousarray(np.asarray(ref, np.float64))
    out = ctypes.c_double()
    _check(lib.dmr_hypervolume(pts.ctypes.data if len(pts) else None, len(pts), len(r), r.ctypes.data,
                               ctypes.addressof(out)))
    return out.value


def refine(coarse, m, stream=None):
    """Grid refinement (Sec. 2.4): coords [C, 2, 3, P] on m points per axis ->
    [C, 2, 3, P'] on 2m - 1 points per axis, computed on the GPU.  numpy in,
    numpy out; a torch tensor in gives a torch tensor on the same device."""
    lib = load()
    M = [2 * int(a) - 1 for a in m]
    C = int(coarse.shape[0])
    mm = (ctypes.c_int * 3)(*[int(a) for a in m])
    if _is_torch(coarse):
        import torch

        src = coarse.contiguous().to(torch.float64)
        out = torch.empty((C, 2, 3, M[0] * M[1] * M[2]), dtype=torch.float64, device=src.device)
        st = stream if stream is not None else (torch.cuda.current_stream().cuda_stream if src.is_cuda else 0)
        _check(lib.dmr_refine(src.data_ptr(), C, ctypes.addressof(mm), out.data_ptr(), st))
        return out
    src = np.ascontiguousarray(coarse, np.float64)
    out = np.zeros((C, 2, 3, M[0] * M[1] * M[2]), np.float64)
    _check(lib.dmr_refine(src.ctypes.data, C, ctypes.addressof(mm), out.ctypes.data, stream or 0))
    return out


class Problem:
    """One registration problem plus its candidate population (C-ABI handle)."""

    def __init__(self, img_s, img_t, spacing_s, spacing_t, mesh_pts, guide=None, black_rule=True,
                 model=SPRING, lam=1.0, mu=1.0, storage="f32", max_candidates=1, stream=None,
                 img_dtype=None, guide_sets=None):
        lib = load()
        self._lib = lib
        d = _Desc()
        imgs = [img_s, img_t]
        if img_dtype is None:
            img_dtype = "f32"
        idt = _DT[img_dtype] if isinstance(img_dtype, str) else int(img_dtype)
        self._keep = []
        for k, im in enumerate(imgs):
            if _is_torch(im):
                shape = tuple(im.shape)
                a = _Arg(im, np.float32 if idt == F32 else np.uint16)
            else:
                shape = np.asarray(im).shape
                a = _Arg(im, np.float32 if idt == F32 else np.uint16)
            self._keep.append(a)
            d.img[k] = a.ptr
            nz, ny, nx = shape
            d.dims[k][0], d.dims[k][1], d.dims[k][2] = nx, ny, nz
        sps = [spacing_s, spacing_t]
        for k in range(2):
            for a in range(3):
                d.spacing[k][a] = float(sps[k][a])
        d.img_dtype = idt
        d.storage_dtype = _DT[storage] if isinstance(storage, str) else int(storage)
        for a in range(3):
            d.mesh_pts[a] = int(mesh_pts[a])
        self.ng = 0
        if guide is not None and len(guide):
            g = np.ascontiguousarray(np.asarray(guide, np.float64).reshape(-1, 2, 3))
            self._guide = g
            d.guide = g.ctypes.data
            d.n_guide = g.shape[0]
            self.ng = g.shape[0]
            if guide_sets is not None:
                gs = np.ascontiguousarray(np.asarray(guide_sets, np.int32).reshape(-1))
                if gs.shape[0] != self.ng:
                    raise ValueError("guide_sets needs one set id per guidance pair")
                self._gsets = gs
                d.guide_set = gs.ctypes.data
        d.black_rule = int(bool(black_rule))
        d.deform_model = int(model)
        d.lam = float(lam)
        d.mu = float(mu)
        d.max_candidates = int(max_candidates)
        d.stream = stream
        h = ctypes.c_void_p()
        _check(lib.dmr_problem_create(ctypes.byref(d), ctypes.byref(h)))
        self.h = h
        self._keep = None
        P, T = ctypes.c_int(), ctypes.c_int()
        lib.dmr_problem_info(self.h, ctypes.byref(P), ctypes.byref(T))
        self.P, self.ntet = P.value, T.value
        self.C = 0
        self.gmax = 0
        self._groups = None

    def close(self):
        if getattr(self, "h", None):
            self._lib.dmr_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        _check(self._lib.dmr_set_stream(self.h, stream))

    def tets(self):
        out = np.zeros((self.ntet, 4), np.int32)
        _check(self._lib.dmr_tets_out(self.h, out.ctypes.data))
        return out

    def set_tile(self, warps=0, voxels_per_warp=0):
        _check(self._lib.dmr_set_tile(self.h, int(warps), int(voxels_per_warp)))

    def tile(self):
        w, v = ctypes.c_int(), ctypes.c_int()
        _check(self._lib.dmr_get_tile(self.h, ctypes.addressof(w), ctypes.addressof(v)))
        return w.value, v.value

    def autotune(self, n_cand=0):
        """Pick the fastest raster tile shape; returns (warps, voxels per warp,
        {(warps, voxels): ms})."""
        w, v = ctypes.c_int(), ctypes.c_int()
        tab = (ctypes.c_float * 9)()
        _check(self._lib.dmr_autotune(self.h, int(n_cand), ctypes.addressof(w), ctypes.addressof(v),
                                      ctypes.addressof(tab)))
        table = {(W, V): tab[3 * i + j] for i, W in enumerate((4, 8, 16)) for j, V in enumerate((32, 64, 128))}
        return w.value, v.value, table

    # -- FOS --------------------------------------------------------------
    def set_fos(self, groups):
        ptr = np.zeros(len(groups) + 1, np.int32)
        for g, pts in enumerate(groups):
            ptr[g + 1] = ptr[g] + len(pts)
        flat = np.ascontiguousarray(np.concatenate([np.asarray(x, np.int32) for x in groups]))
        _check(self._lib.dmr_set_fos(self.h, len(groups), ptr.ctypes.data, flat.ctypes.data))
        mg, mt, nw = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self._lib.dmr_fos_info(self.h, ctypes.byref(mg), ctypes.byref(mt), ctypes.byref(nw)))
        self.gmax, self.max_touched, self.n_waves = mg.value, mt.value, nw.value
        self._groups = [np.asarray(x, np.int32) for x in groups]

    def waves(self):
        wp = np.zeros(self.n_waves + 1, np.int32)
        wg = np.zeros(len(self._groups), np.int32)
        _check(self._lib.dmr_fos_waves(self.h, wp.ctypes.data, wg.ctypes.data))
        return [wg[wp[w]:wp[w + 1]] for w in range(self.n_waves)]

    # -- evaluation -------------------------------------------------------
    def eval_full(self, coords, out=None):
        C = coords.shape[0]
        a = _Arg(coords, np.float64)
        obj = out if out is not None else _out_like(coords, (C, 4), np.float64)
        _check(self._lib.dmr_eval_full(self.h, C, a.ptr, _addr(obj)))
        self.C = C
        return obj

    def eval_partial(self, group_ids, cand_ids, trial_coords, out=None):
        n = len(group_ids)
        g = _Arg(group_ids, np.int32)
        c = _Arg(cand_ids, np.int32)
        tc = _Arg(trial_coords, np.float64)
        obj = out if out is not None else _out_like(trial_coords, (n, 4), np.float64)
        _check(self._lib.dmr_eval_partial(self.h, n, g.ptr, c.ptr, tc.ptr, _addr(obj)))
        self._ntr = n
        return obj

    def commit(self, accept):
        a = _Arg(accept, np.uint8)
        _check(self._lib.dmr_commit(self.h, a.ptr))

    def commit_improving(self, want_accept=True):
        out = np.zeros(self._ntr, np.uint8) if want_accept else None
        _check(self._lib.dmr_commit_improving(self.h, out.ctypes.data if out is not None else None))
        return out

    def objectives(self, cands=None):
        cands = np.arange(self.C, dtype=np.int32) if cands is None else np.asarray(cands, np.int32)
        out = np.zeros((len(cands), 4), np.float64)
        _check(self._lib.dmr_objectives_out(self.h, len(cands), cands.ctypes.data, out.ctypes.data))
        return out

    def link_check(self, cands=None):
        """Points outside their link per (candidate, mesh), [n, 2] (Sec. 2.3.4)."""
        cands = np.arange(self.C, dtype=np.int32) if cands is None else np.asarray(cands, np.int32)
        out = np.zeros((len(cands), 2), np.int32)
        _check(self._lib.dmr_link_check(self.h, len(cands), cands.ctypes.data, out.ctypes.data))
        return out

    def coords(self, c):
        out = np.zeros((2, 3, self.P), np.float64)
        _check(self._lib.dmr_coords_out(self.h, int(c), out.ctypes.data))
        return out

    def terms(self, c):
        cov = np.zeros((self.ntet, 2), np.int32)
        ssd = np.zeros((self.ntet, 2), np.float64)
        de = np.zeros(self.ntet, np.float64)
        fo = np.zeros(self.ntet, np.int32)
        _check(self._lib.dmr_terms_out(self.h, int(c), cov.ctypes.data, ssd.ctypes.data, de.ctypes.data,
                                       fo.ctypes.data))
        return {"cov": cov, "ssd": ssd, "def": de, "fold": fo}

    def landmarks(self, c):
        n = max(self.ng, 1)
        loc = np.zeros((2, n), np.int32)
        gt = np.zeros((2, n), np.float64)
        _check(self._lib.dmr_landmarks_out(self.h, int(c), loc.ctypes.data, gt.ctypes.data))
        return loc[:, : self.ng], gt[:, : self.ng]

    def trial(self, k, cap=None):
        cap = cap or max(self.max_touched, 1)
        tets = np.zeros(cap, np.int32)
        cov = np.zeros((cap, 2), np.int32)
        ssd = np.zeros((cap, 2), np.float64)
        de = np.zeros(cap, np.float64)
        fo = np.zeros(cap, np.int32)
        n = _check(self._lib.dmr_trial_out(self.h, int(k), tets.ctypes.data, cov.ctypes.data, ssd.ctypes.data,
                                           de.ctypes.data, fo.ctypes.data))
        return {"tets": tets[:n], "cov": cov[:n], "ssd": ssd[:n], "def": de[:n], "fold": fo[:n]}

    def eval_one_noalloc(self, coords, out):
        """Objectives of one candidate (device tensor [2, 3, P]) into ``out``
        (device tensor [4]) without any allocation in the library.  Both must
        already be contiguous float64 CUDA tensors of those sizes on the
        current device: this method converts nothing, since a converted copy
        would itself be an allocation (and could be freed before the queued
        kernels read it)."""
        import torch

        dev = torch.cuda.current_device()
        for name, t, n in (("coords", coords, 6 * self.P), ("out", out, 4)):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise DmrError("eval_one_noalloc: %s must be a contiguous float64 CUDA tensor" % name)
            if t.device.index != dev:
                raise DmrError("eval_one_noalloc: %s is on cuda:%d, the current device is cuda:%d"
                               % (name, t.device.index, dev))
            if (t.numel() != n) if name == "coords" else (t.numel() < n):
                raise DmrError("eval_one_noalloc: %s holds %d values, needs %s%d" % (
                    name, t.numel(), "" if name == "coords" else "at least ", n))
        _check(self._lib.dmr_eval_one_noalloc(self.h, coords.data_ptr(), out.data_ptr()))
        return out

    def samples(self, reset=False):
        v = ctypes.c_longlong()
        _check(self._lib.dmr_samples(self.h, ctypes.byref(v), int(bool(reset))))
        return v.value

    def sample_counts(self, reset=False):
        """(counted, executed) voxel-samples since the last reset."""
        c, e = ctypes.c_longlong(), ctypes.c_longlong()
        _check(self._lib.dmr_sample_counts(self.h, ctypes.byref(c), ctypes.byref(e), int(bool(reset))))
        return c.value, e.value

    def plan_generation(self, cand_ids, deltas):
        c = _Arg(cand_ids, np.int32)
        d = _Arg(deltas, np.float64)
        h = ctypes.c_void_p()
        _check(self._lib.dmr_plan_generation(self.h, len(cand_ids), c.ptr, d.ptr, ctypes.byref(h)))
        return Plan(self, h)


class Batch:
    """Several independent problems served by one set of launches per wave."""

    def __init__(self, problems):
        self.problems = list(problems)
        lib = problems[0]._lib
        arr = (ctypes.c_void_p * len(self.problems))(*[p.h.value for p in self.problems])
        h = ctypes.c_void_p()
        _check(lib.dmr_batch_create(len(self.problems), ctypes.addressof(arr), ctypes.byref(h)))
        self.h = h
        self._lib = lib

    def plan_generation(self, cand_ids, deltas):
        n = len(self.problems)
        cargs = [_Arg(c, np.int32) for c in cand_ids]
        dargs = [_Arg(d, np.float64) for d in deltas]
        nc = (ctypes.c_int * n)(*[len(c) for c in cand_ids])
        cp = (ctypes.c_void_p * n)(*[a.ptr for a in cargs])
        dp = (ctypes.c_void_p * n)(*[a.ptr for a in dargs])
        h = ctypes.c_void_p()
        _check(self._lib.dmr_batch_plan_generation(self.h, ctypes.addressof(nc), ctypes.addressof(cp),
                                                   ctypes.addressof(dp), ctypes.byref(h)))
        return Plan(self.problems[0], h)

    def close(self):
        if getattr(self, "h", None):
            self._lib.dmr_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """A CUDA graph running one GOMEA generation of partial evaluations."""

    def __init__(self, prob, h):
        self.prob = prob
        self.h = h
        n = ctypes.c_int()
        _check(prob._lib.dmr_plan_launches(self.h, ctypes.byref(n)))
        self.launches = n.value

    def run(self):
        _check(self.prob._lib.dmr_plan_run(self.h))

    def update(self, deltas):
        """New proposal offsets for later runs: one array (single problem) or
        a list with one per problem, laid out as at plan creation; numpy or
        torch (host or device)."""
        arrs = deltas if isinstance(deltas, (list, tuple)) else [deltas]
        args = [_Arg(a, np.float64) for a in arrs]
        ptrs = (ctypes.c_void_p * len(args))(*[a.ptr for a in args])
        self._keep = args
        _check(self.prob._lib.dmr_plan_update(self.h, ctypes.addressof(ptrs)))

    def kernel_ms(self):
        """(set-up ms, raster ms) of the last completed run; set-up is -1 (not
        timed: only the raster kernels carry timing events)."""
        su, ra = ctypes.c_float(), ctypes.c_float()
        _check(self.prob._lib.dmr_plan_kernel_ms(self.h, ctypes.addressof(su), ctypes.addressof(ra)))
        return su.value, ra.value

    def close(self):
        if getattr(self, "h", None):
            self.prob._lib.dmr_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """The learned-proposal network; tensors are torch CUDA tensors."""

    def __init__(self, seed=0, stream=None):
        self._lib = load()
        h = ctypes.c_void_p()
        _check(self._lib.dmr_mlp_create(int(seed), stream, ctypes.byref(h)))
        self.h = h
        self.n_params = self._lib.dmr_mlp_n_params()

    def params(self):
        out = np.zeros(self.n_params, np.float32)
        _check(self._lib.dmr_mlp_params(self.h, out.ctypes.data, None))
        return out

    def set_params(self, p):
        a = np.ascontiguousarray(p, np.float32)
        assert a.size == self.n_params
        _check(self._lib.dmr_mlp_params(self.h, None, a.ctypes.data))

    @staticmethod
    def features(prob, coords):
        """coords: torch CUDA float64 [C, 2, 3, P] -> BF16 (as int16) [C*P, 256]."""
        import torch

        C = coords.shape[0]
        X = torch.empty((C * prob.P, 256), dtype=torch.bfloat16, device=coords.device)
        c = coords.contiguous()
        _check(load().dmr_mlp_features(prob.h, c.data_ptr(), C, X.data_ptr()))
        return X

    def forward(self, X):
        import torch

        out = torch.empty((X.shape[0], 6), dtype=torch.float32, device=X.device)
        Xc = X.contiguous()
        _check(self._lib.dmr_mlp_forward(self.h, Xc.data_ptr(), X.shape[0], out.data_ptr()))
        return out

    def train_step(self, X, Y, lr, want_grad=False, want_loss=True):
        """One step; returns the loss (and the gradient with want_grad).  With
        want_loss=False and no gradient the step is only enqueued (returns
        None) and the inputs must stay alive until the stream reaches it."""
        Xc, Yc = X.contiguous(), Y.contiguous().float()
        loss = ctypes.c_float()
        g = np.zeros(self.n_params, np.float32) if want_grad else None
        lp = ctypes.addressof(loss) if (want_loss or want_grad) else None
        _check(self._lib.dmr_mlp_train_step(self.h, Xc.data_ptr(), Yc.data_ptr(), X.shape[0], float(lr), lp,
                                            g.ctypes.data if g is not None else None))
        if lp is None:
            return None
        return (loss.value, g) if want_grad else loss.value

    def close(self):
        if getattr(self, "h", None):
            self._lib.dmr_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
