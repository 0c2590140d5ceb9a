"""CPU oracle for voxel integration and multi-plane segmentation (arXiv 2510.01592).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.  The
CUDA library never loads it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, compiled with contraction off);
this module compiles it on first use and wraps it with numpy arrays.

Every function is pinned by the ``-m "not gpu"`` tests in ``tests/``:
``test_oracle_integrate.py`` (Eq. 1 keying and sums), ``test_oracle_normals.py``
(Eq. 3 / Eq. 4), ``test_oracle_ccl.py`` (Algorithm 1), ``test_oracle_ransac.py``
(Sec. III.C stages a-c, Philox), ``test_oracle_refit_hull.py`` (refit, hull).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_build/liboracle.so`` (gcc, no contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=gnu11", "-pthread", "-shared", "-fPIC",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Voxel(C.Structure):
    _fields_ = [("vid", C.c_uint32), ("ijk", C.c_int32 * 3), ("S", C.c_int64 * 3), ("c", C.c_uint32),
                ("M", C.c_int32 * 3), ("mu", C.c_float * 3), ("n", C.c_float * 3), ("nbr", C.c_uint32),
                ("status", C.c_uint32), ("label", C.c_uint32)]


class Plane(C.Structure):
    _fields_ = [("label", C.c_uint32), ("n_points", C.c_uint32), ("inlier_count", C.c_uint32),
                ("best_h", C.c_int32), ("ill_conditioned", C.c_int32), ("ransac_n", C.c_float * 3),
                ("ransac_d", C.c_float), ("refit_n", C.c_double * 3), ("refit_d", C.c_double),
                ("basis_u", C.c_float * 3), ("basis_v", C.c_float * 3), ("origin", C.c_float * 3),
                ("hull_off", C.c_uint32), ("hull_n", C.c_uint32), ("point_off", C.c_uint32), ("round", C.c_uint32),
                ("cond", C.c_double)]


class Params(C.Structure):
    _fields_ = [("n_th", C.c_uint32), ("cos_step", C.c_float), ("d_th2", C.c_float), ("cos_ccl", C.c_float),
                ("min_cluster", C.c_uint32), ("n_hyp", C.c_uint32), ("eps", C.c_float), ("seed", C.c_uint64),
                ("classify", C.c_uint32), ("planes_per_cluster", C.c_uint32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp = C.c_void_p
            L.orc_map_create.restype = vp
            L.orc_map_create.argtypes = [C.POINTER(C.c_int32), C.POINTER(C.c_float), C.c_float]
            L.orc_map_destroy.argtypes = [vp]
            L.orc_integrate.argtypes = [vp, C.POINTER(C.c_float), C.c_uint64, C.POINTER(C.c_float)]
            L.orc_map_counts.argtypes = [vp, C.POINTER(C.c_uint64)]
            L.orc_count_occupied.argtypes = [vp]
            L.orc_count_occupied.restype = C.c_uint32
            L.orc_export_sums.argtypes = [vp, C.POINTER(C.c_uint32), C.POINTER(C.c_int64), C.POINTER(C.c_uint32)]
            L.orc_map_scroll.argtypes = [vp, C.POINTER(C.c_int32)]
            L.orc_scroll_target.argtypes = [vp, C.POINTER(C.c_float), C.POINTER(C.c_int32)]
            L.orc_map_window.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_float),
                                         C.POINTER(C.c_uint64)]
            L.orc_jacobi3_f32.argtypes = [C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_float),
                                          C.POINTER(C.c_float), C.POINTER(C.c_float)]
            L.orc_philox4x64.argtypes = [C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
            L.orc_hull_i32.argtypes = [C.POINTER(C.c_int32), C.c_uint32, C.POINTER(C.c_int32)]
            L.orc_hull_i32.restype = C.c_uint32
            L.orc_fit_planes.restype = vp
            L.orc_fit_planes.argtypes = [C.POINTER(C.c_float), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                         C.c_uint32, C.POINTER(Params)]
            L.orc_ransac_counts.restype = C.c_int32
            L.orc_ransac_counts.argtypes = [C.POINTER(C.c_float), C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint64,
                                            C.c_float, C.POINTER(C.c_int64), C.POINTER(C.c_float)]
            L.orc_segment.restype = vp
            L.orc_segment.argtypes = [vp, C.POINTER(Params)]
            L.orc_result_free.argtypes = [vp]
            L.orc_result_sizes.argtypes = [vp, C.POINTER(C.c_uint32)]
            for name, t in (("orc_result_planes", Plane), ("orc_result_hull", C.c_int32),
                            ("orc_result_pts", C.c_float), ("orc_result_pt_vid", C.c_uint32),
                            ("orc_result_inlier", C.c_uint8)):
                getattr(L, name).restype = C.POINTER(t)
                getattr(L, name).argtypes = [vp]
            L.orc_map_n_vox.argtypes = [vp]
            L.orc_map_n_vox.restype = C.c_uint32
            L.orc_map_voxels.argtypes = [vp]
            L.orc_map_voxels.restype = C.POINTER(Voxel)
            L.orc_clear_rays.argtypes = [vp, C.POINTER(C.c_float), C.c_uint64, C.POINTER(C.c_float),
                                         C.POINTER(C.c_uint64)]
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_get_threads.restype = C.c_int
            L.orc_voxel_size.restype = C.c_uint32
            L.orc_plane_size.restype = C.c_uint32
            assert L.orc_voxel_size() == C.sizeof(Voxel), "oracle voxel layout mismatch"
            assert L.orc_plane_size() == C.sizeof(Plane), "oracle plane layout mismatch"
            _lib = L
    return _lib


def set_threads(n: int) -> None:
    """Host threads for the stages whose items are independent (integration,
    normals, per-cluster fits); results do not depend on it."""
    lib().orc_set_threads(int(n))


def threads() -> int:
    return int(lib().orc_get_threads())


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _u32p(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint32))


def make_params(n_th=3, theta_step_deg=15.0, d_th=0.05, theta_ccl_deg=15.0, min_cluster=50, n_hyp=100,
                eps=0.01, seed=0, classify=1, planes_per_cluster=1) -> Params:
    """Segmentation parameters (paper defaults: N_th=3, theta_th=15 deg, d_th=0.05 m,
    I=100, eps=0.01 m).  Cosines and d_th^2 are formed in double, then rounded to FP32."""
    import math
    return Params(n_th, np.float32(math.cos(math.radians(theta_step_deg))), np.float32(d_th * d_th),
                  np.float32(math.cos(math.radians(theta_ccl_deg))), min_cluster, n_hyp, np.float32(eps), seed,
                  classify, planes_per_cluster)


def _planes_to_dict(planes, n):
    out = {k: [] for k in ("label", "n_points", "inlier_count", "best_h", "ill_conditioned", "ransac_n",
                           "ransac_d", "refit_n", "refit_d", "basis_u", "basis_v", "origin", "hull_off",
                           "hull_n", "point_off", "round", "cond")}
    for i in range(n):
        p = planes[i]
        for k in out:
            v = getattr(p, k)
            out[k].append(list(v) if hasattr(v, "__len__") else v)
    dt = {"label": np.uint32, "n_points": np.uint32, "inlier_count": np.uint32, "best_h": np.int32,
          "ill_conditioned": np.int32, "ransac_n": np.float32, "ransac_d": np.float32, "refit_n": np.float64,
          "refit_d": np.float64, "basis_u": np.float32, "basis_v": np.float32, "origin": np.float32,
          "hull_off": np.uint32, "hull_n": np.uint32, "point_off": np.uint32, "round": np.uint32,
          "cond": np.float64}
    res = {}
    for k, v in out.items():
        a = np.array(v, dtype=dt[k])
        if a.ndim == 1 and k in ("ransac_n", "refit_n", "basis_u", "basis_v", "origin"):
            a = a.reshape(0, 3)
        res[k] = a
    return res


def _read_result(h):
    L = lib()
    sz = (C.c_uint32 * 3)()
    L.orc_result_sizes(h, sz)
    n_planes, n_hull, n_pts = sz[0], sz[1], sz[2]
    planes = _planes_to_dict(L.orc_result_planes(h), n_planes)
    hull = np.ctypeslib.as_array(L.orc_result_hull(h), shape=(n_hull, 2)).copy() if n_hull else np.zeros((0, 2), np.int32)
    pts = np.ctypeslib.as_array(L.orc_result_pts(h), shape=(n_pts, 3)).copy() if n_pts else np.zeros((0, 3), np.float32)
    inl = np.ctypeslib.as_array(L.orc_result_inlier(h), shape=(n_pts,)).copy() if n_pts else np.zeros(0, np.uint8)
    vid_ptr = L.orc_result_pt_vid(h)
    vid = np.ctypeslib.as_array(vid_ptr, shape=(n_pts,)).copy() if (n_pts and bool(vid_ptr)) else None
    return {"planes": planes, "hull": hull, "pts": pts, "inlier": inl, "pt_vid": vid}


class OracleMap:
    """Dense CPU voxel map over a ``dims`` grid at ``origin`` with voxel size 1/inv_res."""

    def __init__(self, dims, origin, voxel_size):
        self.dims = np.asarray(dims, np.int32)
        self.origin = np.asarray(origin, np.float32)
        self.inv_res = np.float32(1.0 / float(voxel_size))
        self._h = lib().orc_map_create(self.dims.ctypes.data_as(C.POINTER(C.c_int32)), _fp(self.origin),
                                       C.c_float(self.inv_res))
        if not self._h:
            raise MemoryError("oracle map allocation failed")

    def close(self):
        if self._h:
            lib().orc_map_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def integrate(self, xyz, pose=None):
        xyz = np.ascontiguousarray(xyz, np.float32).reshape(-1, 3)
        if pose is None:
            pose = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32)
        pose = np.ascontiguousarray(pose, np.float32).reshape(12)
        st = lib().orc_integrate(self._h, _fp(xyz), xyz.shape[0], _fp(pose))
        if st:
            raise RuntimeError(f"orc_integrate failed: {st}")

    def clear_rays(self, xyz, pose):
        """Eq. 2: clears every occupied voxel that a ray from the sensor (the
        pose's translation) to a point passes through before the point's own
        voxel; returns the number of voxels cleared."""
        xyz = np.ascontiguousarray(xyz, np.float32).reshape(-1, 3)
        pose = np.ascontiguousarray(pose, np.float32).reshape(12)
        k = C.c_uint64()
        st = lib().orc_clear_rays(self._h, _fp(xyz), xyz.shape[0], _fp(pose), C.byref(k))
        if st:
            raise RuntimeError(f"orc_clear_rays failed: {st}")
        return int(k.value)

    def counts(self):
        out = (C.c_uint64 * 2)()
        lib().orc_map_counts(self._h, out)
        return int(out[0]), int(out[1])

    def scroll(self, shift):
        """Moves the window by whole bricks (shift: 3 ints); voxels whose brick
        leaves it are evicted."""
        sh = np.ascontiguousarray(shift, np.int32).reshape(3)
        st = lib().orc_map_scroll(self._h, sh.ctypes.data_as(C.POINTER(C.c_int32)))
        if st:
            raise RuntimeError(f"orc_map_scroll failed: {st}")

    def scroll_target(self, center):
        """The brick shift that centres the window on center (map frame)."""
        c = np.ascontiguousarray(center, np.float32).reshape(3)
        sh = np.zeros(3, np.int32)
        lib().orc_scroll_target(self._h, _fp(c), sh.ctypes.data_as(C.POINTER(C.c_int32)))
        return sh

    def scroll_to(self, center):
        sh = self.scroll_target(center)
        if sh.any():
            self.scroll(sh)
        return sh

    def window(self):
        """Window offset w (voxels), sum anchor A (2^-20 m units), position
        origin (map frame) and the occupied voxels evicted so far."""
        w = np.zeros(3, np.int32)
        A = np.zeros(3, np.int64)
        po = np.zeros(3, np.float32)
        ev = C.c_uint64()
        lib().orc_map_window(self._h, w.ctypes.data_as(C.POINTER(C.c_int32)), A.ctypes.data_as(C.POINTER(C.c_int64)),
                             _fp(po), C.byref(ev))
        return {"offset": w, "anchor": A, "position_origin": po, "voxels_evicted": int(ev.value)}

    def export_sums(self):
        n = lib().orc_count_occupied(self._h)
        vid = np.zeros(n, np.uint32)
        S = np.zeros((n, 3), np.int64)
        c = np.zeros(n, np.uint32)
        if n:
            lib().orc_export_sums(self._h, _u32p(vid), S.ctypes.data_as(C.POINTER(C.c_int64)), _u32p(c))
        return vid, S, c

    def segment(self, params: Params):
        h = lib().orc_segment(self._h, C.byref(params))
        if not h:
            raise MemoryError("orc_segment failed")
        try:
            res = _read_result(h)
        finally:
            lib().orc_result_free(h)
        res["voxels"] = self.voxels()
        return res

    def voxels(self):
        """Per-occupied-voxel state of the last segmentation, in vid order."""
        n = lib().orc_map_n_vox(self._h)
        if n == 0:
            arr = np.zeros(0, dtype=np.dtype(Voxel))
        else:
            ptr = lib().orc_map_voxels(self._h)
            buf = (C.c_char * (n * C.sizeof(Voxel))).from_address(C.addressof(ptr.contents))
            arr = np.frombuffer(bytes(buf), dtype=_voxel_dtype())
        return {"vid": arr["vid"].copy(), "ijk": arr["ijk"].copy(), "S": arr["S"].copy(), "c": arr["c"].copy(),
                "M": arr["M"].copy(), "mu": arr["mu"].copy(), "n": arr["n"].copy(), "nbr": arr["nbr"].copy(),
                "status": arr["status"].copy(), "label": arr["label"].copy()}


def _voxel_dtype():
    return np.dtype({"names": ["vid", "ijk", "S", "c", "M", "mu", "n", "nbr", "status", "label"],
                     "formats": [np.uint32, (np.int32, 3), (np.int64, 3), np.uint32, (np.int32, 3),
                                 (np.float32, 3), (np.float32, 3), np.uint32, np.uint32, np.uint32],
                     "offsets": [getattr(Voxel, f).offset for f in
                                 ["vid", "ijk", "S", "c", "M", "mu", "n", "nbr", "status", "label"]],
                     "itemsize": C.sizeof(Voxel)})


def fit_planes(xyz, cl_off, params: Params, labels=None):
    """Sec. III.C stages a-c plus refit and hull on caller-formed clusters."""
    xyz = np.ascontiguousarray(xyz, np.float32).reshape(-1, 3)
    off = np.ascontiguousarray(cl_off, np.uint32)
    k = off.shape[0] - 1
    lab = None if labels is None else np.ascontiguousarray(labels, np.uint32)
    h = lib().orc_fit_planes(_fp(xyz), _u32p(off), _u32p(lab) if lab is not None else None, k, C.byref(params))
    if not h:
        raise MemoryError("orc_fit_planes failed")
    try:
        return _read_result(h)
    finally:
        lib().orc_result_free(h)


def jacobi3_f32(a6, sweeps=6):
    """FP32 cyclic Jacobi on {a00,a11,a22,a01,a02,a12}: (normal, diagonal, V)."""
    a = np.ascontiguousarray(a6, np.float32).reshape(6)
    n = np.zeros(3, np.float32)
    d = np.zeros(3, np.float32)
    v = np.zeros(9, np.float32)
    lib().orc_jacobi3_f32(_fp(a), sweeps, _fp(n), _fp(d), _fp(v))
    return n, d, v.reshape(3, 3)


def philox4x64(ctr, key):
    c = np.ascontiguousarray(ctr, np.uint64).reshape(4)
    k = np.ascontiguousarray(key, np.uint64).reshape(2)
    o = np.zeros(4, np.uint64)
    p = lambda a: a.ctypes.data_as(C.POINTER(C.c_uint64))
    lib().orc_philox4x64(p(c), p(k), p(o))
    return o


def ransac_counts(pts, label, n_hyp, seed, eps):
    """Per-hypothesis inlier counts (-1: degenerate sample), planes (n, d) and the selected h."""
    pts = np.ascontiguousarray(pts, np.float32).reshape(-1, 3)
    counts = np.zeros(n_hyp, np.int64)
    planes = np.zeros((n_hyp, 4), np.float32)
    best = lib().orc_ransac_counts(_fp(pts), pts.shape[0], label, n_hyp, seed, C.c_float(np.float32(eps)),
                                   counts.ctypes.data_as(C.POINTER(C.c_int64)), _fp(planes))
    return counts, planes, int(best)


def hull_i32(xy):
    """Monotone-chain hull of integer points: CCW from the lexicographic minimum."""
    xy = np.array(xy, np.int32).reshape(-1, 2).copy()
    out = np.zeros((xy.shape[0] + 1, 2), np.int32)
    k = lib().orc_hull_i32(xy.ctypes.data_as(C.POINTER(C.c_int32)), xy.shape[0],
                           out.ctypes.data_as(C.POINTER(C.c_int32)))
    return out[:k].copy()
