"""ctypes binding of libvoxmps.so (include/vm.h).

Argument marshalling only: every step of integration and segmentation runs in
the library's CUDA kernels.  There is no CPU fallback -- if the library is not
built or cannot load, every call raises.

The low-level functions carry the C names (``vm_create``, ``vm_integrate``,
``vm_segment``, ``vm_fit_planes`` ...).  ``VoxelMap`` wraps a map handle;
torch is used only for device memory and streams.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

VM_MAP_STAGE_TIMING = 1
VM_MAP_EAGER = 2
N_STAGES = 16  # upper bound of the library's stage count

VM_OK, VM_ERR_INVALID_ARG, VM_ERR_OUT_OF_MEMORY, VM_ERR_CAPACITY, VM_ERR_CUDA, VM_ERR_TIMEOUT, VM_ERR_EXTENT = range(7)
STATUS_NAMES = {0: "VM_OK", 1: "VM_ERR_INVALID_ARG", 2: "VM_ERR_OUT_OF_MEMORY", 3: "VM_ERR_CAPACITY",
                4: "VM_ERR_CUDA", 5: "VM_ERR_TIMEOUT", 6: "VM_ERR_EXTENT"}


class VmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class vm_map_params(C.Structure):
    _fields_ = [("origin", C.c_float * 3), ("dims", C.c_int32 * 3), ("voxel_size", C.c_float),
                ("brick_capacity", C.c_uint32), ("flags", C.c_uint32)]


class vm_segment_params(C.Structure):
    _fields_ = [("n_th", C.c_uint32), ("cos_step", C.c_float), ("d_th2", C.c_float), ("cos_ccl", C.c_float),
                ("min_cluster", C.c_uint32), ("n_hyp", C.c_uint32), ("eps", C.c_float), ("seed", C.c_uint64),
                ("classify", C.c_uint32), ("planes_per_cluster", C.c_uint32)]


class vm_plane(C.Structure):
    _fields_ = [("normal", C.c_float * 3), ("offset", C.c_float), ("inlier_count", C.c_uint32),
                ("label", C.c_uint32), ("ransac_normal", C.c_float * 3), ("ransac_offset", C.c_float),
                ("basis_u", C.c_float * 3), ("basis_v", C.c_float * 3), ("hull_origin", C.c_float * 3),
                ("hull_offset", C.c_uint32), ("hull_count", C.c_uint32), ("n_points", C.c_uint32),
                ("best_h", C.c_int32), ("flags", C.c_uint32)]


class vm_planes(C.Structure):
    _fields_ = [("planes", C.POINTER(vm_plane)), ("n_planes", C.c_uint32), ("hull_xy", C.POINTER(C.c_int32)),
                ("hull_xyz", C.POINTER(C.c_float)), ("n_hull", C.c_uint32)]


class vm_stats(C.Structure):
    _fields_ = [("points_integrated", C.c_uint64), ("points_dropped", C.c_uint64),
                ("points_no_capacity", C.c_uint64), ("bricks_allocated", C.c_uint32),
                ("brick_capacity", C.c_uint32), ("occupied_voxels", C.c_uint32), ("steppable_voxels", C.c_uint32),
                ("clusters", C.c_uint32), ("clustered_points", C.c_uint32), ("device_bytes", C.c_uint64),
                ("voxels_cleared", C.c_uint64), ("voxels_evicted", C.c_uint64)]


class vm_fit_tuning(C.Structure):
    _fields_ = [("tile", C.c_uint32), ("hyp_per_thread", C.c_uint32), ("ctas_per_sm", C.c_uint32),
                ("schedule", C.c_uint32)]


class vm_server_params(C.Structure):
    _fields_ = [("mode", C.c_uint32), ("max_batch", C.c_uint32), ("max_inflight", C.c_uint32),
                ("device", C.c_uint32), ("hbm_budget", C.c_uint64), ("hbm_reserve", C.c_uint64),
                ("params", vm_segment_params), ("tuning", vm_fit_tuning)]


class vm_server_result(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("stream", C.c_uint32), ("status", C.c_int), ("planes", vm_planes),
                ("t_arrival", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double)]


class vm_server_stats(C.Structure):
    _fields_ = [("streams_open", C.c_uint32), ("streams_admitted", C.c_uint32), ("streams_waiting", C.c_uint32),
                ("reserved", C.c_uint32), ("requests_submitted", C.c_uint64), ("requests_done", C.c_uint64),
                ("steps", C.c_uint64), ("fallbacks", C.c_uint64), ("hbm_budget", C.c_uint64),
                ("hbm_committed", C.c_uint64), ("mean_step_requests", C.c_double), ("launch_seconds", C.c_double),
                ("complete_seconds", C.c_double), ("graph_captures", C.c_uint64), ("allocations", C.c_uint64)]


# name -> (restype, argtypes); every name is declared in include/vm.h
_SIGS = {
    "vm_create": (C.c_int, [C.POINTER(vm_map_params), C.c_void_p, C.POINTER(C.c_void_p)]),
    "vm_integrate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint32, C.POINTER(C.c_float), C.c_int]),
    "vm_integrate_ex": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint32, C.POINTER(C.c_float), C.c_int, C.c_uint32]),
    "vm_segment": (C.c_int, [C.c_void_p, C.POINTER(vm_segment_params), C.POINTER(vm_planes)]),
    "vm_planes_free": (C.c_int, [C.POINTER(vm_planes)]),
    "vm_reset": (C.c_int, [C.c_void_p]),
    "vm_scroll": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "vm_scroll_target": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_int32)]),
    "vm_scroll_to": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_int32)]),
    "vm_get_window": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_float)]),
    "vm_destroy": (C.c_int, [C.c_void_p]),
    "vm_get_stats": (C.c_int, [C.c_void_p, C.POINTER(vm_stats)]),
    "vm_fit_planes": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, C.POINTER(vm_segment_params),
                                C.c_void_p, C.POINTER(vm_planes)]),
    "vm_export_voxels": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32,
                                   C.POINTER(C.c_uint32)]),
    "vm_export_labels": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_uint32, C.POINTER(C.c_uint32)]),
    "vm_export_clusters": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32,
                                     C.POINTER(C.c_uint32)]),
    "vm_fit_plan_create": (C.c_int, [C.c_uint32, C.c_uint32, C.POINTER(vm_segment_params), C.c_void_p, C.c_uint32,
                                     C.POINTER(C.c_void_p)]),
    "vm_fit_plan_run": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32,
                                  C.POINTER(vm_planes)]),
    "vm_fit_plan_launch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32]),
    "vm_fit_plan_wait": (C.c_int, [C.c_void_p, C.POINTER(vm_planes)]),
    "vm_fit_plan_set_tuning": (C.c_int, [C.c_void_p, C.POINTER(vm_fit_tuning)]),
    "vm_fit_plan_get_tuning": (C.c_int, [C.c_void_p, C.POINTER(vm_fit_tuning)]),
    "vm_fit_plan_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, C.c_uint32,
                                       C.POINTER(vm_fit_tuning), C.POINTER(C.c_float), C.POINTER(C.c_uint32)]),
    "vm_fit_plan_stage_times": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, C.POINTER(C.c_uint32)]),
    "vm_fit_plan_destroy": (C.c_int, [C.c_void_p]),
    "vm_server_create": (C.c_int, [C.POINTER(vm_server_params), C.POINTER(C.c_void_p)]),
    "vm_server_open": (C.c_int, [C.c_void_p, C.POINTER(vm_map_params), C.POINTER(C.c_uint32)]),
    "vm_server_submit": (C.c_int, [C.c_void_p, C.c_uint32, C.c_void_p, C.c_uint32, C.POINTER(C.c_float), C.c_int,
                                   C.c_double, C.POINTER(C.c_uint64)]),
    "vm_server_poll": (C.c_int, [C.c_void_p, C.POINTER(vm_server_result), C.c_uint32, C.POINTER(C.c_uint32),
                                 C.c_int]),
    "vm_server_drain": (C.c_int, [C.c_void_p, C.c_int]),
    "vm_server_close": (C.c_int, [C.c_void_p, C.c_uint32]),
    "vm_server_get_stats": (C.c_int, [C.c_void_p, C.POINTER(vm_server_stats)]),
    "vm_server_footprint": (C.c_uint64, [C.POINTER(vm_map_params), C.POINTER(vm_segment_params)]),
    "vm_server_now": (C.c_double, [C.c_void_p]),
    "vm_server_destroy": (C.c_int, [C.c_void_p]),
    "vm_set_fit_tuning": (C.c_int, [C.c_void_p, C.POINTER(vm_fit_tuning)]),
    "vm_get_fit_tuning": (C.c_int, [C.c_void_p, C.POINTER(vm_fit_tuning)]),
    "vm_autotune_segment": (C.c_int, [C.c_void_p, C.POINTER(vm_segment_params), C.c_uint32,
                                      C.POINTER(vm_fit_tuning), C.POINTER(C.c_float), C.POINTER(C.c_uint32)]),
    "vm_stage_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "vm_stage_times": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, C.POINTER(C.c_uint32)]),
    "vm_stage_name": (C.c_char_p, [C.c_uint32]),
    "vm_launch_count": (C.c_uint64, []),
    "vm_graph_shape": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]),
    "vm_capture_count": (C.c_uint64, []),
    "vm_allocation_count": (C.c_uint64, []),
    "vm_last_error": (C.c_char_p, []),
    "vm_version": (C.c_char_p, []),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libvoxmps.so (building it first if needed).  Raises if it cannot."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libvoxmps.so is missing at {path}; run paper_2510_01592_gb300.build.build()")
            L = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(st):
    if st != VM_OK:
        raise VmError(st, load().vm_last_error().decode(errors="replace"))


def segment_params(n_th=3, theta_step_deg=15.0, d_th=0.05, theta_ccl_deg=15.0, min_cluster=50, n_hyp=100, eps=0.01,
                   seed=0, classify=1, planes_per_cluster=1) -> vm_segment_params:
    """Paper defaults (Sec. III.C, Sec. IV-A); cosines and d_th^2 in double, then FP32."""
    return vm_segment_params(n_th, np.float32(math.cos(math.radians(theta_step_deg))), np.float32(d_th * d_th),
                             np.float32(math.cos(math.radians(theta_ccl_deg))), min_cluster, n_hyp,
                             np.float32(eps), seed, classify, planes_per_cluster)


def _planes_to_numpy(out: vm_planes):
    n = out.n_planes
    dt = np.dtype([("normal", np.float32, 3), ("offset", np.float32), ("inlier_count", np.uint32),
                   ("label", np.uint32), ("ransac_normal", np.float32, 3), ("ransac_offset", np.float32),
                   ("basis_u", np.float32, 3), ("basis_v", np.float32, 3), ("hull_origin", np.float32, 3),
                   ("hull_offset", np.uint32), ("hull_count", np.uint32), ("n_points", np.uint32),
                   ("best_h", np.int32), ("flags", np.uint32)])
    assert dt.itemsize == C.sizeof(vm_plane)
    if n:
        raw = C.string_at(out.planes, n * C.sizeof(vm_plane))
        planes = np.frombuffer(raw, dtype=dt).copy()
    else:
        planes = np.zeros(0, dtype=dt)
    nh = out.n_hull
    hull_xy = np.ctypeslib.as_array(out.hull_xy, shape=(nh, 2)).copy() if nh else np.zeros((0, 2), np.int32)
    hull_xyz = np.ctypeslib.as_array(out.hull_xyz, shape=(nh, 3)).copy() if nh else np.zeros((0, 3), np.float32)
    return {"planes": planes, "hull_xy": hull_xy, "hull_xyz": hull_xyz}


def _ptr(x):
    """Device or host data pointer of a torch tensor / numpy array (or None)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    return C.c_void_p(x.ctypes.data)


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def order_after_torch(xyz, stream=None):
    """Makes work on `stream` (a torch stream the library will use, or None for
    a stream the library owns) start after the kernels torch has queued to
    produce the CUDA tensor xyz: a device-side wait when the stream is a torch
    stream, else the producing stream is synchronised."""
    if not (hasattr(xyz, "is_cuda") and xyz.is_cuda):
        return
    import torch
    cur = torch.cuda.current_stream(xyz.device)
    if isinstance(stream, torch.cuda.Stream):
        if stream != cur:
            stream.wait_stream(cur)
    else:
        cur.synchronize()


class VoxelMap:
    """A device-resident voxel map (Sec. III.B) with multi-plane segmentation (Sec. III.C)."""

    def __init__(self, dims, origin, voxel_size, brick_capacity=0, stream=None, stage_timing=False, eager=False):
        """eager: launch the segmentation kernel by kernel instead of replaying a
        captured CUDA graph (stage timing implies eager launches)."""
        L = load()
        flags = (VM_MAP_STAGE_TIMING if stage_timing else 0) | (VM_MAP_EAGER if eager else 0)
        p = vm_map_params((C.c_float * 3)(*[float(o) for o in origin]), (C.c_int32 * 3)(*[int(d) for d in dims]),
                          float(voxel_size), int(brick_capacity), flags)
        h = C.c_void_p()
        self._stream = stream
        _check(L.vm_create(C.byref(p), _stream_handle(stream), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().vm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def integrate(self, xyz, pose, clear=False):
        """xyz: float32 [n, 3] torch tensor (CUDA or CPU) or numpy array; pose: 12 floats, sensor->map.
        clear: first clear the voxels the points' rays pass through (Eq. 2)."""
        pose = np.ascontiguousarray(pose, np.float32).reshape(12)
        on_dev = 1 if (hasattr(xyz, "is_cuda") and xyz.is_cuda) else 0
        if hasattr(xyz, "is_contiguous"):
            assert xyz.dtype.is_floating_point and xyz.element_size() == 4 and xyz.is_contiguous()
            n = xyz.numel() // 3
        else:
            xyz = np.ascontiguousarray(xyz, np.float32)
            n = xyz.size // 3
        order_after_torch(xyz, self._stream)
        _check(load().vm_integrate_ex(self._h, _ptr(xyz), n, pose.ctypes.data_as(C.POINTER(C.c_float)), on_dev,
                                      VM_INTEGRATE_CLEAR if clear else 0))

    def segment(self, params: vm_segment_params | None = None):
        params = params or segment_params()
        out = vm_planes()
        st = load().vm_segment(self._h, C.byref(params), C.byref(out))
        try:
            if st not in (VM_OK, VM_ERR_CAPACITY):
                _check(st)
            res = _planes_to_numpy(out)
            res["status"] = st
        finally:
            load().vm_planes_free(C.byref(out))
        return res

    @property
    def fit_tuning(self):
        t = vm_fit_tuning()
        _check(load().vm_get_fit_tuning(self._h, C.byref(t)))
        return _tuning_dict(t)

    def set_fit_tuning(self, tuning: dict | None):
        """Fit schedule of this map's segmentations (results do not depend on it); None: the default."""
        if tuning is None:
            _check(load().vm_set_fit_tuning(self._h, None))
            return
        t = vm_fit_tuning(int(tuning["tile"]), int(tuning["hyp_per_thread"]), int(tuning["ctas_per_sm"]),
                          1 if tuning.get("schedule") == "warp" else 0)
        _check(load().vm_set_fit_tuning(self._h, C.byref(t)))

    def autotune(self, params: vm_segment_params | None = None, reps: int = 3):
        """Times the segmentation of the map as it stands under each candidate
        schedule and keeps the fastest; returns (tuning dict, ms, candidates)."""
        params = params or segment_params()
        t, ms, n = vm_fit_tuning(), C.c_float(), C.c_uint32()
        _check(load().vm_autotune_segment(self._h, C.byref(params), int(reps), C.byref(t), C.byref(ms),
                                          C.byref(n)))
        return _tuning_dict(t), float(ms.value), int(n.value)

    def reset(self):
        _check(load().vm_reset(self._h))

    def scroll(self, shift):
        """Moves the window by whole bricks (3 ints); voxels whose brick leaves
        it are evicted."""
        sh = (C.c_int32 * 3)(*[int(v) for v in np.asarray(shift).reshape(3)])
        _check(load().vm_scroll(self._h, sh))

    def scroll_target(self, center):
        """The brick shift that centres the window on center (map frame)."""
        c = (C.c_float * 3)(*[float(v) for v in np.asarray(center, np.float32).reshape(3)])
        sh = (C.c_int32 * 3)()
        _check(load().vm_scroll_target(self._h, c, sh))
        return np.array(sh[:], np.int32)

    def scroll_to(self, center):
        """Centres the window on center (map frame); returns the brick shift."""
        c = (C.c_float * 3)(*[float(v) for v in np.asarray(center, np.float32).reshape(3)])
        sh = (C.c_int32 * 3)()
        _check(load().vm_scroll_to(self._h, c, sh))
        return np.array(sh[:], np.int32)

    def window(self):
        """Window offset (voxels) and position origin (map frame)."""
        w = (C.c_int32 * 3)()
        po = (C.c_float * 3)()
        _check(load().vm_get_window(self._h, w, po))
        return {"offset": np.array(w[:], np.int32), "position_origin": np.array(po[:], np.float32)}

    def stats(self):
        s = vm_stats()
        st = load().vm_get_stats(self._h, C.byref(s))
        if st not in (VM_OK, VM_ERR_CAPACITY):
            _check(st)
        return {f: getattr(s, f) for f, _ in vm_stats._fields_} | {"status": st}

    def graph_shape(self):
        """Nodes, edges and programmatic edges of the captured segmentation graph."""
        n, e, p = C.c_uint32(), C.c_uint32(), C.c_uint32()
        _check(load().vm_graph_shape(self._h, C.byref(n), C.byref(e), C.byref(p)))
        return {"nodes": n.value, "edges": e.value, "programmatic": p.value}

    def stage_times(self):
        """{stage: (ms, calls)} accumulated since the previous call."""
        return stage_times(self._h)

    def export_voxels(self):
        L = load()
        n = C.c_uint32()
        _check(L.vm_export_voxels(self._h, None, None, None, 0, C.byref(n)))
        k = n.value
        vid = np.zeros(k, np.uint32)
        S = np.zeros((k, 3), np.int64)
        c = np.zeros(k, np.uint32)
        _check(L.vm_export_voxels(self._h, _ptr(vid), _ptr(S), _ptr(c), k, C.byref(n)))
        return vid, S, c

    def export_labels(self):
        L = load()
        n = C.c_uint32()
        _check(L.vm_export_labels(self._h, None, None, None, None, None, 0, C.byref(n)))
        k = n.value
        vid = np.zeros(k, np.uint32)
        nrm = np.zeros((k, 3), np.float32)
        st = np.zeros(k, np.uint8)
        lab = np.zeros(k, np.uint32)
        nbr = np.zeros(k, np.uint32)
        _check(L.vm_export_labels(self._h, _ptr(vid), _ptr(nrm), _ptr(st), _ptr(lab), _ptr(nbr), k, C.byref(n)))
        return {"vid": vid, "n": nrm, "status": st, "label": lab, "nbr": nbr}

    def export_clusters(self):
        L = load()
        n = C.c_uint32()
        _check(L.vm_export_clusters(self._h, None, None, None, 0, C.byref(n)))
        k = n.value
        pts = np.zeros((k, 3), np.float32)
        vid = np.zeros(k, np.uint32)
        inl = np.zeros(k, np.uint8)
        _check(L.vm_export_clusters(self._h, _ptr(pts), _ptr(vid), _ptr(inl), k, C.byref(n)))
        return {"pts": pts, "pt_vid": vid, "inlier": inl}


def fit_planes(xyz, off, params: vm_segment_params | None = None, labels=None, stream=None):
    """Batched RANSAC + refit + hull on caller clusters; xyz, off, labels are CUDA tensors."""
    params = params or segment_params()
    k = int(off.numel()) - 1
    out = vm_planes()
    _check(load().vm_fit_planes(_ptr(xyz), _ptr(off), _ptr(labels), k, C.byref(params), _stream_handle(stream),
                                C.byref(out)))
    try:
        return _planes_to_numpy(out)
    finally:
        load().vm_planes_free(C.byref(out))


VM_INTEGRATE_CLEAR = 1
VM_FIT_STAGE_TIMING = 1
VM_FIT_EAGER = 2


def _tuning_dict(t: vm_fit_tuning):
    return {"tile": t.tile, "hyp_per_thread": t.hyp_per_thread, "ctas_per_sm": t.ctas_per_sm,
            "schedule": "warp" if t.schedule else "cta"}


class FitPlan:
    """A reusable batched fit (vm_fit_plan_*): buffers sized once, the whole fit
    replayed as one CUDA graph per run.  xyz, off, labels are CUDA tensors."""

    def __init__(self, k_cap, n_cap, params: vm_segment_params | None = None, stream=None, eager=False,
                 stage_timing=False):
        self.params = params or segment_params()
        h = C.c_void_p()
        flags = (VM_FIT_EAGER if eager else 0) | (VM_FIT_STAGE_TIMING if stage_timing else 0)
        _check(load().vm_fit_plan_create(int(k_cap), int(n_cap), C.byref(self.params), _stream_handle(stream),
                                         flags, C.byref(h)))
        self._h = h

    def stage_times(self):
        """{stage: (ms, calls)} since the previous call (plans made with stage_timing=True)."""
        ms = (C.c_double * N_STAGES)()
        calls = (C.c_uint64 * N_STAGES)()
        n = C.c_uint32()
        _check(load().vm_fit_plan_stage_times(self._h, ms, calls, N_STAGES, C.byref(n)))
        L = load()
        return {L.vm_stage_name(i).decode(): (ms[i], calls[i]) for i in range(n.value) if calls[i]}

    def close(self):
        if getattr(self, "_h", None):
            load().vm_fit_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, xyz, off, labels=None):
        k = int(off.numel()) - 1
        out = vm_planes()
        _check(load().vm_fit_plan_run(self._h, _ptr(xyz), _ptr(off), _ptr(labels), k, C.byref(out)))
        try:
            return _planes_to_numpy(out)
        finally:
            load().vm_planes_free(C.byref(out))

    def launch(self, xyz, off, labels=None):
        _check(load().vm_fit_plan_launch(self._h, _ptr(xyz), _ptr(off), _ptr(labels), int(off.numel()) - 1))

    def wait(self):
        _check(load().vm_fit_plan_wait(self._h, None))

    @property
    def tuning(self):
        t = vm_fit_tuning()
        _check(load().vm_fit_plan_get_tuning(self._h, C.byref(t)))
        return _tuning_dict(t)

    def set_tuning(self, tile, hyp_per_thread, ctas_per_sm, schedule="cta"):
        t = vm_fit_tuning(int(tile), int(hyp_per_thread), int(ctas_per_sm), 1 if schedule == "warp" else 0)
        _check(load().vm_fit_plan_set_tuning(self._h, C.byref(t)))

    def autotune(self, xyz, off, labels=None, reps=2):
        """Times every candidate schedule on this batch and keeps the fastest;
        returns (tuning dict, ms per fit, candidates timed)."""
        t, ms, n = vm_fit_tuning(), C.c_float(), C.c_uint32()
        _check(load().vm_fit_plan_autotune(self._h, _ptr(xyz), _ptr(off), _ptr(labels), int(off.numel()) - 1,
                                           int(reps), C.byref(t), C.byref(ms), C.byref(n)))
        return _tuning_dict(t), float(ms.value), int(n.value)


def stage_times(handle=None):
    L = load()
    ms = (C.c_double * N_STAGES)()
    calls = (C.c_uint64 * N_STAGES)()
    n = C.c_uint32()
    _check(L.vm_stage_times(handle, ms, calls, N_STAGES, C.byref(n)))
    return {L.vm_stage_name(i).decode(): (ms[i], int(calls[i])) for i in range(min(n.value, N_STAGES))}


def set_fit_stage_timing(enable: bool):
    """Stage timing of this thread's fit_planes calls."""
    _check(load().vm_stage_timing(None, 1 if enable else 0))


def launch_count() -> int:
    return int(load().vm_launch_count())


def capture_count() -> int:
    return int(load().vm_capture_count())


def allocation_count() -> int:
    return int(load().vm_allocation_count())


# C-ABI names re-exported for callers who want the raw entry points.
def __getattr__(name):
    if name in _SIGS:
        return getattr(load(), name)
    raise AttributeError(name)
