"""Python binding of the multi-stream server (vm_server_* in include/vm.h).

Argument marshalling only: the scheduler, admission, continuous batching and
every kernel live in libvoxmps.so.  Point buffers handed to ``submit`` are kept
alive here until their result has been polled.
"""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np

from . import vm

BATCHED = 0
STREAMS = 1


def _map_params(dims, origin, voxel_size, brick_capacity=0):
    return vm.vm_map_params((C.c_float * 3)(*[float(o) for o in origin]), (C.c_int32 * 3)(*[int(d) for d in dims]),
                            float(voxel_size), int(brick_capacity), 0)


def footprint(dims, origin, voxel_size, brick_capacity=0, params: vm.vm_segment_params | None = None) -> int:
    """Device bytes a stream with this map would reserve on admission."""
    params = params or vm.segment_params()
    return int(vm.load().vm_server_footprint(C.byref(_map_params(dims, origin, voxel_size, brick_capacity)),
                                             C.byref(params)))


class Server:
    """Many sensor streams, one device-resident map each; requests (integrate a
    frame + segment) are scheduled by the library's own thread."""

    def __init__(self, params: vm.vm_segment_params | None = None, mode: str = "batched", max_batch: int = 16,
                 max_inflight: int = 2, device: int = 0, hbm_budget: int = 0, hbm_reserve: int = 4 << 30,
                 tuning: dict | None = None):
        self.params = params or vm.segment_params()
        t = vm.vm_fit_tuning()
        if tuning:
            t = vm.vm_fit_tuning(int(tuning["tile"]), int(tuning["hyp_per_thread"]), int(tuning["ctas_per_sm"]),
                                 1 if tuning.get("schedule") == "warp" else 0)
        sp = vm.vm_server_params(BATCHED if mode == "batched" else STREAMS, int(max_batch), int(max_inflight),
                                 int(device), int(hbm_budget), int(hbm_reserve), self.params, t)
        h = C.c_void_p()
        vm._check(vm.load().vm_server_create(C.byref(sp), C.byref(h)))
        self._h = h
        self._keep = {}
        self._lock = threading.Lock()

    def close(self):
        if getattr(self, "_h", None):
            vm.load().vm_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def open(self, dims, origin, voxel_size, brick_capacity=0) -> int:
        sid = C.c_uint32()
        vm._check(vm.load().vm_server_open(self._h, C.byref(_map_params(dims, origin, voxel_size, brick_capacity)),
                                           C.byref(sid)))
        return int(sid.value)

    def close_stream(self, sid: int):
        vm._check(vm.load().vm_server_close(self._h, int(sid)))

    def now(self) -> float:
        return float(vm.load().vm_server_now(self._h))

    def submit(self, sid: int, xyz, pose, t_arrival: float = -1.0) -> int:
        """xyz: CUDA tensor or host array float32[n, 3] (kept alive until polled;
        a CUDA tensor's producing torch stream is synchronised first); pose: 12
        floats, sensor->map row-major [R|t]."""
        on_dev = hasattr(xyz, "is_cuda") and xyz.is_cuda
        vm.order_after_torch(xyz)  # the server's streams are its own
        if not on_dev:
            xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.float32))
        n = int(xyz.shape[0])
        pz = (C.c_float * 12)(*[float(v) for v in np.asarray(pose, dtype=np.float32).reshape(12)])
        t = C.c_uint64()
        vm._check(vm.load().vm_server_submit(self._h, int(sid), vm._ptr(xyz), n, pz, 1 if on_dev else 0,
                                             float(t_arrival), C.byref(t)))
        with self._lock:
            self._keep[int(t.value)] = xyz
        return int(t.value)

    def poll(self, max_results: int = 64, timeout_ms: int = 0, with_planes: bool = True):
        """Finished requests: list of dicts (ticket, stream, status, t_arrival,
        t_start, t_done, and the planes as VoxelMap.segment returns them)."""
        buf = (vm.vm_server_result * max_results)()
        n = C.c_uint32()
        vm._check(vm.load().vm_server_poll(self._h, buf, max_results, C.byref(n), int(timeout_ms)))
        out = []
        for i in range(n.value):
            r = buf[i]
            d = {"ticket": int(r.ticket), "stream": int(r.stream), "status": int(r.status),
                 "t_arrival": r.t_arrival, "t_start": r.t_start, "t_done": r.t_done}
            if r.status == vm.VM_OK and with_planes:
                d.update(vm._planes_to_numpy(r.planes))
            vm.load().vm_planes_free(C.byref(r.planes))
            with self._lock:
                self._keep.pop(d["ticket"], None)
            out.append(d)
        return out

    def drain(self, timeout_ms: int = -1):
        vm._check(vm.load().vm_server_drain(self._h, int(timeout_ms)))

    def stats(self) -> dict:
        s = vm.vm_server_stats()
        vm._check(vm.load().vm_server_get_stats(self._h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in vm.vm_server_stats._fields_ if f != "reserved"}
