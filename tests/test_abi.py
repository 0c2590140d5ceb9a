"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/vm.h declares; without a GPU its calls fail with a status (no crash,
no CPU fallback).  The Python binding's structs match the header's sizes."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("vm_create", "vm_integrate", "vm_segment", "vm_destroy", "vm_fit_planes", "vm_planes_free",
              "vm_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2510_01592_gb300 import vm
    L = vm.load()
    for n in _declared():
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", vm.lib_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (vm_[a-z_0-9]+)\b", out))
    assert set(_declared()) <= exported
    assert L.vm_version().startswith(b"voxmps")


def test_binding_struct_sizes_match_header():
    """Compile a probe against include/vm.h with the host compiler and compare sizeof."""
    from paper_2510_01592_gb300 import vm
    probe = r'''
#include <stdio.h>
#include <stddef.h>
#include "vm.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(vm_map_params), sizeof(vm_segment_params),
         sizeof(vm_plane), sizeof(vm_planes), sizeof(vm_stats), offsetof(vm_plane, hull_offset),
         offsetof(vm_segment_params, seed), sizeof(vm_fit_tuning), sizeof(vm_server_params),
         offsetof(vm_server_params, tuning), sizeof(vm_server_result), sizeof(vm_server_stats));
  return 0;
}
'''
    d = os.path.join(ROOT, "paper_2510_01592_gb300", "_build")
    os.makedirs(d, exist_ok=True)
    src = os.path.join(d, "abi_probe.c")
    exe = os.path.join(d, "abi_probe")
    open(src, "w").write(probe)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
    got = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    want = [C.sizeof(vm.vm_map_params), C.sizeof(vm.vm_segment_params), C.sizeof(vm.vm_plane),
            C.sizeof(vm.vm_planes), C.sizeof(vm.vm_stats), vm.vm_plane.hull_offset.offset,
            vm.vm_segment_params.seed.offset, C.sizeof(vm.vm_fit_tuning), C.sizeof(vm.vm_server_params),
            vm.vm_server_params.tuning.offset, C.sizeof(vm.vm_server_result), C.sizeof(vm.vm_server_stats)]
    assert got == want


def test_calls_fail_with_a_status_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2510_01592_gb300 import vm
    with pytest.raises(vm.VmError) as ei:
        vm.VoxelMap((8, 8, 8), (0, 0, 0), 0.05)
    assert ei.value.status in (vm.VM_ERR_CUDA, vm.VM_ERR_OUT_OF_MEMORY)


def test_invalid_arguments_rejected_before_any_device_work():
    from paper_2510_01592_gb300 import vm
    L = vm.load()
    h = C.c_void_p()
    bad = vm.vm_map_params((C.c_float * 3)(0, 0, 0), (C.c_int32 * 3)(0, 8, 8), 0.05, 0, 0)
    assert L.vm_create(C.byref(bad), None, C.byref(h)) == vm.VM_ERR_INVALID_ARG
    huge = vm.vm_map_params((C.c_float * 3)(0, 0, 0), (C.c_int32 * 3)(2000, 8, 8), 0.01, 0, 0)
    assert L.vm_create(C.byref(huge), None, C.byref(h)) == vm.VM_ERR_INVALID_ARG  # 20 m > 16 m
    assert L.vm_segment(None, None, None) == vm.VM_ERR_INVALID_ARG
    p = vm.segment_params(n_hyp=0)
    out = vm.vm_planes()
    assert L.vm_fit_planes(None, None, None, 1, C.byref(p), None, C.byref(out)) == vm.VM_ERR_INVALID_ARG
    assert b"n_hyp" in L.vm_last_error()


def test_server_footprint_is_host_arithmetic():
    """vm_server_footprint needs no GPU: it grows with the brick capacity and the
    resolution, and a capacity above the grid's brick count changes nothing."""
    from paper_2510_01592_gb300 import serve
    small = serve.footprint((200, 200, 100), (0, 0, 0), 0.02, brick_capacity=1000)
    big = serve.footprint((200, 200, 100), (0, 0, 0), 0.02, brick_capacity=4000)
    fine = serve.footprint((400, 400, 200), (0, 0, 0), 0.01, brick_capacity=4000)
    assert 0 < small < big < fine
    n_bricks = 25 * 25 * 13
    assert serve.footprint((200, 200, 100), (0, 0, 0), 0.02, brick_capacity=0) == \
        serve.footprint((200, 200, 100), (0, 0, 0), 0.02, brick_capacity=10 * n_bricks)
    assert big - small > 3000 * 512 * 28  # at least the pool's sums and counts per brick


def test_parameter_and_handle_checks_need_no_gpu():
    """Segment parameters are validated on the host by every entry point that
    takes them (n_hyp range, non-negative eps, at most 8 planes a cluster, one
    round outside vm_segment), and a null map is refused by the window calls."""
    from paper_2510_01592_gb300 import vm
    L = vm.load()
    out = vm.vm_planes()
    h = C.c_void_p()
    cases = [(dict(n_hyp=2000), b"n_hyp"), (dict(eps=float("nan")), b"eps"), (dict(eps=-0.01), b"eps"),
             (dict(planes_per_cluster=9), b"at most 8"), (dict(planes_per_cluster=2), b"vm_segment only")]
    for kw, msg in cases:
        p = vm.segment_params(**kw)
        assert L.vm_fit_planes(None, None, None, 1, C.byref(p), None, C.byref(out)) == vm.VM_ERR_INVALID_ARG
        assert msg in L.vm_last_error()
        assert L.vm_fit_plan_create(10, 100, C.byref(p), None, 0, C.byref(h)) == vm.VM_ERR_INVALID_ARG
        assert msg in L.vm_last_error()
    sh, ctr = (C.c_int32 * 3)(1, 0, 0), (C.c_float * 3)(0, 0, 0)
    assert L.vm_scroll(None, sh) == vm.VM_ERR_INVALID_ARG
    assert L.vm_scroll_to(None, ctr, sh) == vm.VM_ERR_INVALID_ARG
    assert L.vm_scroll_target(None, ctr, sh) == vm.VM_ERR_INVALID_ARG
    assert L.vm_get_window(None, sh, ctr) == vm.VM_ERR_INVALID_ARG
    assert L.vm_integrate(None, None, 0, None, 0) == vm.VM_ERR_INVALID_ARG
    assert L.vm_graph_shape(None, None, None, None) == vm.VM_ERR_INVALID_ARG
    assert L.vm_destroy(None) == vm.VM_OK  # like free(NULL)


def test_binding_constants_match_header():
    """Every status code and flag the header defines has the same value in the
    Python binding (status names included)."""
    from paper_2510_01592_gb300 import vm
    src = open(os.path.join(ROOT, "include", "vm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = {n: int(v) for n, v in re.findall(r"\b(VM_[A-Z_]+)\s*=\s*(\d+)", src)}
    consts.update({n: int(v) for n, v in re.findall(r"#define\s+(VM_[A-Z_]+)\s+(\d+)u?", src)})
    assert {"VM_OK", "VM_ERR_EXTENT", "VM_MAP_EAGER", "VM_INTEGRATE_CLEAR", "VM_FIT_EAGER"} <= set(consts)
    for name, value in consts.items():
        if name.startswith("VM_SERVE_"):
            from paper_2510_01592_gb300 import serve
            assert getattr(serve, name[len("VM_SERVE_"):]) == value, name  # serve.BATCHED, serve.STREAMS
            continue
        assert getattr(vm, name) == value, name
        if name.startswith("VM_ERR_") or name == "VM_OK":
            assert vm.STATUS_NAMES[value] == name
