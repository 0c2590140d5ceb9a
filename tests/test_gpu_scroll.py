"""GPU: the robot-centric map window (Sec. III.B: the map's centre follows the
robot) against the oracle, bit for bit: sums, counts and voxel ids after
random integrations and whole-brick scrolls; the evicted-voxel count; a
camera-following window over the paper-scale trajectory with Eq. 2 clearing,
segmented at the end; graph replays that follow the window without a new
capture; a pool that only fits the window reused after evictions; invalid
shifts refused."""
import numpy as np
import pytest

import synth
from parity import compare_labels, compare_planes, compare_sums

pytestmark = pytest.mark.gpu

N = (48, 40, 24)
ORIGIN = (0.3, -0.2, 0.1)
RES = 0.02


@pytest.fixture(scope="module")
def vmmod():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_01592_gb300 import vm
    vm.load()
    return vm


def test_random_integrations_and_scrolls_match_the_oracle(orc, vmmod):
    rng = np.random.default_rng(0)
    gm = vmmod.VoxelMap(N, ORIGIN, RES)
    om = orc.OracleMap(N, ORIGIN, RES)
    eye = np.eye(3, 4, dtype=np.float32).reshape(12)
    shifts = [(1, 0, 0), (0, -1, 1), (-2, 1, 0), (3, 2, -1), (0, 0, 0), (-1, -1, -1), (5, 0, 0), (-5, 0, 0)]
    for sh in [None] + shifts:
        if sh is not None:
            gm.scroll(sh)
            om.scroll(sh)
        w = om.window()["offset"]
        lo = np.float32(ORIGIN) + w * RES - 0.1
        p = (lo + rng.uniform(0, 1, (20000, 3)) * (np.array(N) * RES + 0.2)).astype(np.float32)
        gm.integrate(p, eye)
        om.integrate(p)
        compare_sums(gm, om)
        assert np.array_equal(gm.window()["offset"], w)
        assert np.array_equal(gm.window()["position_origin"], om.window()["position_origin"])
    assert gm.stats()["voxels_evicted"] == om.window()["voxels_evicted"] > 0
    gp, op = vmmod.segment_params(n_hyp=32, classify=0), orc.make_params(n_hyp=32, classify=0)
    compare_planes(gm.segment(gp), om.segment(op), gm.export_clusters())


def _follow(vm, orc, frames, clear, dims=(240, 240, 160), eager=False, capacity=0):
    spec = synth.config2_spec()
    gm = vm.VoxelMap(dims, spec.origin, spec.voxel_size, eager=eager, brick_capacity=capacity)
    om = orc.OracleMap(dims, spec.origin, spec.voxel_size) if orc else None
    scene = synth.config2_scene()
    for i, f in enumerate(frames):
        pts, pose = synth.config2_frame(f, scene, device="cuda")
        cam = pose.reshape(3, 4)[:, 3]
        sh = gm.scroll_to(cam)
        if om is not None:
            assert np.array_equal(om.scroll_to(cam), sh)
        gm.integrate(pts, pose, clear=clear)
        if om is not None:
            if clear:
                om.clear_rays(pts.cpu().numpy(), pose)
            om.integrate(pts.cpu().numpy(), pose)
            if i % 8 == 7:
                compare_sums(gm, om)
    return gm, om


def test_camera_following_window_with_clearing_matches_the_oracle(orc, vmmod):
    frames = list(range(1, 200, 6))
    gm, om = _follow(vmmod, orc, frames, clear=True)
    compare_sums(gm, om)
    assert np.array_equal(gm.window()["offset"], om.window()["offset"])
    assert gm.stats()["voxels_evicted"] == om.window()["voxels_evicted"] > 0
    assert gm.window()["offset"][0] >= 80  # the window moved with the camera
    gp, op = vmmod.segment_params(n_hyp=100), orc.make_params(n_hyp=100)
    ores = om.segment(op)
    gres = gm.segment(gp)
    compare_labels(gm.export_labels(), ores["voxels"])
    compare_planes(gres, ores, gm.export_clusters())
    assert len(gres["planes"]) >= 5


def test_graph_replays_follow_the_window(vmmod):
    """Segmenting every few frames while the window moves: the captured graph
    (no re-capture after a scroll) gives what kernel-by-kernel launches give."""
    frames = list(range(1, 120, 3))
    out = []
    for eager in (False, True):
        spec = synth.config2_spec()
        m = vmmod.VoxelMap((240, 240, 160), spec.origin, spec.voxel_size, eager=eager)
        scene = synth.config2_scene()
        res = []
        c0 = vmmod.capture_count()
        for i, f in enumerate(frames):
            pts, pose = synth.config2_frame(f, scene, device="cuda")
            m.scroll_to(pose.reshape(3, 4)[:, 3])
            m.integrate(pts, pose)
            if i % 4 == 3:
                res.append(m.segment(vmmod.segment_params(n_hyp=64)))
        captures = vmmod.capture_count() - c0
        out.append((res, m.window()["offset"].copy(), captures))
        m.close()
    (ga, wa, ca), (gb, wb, _) = out
    assert np.array_equal(wa, wb) and wa[0] > 0
    assert ca <= 4  # captures only when the scratch grows, not per scroll
    for a, b in zip(ga, gb):
        for key in ("planes", "hull_xy", "hull_xyz"):
            assert np.array_equal(a[key], b[key]), key


def test_evictions_free_the_pool_for_new_bricks(orc, vmmod):
    """A pool that holds little more than one window: walking the trajectory
    only fits because evicted bricks are reused."""
    frames = list(range(1, 300, 10))
    gm, om = _follow(vmmod, orc, frames, clear=False, dims=(160, 160, 120), capacity=600)
    st = gm.stats()
    assert st["points_no_capacity"] == 0 and st["bricks_allocated"] <= 600
    assert st["voxels_evicted"] > 0
    compare_sums(gm, om)


def test_far_scroll_empties_the_map_and_bad_shifts_are_refused(vmmod):
    m = vmmod.VoxelMap(N, ORIGIN, RES)
    p = np.random.default_rng(3).uniform(0.3, 1.0, (5000, 3)).astype(np.float32)
    m.integrate(p, np.eye(3, 4, dtype=np.float32).reshape(12))
    n0 = len(m.export_voxels()[0])
    m.scroll((100, 0, 0))
    assert len(m.export_voxels()[0]) == 0 and m.stats()["voxels_evicted"] == n0
    assert m.stats()["bricks_allocated"] == 0
    w = m.window()["offset"].copy()
    with pytest.raises(vmmod.VmError) as ei:
        m.scroll((1 << 21, 0, 0))
    assert ei.value.status == vmmod.VM_ERR_INVALID_ARG
    assert np.array_equal(m.window()["offset"], w)
    with pytest.raises(vmmod.VmError):
        m.scroll_to((float("nan"), 0.0, 0.0))


def test_odd_pool_capacity_above_the_small_scan(orc, vmmod):
    """An odd brick capacity (16,385: the scroll's scan takes the multi-CTA
    look-back path, whose state holds 64-bit words) against the oracle."""
    dims, origin, res = (264, 264, 128), (-6.6, -6.6, -3.2), 0.05
    gm = vmmod.VoxelMap(dims, origin, res, brick_capacity=16385)
    om = orc.OracleMap(dims, origin, res)
    rng = np.random.default_rng(4)
    eye = np.eye(3, 4, dtype=np.float32).reshape(12)
    for sh in [None, (10, 0, 0), (-12, 3, 2)]:
        if sh is not None:
            gm.scroll(sh)
            om.scroll(sh)
        p = (rng.uniform(-1, 1, (200000, 3)) * [3.0, 3.0, 1.5]).astype(np.float32)
        gm.integrate(p, eye)
        om.integrate(p)
        compare_sums(gm, om)
    assert gm.stats()["voxels_evicted"] == om.window()["voxels_evicted"] > 0


@pytest.mark.parametrize("res,w", [(0.01, (2104, -2072, 2104)), (0.05, (544, -528, -528)),
                                   (0.02, (-1040, 1056, -1040))])
def test_far_window_negative_sums_match_the_oracle(orc, vmmod, res, w):
    """A window far from the base origin (about 21 m at 0.01 m voxels, 26 m
    at 0.05 m, either sign): points keyed into its first voxel row can
    quantise one 2^-20 m unit below the window's anchor, so voxel sums are
    negative (tests/test_oracle_scroll.py checks that these inputs reach that
    case on every axis, in single-point and many-point voxels).  Sums and
    counts, means, normals, labels and planes match the oracle bit for bit."""
    dims = (32, 32, 32)
    gm = vmmod.VoxelMap(dims, (0.0, 0.0, 0.0), res)
    om = orc.OracleMap(dims, (0.0, 0.0, 0.0), res)
    sh = np.asarray(w, np.int32) // 8
    gm.scroll(sh)
    om.scroll(sh)
    assert np.array_equal(gm.window()["offset"], w)
    p = synth.far_window_points(w, dims, res)
    eye = np.eye(3, 4, dtype=np.float32).reshape(12)
    for half in (p[0::2], p[1::2]):  # two frames
        gm.integrate(half, eye)
        om.integrate(half)
    compare_sums(gm, om)
    _, S, c = om.export_sums()
    assert ((S < 0) & (c[:, None] == 1)).any() and ((S < 0) & (c[:, None] > 1)).any()
    d_th = max(0.05, 2 * res)  # at 0.05 m voxels the paper's 0.05 m would cut most neighbour pairs
    gp = vmmod.segment_params(n_hyp=64, classify=0, d_th=d_th)
    op = orc.make_params(n_hyp=64, classify=0, d_th=d_th)
    ores = om.segment(op)
    gres = gm.segment(gp)
    compare_labels(gm.export_labels(), ores["voxels"])
    compare_planes(gres, ores, gm.export_clusters())
    assert len(gres["planes"]) >= 3
