"""GPU: ray-cast clearing (Sec. III.B, Eq. 2) against the oracle, bit for bit:
the voxel sums and counts after every clear-then-integrate step of the
paper-scale trajectory and of a LiDAR crop, the number of voxels cleared, the
moved-object scene, and the segmentation of a cleared map."""
import numpy as np
import pytest

import synth
from parity import compare_planes, compare_sums

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vmmod():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_01592_gb300 import vm
    vm.load()
    return vm


def test_trajectory_with_clearing_matches_the_oracle(orc, vmmod):
    spec, scene = synth.config2_spec(), synth.config2_scene()
    gm = vmmod.VoxelMap(spec.dims, spec.origin, spec.voxel_size)
    om = orc.OracleMap(spec.dims, spec.origin, spec.voxel_size)
    cleared = 0
    for f in range(1, 25, 2):
        pts, pose = synth.config2_frame(f, scene, device="cuda")
        gm.integrate(pts, pose, clear=True)
        cleared += om.clear_rays(pts.cpu().numpy(), pose)
        om.integrate(pts.cpu().numpy(), pose)
        if f % 6 == 5:
            compare_sums(gm, om)
    compare_sums(gm, om)
    assert gm.stats()["voxels_cleared"] == cleared and cleared > 0
    op, gp = orc.make_params(n_hyp=100), vmmod.segment_params(n_hyp=100)
    compare_planes(gm.segment(gp), om.segment(op), gm.export_clusters())


def test_moved_object_is_cleared_like_the_oracle(orc, vmmod):
    spec = synth.MapSpec((200, 200, 100), (0.0, 0.0, -0.05), 0.02)
    with_box, without = synth.Scene(), synth.Scene()
    for sc in (with_box, without):
        sc.add(synth._aabb_planes((-50, -50, -1), (50, 50, 0)))
    with_box.add(synth._aabb_planes((1.6, 1.6, 0.0), (2.2, 2.2, 0.5)))
    pose = synth.camera_pose((0.5, 0.5, 1.2), 0.785, 35.0).astype(np.float32).reshape(12)
    cam = synth.Camera()
    a = synth._depth_frame(with_box, cam, pose.reshape(3, 4).astype(np.float64), seed=1, device="cuda")
    b = synth._depth_frame(without, cam, pose.reshape(3, 4).astype(np.float64), seed=2, device="cuda")
    gm = vmmod.VoxelMap(spec.dims, spec.origin, spec.voxel_size)
    om = orc.OracleMap(spec.dims, spec.origin, spec.voxel_size)
    for pts, clear in ((a, False), (b, True), (a, True), (b, True)):
        gm.integrate(pts, pose, clear=clear)
        if clear:
            om.clear_rays(pts.cpu().numpy(), pose)
        om.integrate(pts.cpu().numpy(), pose)
        compare_sums(gm, om)


def test_lidar_crop_with_clearing_matches_the_oracle(orc, vmmod):
    scene = synth.config5_scene()
    origin, dims = (5.3, 2.8, -0.05), (240, 240, 200)
    gm = vmmod.VoxelMap(dims, origin, 0.01)
    om = orc.OracleMap(dims, origin, 0.01)
    for f in (0, 6, 12):
        pts, pose = synth.config5_frame(f, scene, device="cuda")
        gm.integrate(pts, pose, clear=True)
        om.clear_rays(pts.cpu().numpy(), pose)
        om.integrate(pts.cpu().numpy(), pose)
    compare_sums(gm, om)


def test_sensor_outside_the_map_clears_nothing(vmmod):
    spec, scene = synth.config2_spec(), synth.config2_scene()
    gm = vmmod.VoxelMap((100, 100, 100), (2.0, 2.0, 0.0), 0.01)  # a 1 m cube away from the camera
    for f in (1, 2, 3):
        pts, pose = synth.config2_frame(f, scene, device="cuda")
        gm.integrate(pts, pose, clear=True)
    assert gm.stats()["voxels_cleared"] == 0
