"""GPU: sequential multi-plane extraction per cluster (planes_per_cluster > 1)
against the oracle: the same records in (label, round) order, bit for bit
(the refit within tolerance), the same hulls, the first round's inlier sets;
the paper's single plane is round 0 unchanged; graph and kernel-by-kernel
replays agree; the single-round entry points refuse more than one round."""
import numpy as np
import pytest

import synth
from parity import compare_planes
from test_oracle_multiplane import _floor_and_ramp

pytestmark = pytest.mark.gpu

IDENTITY = np.eye(3, 4, dtype=np.float32).reshape(12)


@pytest.fixture(scope="module")
def vmmod():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_01592_gb300 import vm
    vm.load()
    return vm


def _maps(orc, vm, spec, clouds, eager=False):
    gm = vm.VoxelMap(spec.dims, spec.origin, spec.voxel_size, eager=eager)
    om = orc.OracleMap(spec.dims, spec.origin, spec.voxel_size)
    for pts, pose in clouds:
        gm.integrate(pts, pose)
        om.integrate(pts.cpu().numpy() if hasattr(pts, "cpu") else pts, pose)
    return gm, om


@pytest.mark.parametrize("P", [2, 3, 8])
def test_floor_and_ramp_matches_the_oracle(orc, vmmod, P):
    spec, pts = _floor_and_ramp()
    gm, om = _maps(orc, vmmod, spec, [(pts, IDENTITY)])
    gres = gm.segment(vmmod.segment_params(n_hyp=64, planes_per_cluster=P))
    ores = om.segment(orc.make_params(n_hyp=64, planes_per_cluster=P))
    assert list(ores["planes"]["round"][:2]) == [0, 1]
    compare_planes(gres, ores, gm.export_clusters())


@pytest.mark.parametrize("P", [3, 4])
def test_trajectory_with_several_rounds_matches_the_oracle(orc, vmmod, P):
    # every occupied voxel clustered (classify = 0): walls and their ledges
    # share clusters, which then give up two to four planes
    spec, scene = synth.config2_spec(), synth.config2_scene()
    clouds = [synth.config2_frame(f, scene, device="cuda") for f in range(0, 30, 3)]
    gm, om = _maps(orc, vmmod, spec, clouds)
    for seed in (0, 5):
        gres = gm.segment(vmmod.segment_params(n_hyp=100, seed=seed, classify=0, planes_per_cluster=P))
        ores = om.segment(orc.make_params(n_hyp=100, seed=seed, classify=0, planes_per_cluster=P))
        assert (ores["planes"]["round"] == P - 1).any()
        compare_planes(gres, ores, gm.export_clusters())


def test_round_zero_is_the_single_plane_fit(vmmod):
    spec, scene = synth.config2_spec(), synth.config2_scene()
    m = vmmod.VoxelMap(spec.dims, spec.origin, spec.voxel_size)
    for f in range(0, 30, 3):
        m.integrate(*synth.config2_frame(f, scene, device="cuda"))
    one = m.segment(vmmod.segment_params(n_hyp=100, classify=0))
    inl_one = m.export_clusters()["inlier"]
    many = m.segment(vmmod.segment_params(n_hyp=100, classify=0, planes_per_cluster=4))
    inl_many = m.export_clusters()["inlier"]
    p1, pm = one["planes"], many["planes"]
    r0 = ((pm["flags"] >> 8) & 0xFF) == 0
    assert r0.sum() == len(p1) and len(pm) > len(p1)
    for key in p1.dtype.names:
        if key != "hull_offset":
            assert np.array_equal(pm[key][r0], p1[key]), key
    for i, j in zip(np.nonzero(r0)[0], range(len(p1))):  # the same hulls, at other offsets
        a = many["hull_xyz"][pm["hull_offset"][i]:pm["hull_offset"][i] + pm["hull_count"][i]]
        b = one["hull_xyz"][p1["hull_offset"][j]:p1["hull_offset"][j] + p1["hull_count"][j]]
        assert np.array_equal(a, b)
    assert np.array_equal(inl_one, inl_many)
    # records of one cluster are consecutive, in round order; later rounds have fewer points
    lab, rnd = pm["label"].astype(np.int64), (pm["flags"] >> 8) & 0xFF
    assert np.all((np.diff(lab) > 0) | ((np.diff(lab) == 0) & (np.diff(rnd.astype(np.int64)) == 1)))
    later = np.nonzero(rnd > 0)[0]
    assert np.all(pm["n_points"][later] < pm["n_points"][later - 1])
    assert np.all(pm["best_h"][later] >= 0)


def test_graph_and_kernel_by_kernel_agree(vmmod):
    spec, pts = _floor_and_ramp(seed=3)
    spec1, pts1, _ = synth.config1()
    out = []
    for eager in (False, True):
        m = vmmod.VoxelMap(spec.dims, spec.origin, spec.voxel_size, eager=eager)
        m.integrate(pts, IDENTITY)
        m.integrate(pts1 + np.float32([0.5, 0.0, 0.0]), IDENTITY)
        gp = vmmod.segment_params(n_hyp=64, planes_per_cluster=3)
        out.append([m.segment(gp) for _ in range(2)])
        m.close()
    ref = out[0][0]
    for r in out[0][1:] + out[1]:
        for key in ("planes", "hull_xy", "hull_xyz"):
            assert np.array_equal(r[key], ref[key]), key


def test_single_round_entry_points_refuse_several_rounds(vmmod):
    import torch
    xyz = torch.zeros((300, 3), dtype=torch.float32, device="cuda")
    off = torch.tensor([0, 300], dtype=torch.int32, device="cuda")
    with pytest.raises(vmmod.VmError) as ei:
        vmmod.fit_planes(xyz, off, vmmod.segment_params(planes_per_cluster=2))
    assert ei.value.status == vmmod.VM_ERR_INVALID_ARG
    m = vmmod.VoxelMap((10, 10, 10), (0, 0, 0), 0.1)
    with pytest.raises(vmmod.VmError) as ei:
        m.segment(vmmod.segment_params(planes_per_cluster=9))
    assert ei.value.status == vmmod.VM_ERR_INVALID_ARG
    from paper_2510_01592_gb300 import serve
    with pytest.raises(vmmod.VmError) as ei:
        serve.Server(vmmod.segment_params(planes_per_cluster=2))
    assert ei.value.status == vmmod.VM_ERR_INVALID_ARG
