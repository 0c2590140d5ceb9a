"""GPU: the reusable batched fit (vm_fit_plan_*) and its autotuner.  Every
schedule gives the oracle's integer results bit for bit (selected hypothesis,
inlier counts, RANSAC planes, hulls) and the refit within 1e-4 rad / 1e-5 m,
and all schedules give one and the same result (the refit's partial sums do
not follow the tile); a plan that outgrows its sizes grows and still matches."""
import numpy as np
import pytest

import synth
from parity import compare_planes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vmmod():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_01592_gb300 import vm
    vm.load()
    return vm


def _batch(seed, n_clusters, hi):
    xyz, off, _ = synth.config3_clusters(n_clusters=n_clusters, seed=seed, size_hi=hi)
    labels = (np.arange(n_clusters, dtype=np.uint32) * 2654435761 % 1000003).astype(np.uint32)
    return xyz.astype(np.float32), off.astype(np.uint32), labels


def _dev(*arrays):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def _same(a, b):
    for key in ("planes", "hull_xy", "hull_xyz"):
        assert np.array_equal(a[key], b[key]), key


@pytest.mark.parametrize("n_hyp", [64, 100, 256])
def test_every_schedule_matches_the_oracle(orc, vmmod, n_hyp):
    xyz, off, labels = _batch(21, 120, 30000)
    op, gp = orc.make_params(n_hyp=n_hyp, seed=5), vmmod.segment_params(n_hyp=n_hyp, seed=5)
    ores = orc.fit_planes(xyz, off, op, labels=labels)
    dx, doff, dlab = _dev(xyz, off, labels)
    plan = vmmod.FitPlan(len(labels), len(xyz), gp)
    first = None
    for tile, r, c, sched in [(2048, 4, 4, "cta"), (1024, 8, 2, "cta"), (8192, 2, 1, "cta"),
                              (256, 4, 4, "warp"), (512, 8, 8, "warp"), (1024, 2, 1, "warp")]:
        plan.set_tuning(tile, r, c, sched)
        g = plan.run(dx, doff, dlab)
        compare_planes(g, ores)
        if first is None:
            first = g
        else:  # every schedule gives the same result, refit included
            _same(g, first)
    plan.close()


def test_plan_equals_fit_planes_and_replays(orc, vmmod):
    xyz, off, labels = _batch(4, 80, 20000)
    gp = vmmod.segment_params(n_hyp=256, seed=7)
    dx, doff, dlab = _dev(xyz, off, labels)
    ref = vmmod.fit_planes(dx, doff, gp, labels=dlab)
    plan = vmmod.FitPlan(len(labels), len(xyz), gp)
    for _ in range(3):  # graph replays with the same pointers
        g = plan.run(dx, doff, dlab)
        for key in ("planes", "hull_xy", "hull_xyz"):
            assert np.array_equal(g[key], ref[key]), key
    eager = vmmod.FitPlan(len(labels), len(xyz), gp, eager=True)
    ge = eager.run(dx, doff, dlab)
    for key in ("planes", "hull_xy", "hull_xyz"):
        assert np.array_equal(ge[key], ref[key]), key


def test_plan_grows_past_its_sizes(orc, vmmod):
    """Created for 4 clusters / 100 points, then fed larger batches (more
    clusters; more points with the same cluster count; more hull vertices):
    it grows, re-captures and still matches the oracle."""
    gp = vmmod.segment_params(n_hyp=64, seed=2)
    op = orc.make_params(n_hyp=64, seed=2)
    plan = vmmod.FitPlan(4, 100, gp)
    for seed, n, hi in [(1, 3, 500), (2, 3, 60000), (3, 90, 40000)]:
        xyz, off, labels = _batch(seed, n, hi)
        dx, doff, dlab = _dev(xyz, off, labels)
        compare_planes(plan.run(dx, doff, dlab), orc.fit_planes(xyz, off, op, labels=labels))


def test_autotune_picks_a_valid_schedule_with_unchanged_results(orc, vmmod):
    xyz, off, labels = _batch(9, 150, 50000)
    gp = vmmod.segment_params(n_hyp=100, seed=1)
    op = orc.make_params(n_hyp=100, seed=1)
    dx, doff, dlab = _dev(xyz, off, labels)
    plan = vmmod.FitPlan(len(labels), len(xyz), gp)
    before = plan.run(dx, doff, dlab)
    best, ms, n = plan.autotune(dx, doff, dlab, reps=1)
    assert n >= 10 and ms > 0
    assert best == plan.tuning
    after = plan.run(dx, doff, dlab)
    _same(after, before)
    compare_planes(after, orc.fit_planes(xyz, off, op, labels=labels))


def _one(res, c):
    """Cluster c of a batch result as a one-plane result (hull rebased)."""
    p = res["planes"][c:c + 1].copy()
    o, n = int(p["hull_offset"][0]), int(p["hull_count"][0])
    p["hull_offset"][0] = 0
    return {"planes": p, "hull_xy": res["hull_xy"][o:o + n], "hull_xyz": res["hull_xyz"][o:o + n]}


def test_full_size_batch_sampled_against_the_oracle(orc, vmmod):
    """The bench's batching workload at full size (2,000 clusters, 47.7 M points,
    H = 256) in the bench's launch configuration (autotuned plan, graph replay).
    Sampled clusters (the five largest, the five smallest, ten at random) are
    fitted alone by the oracle under their batch index as label: a cluster's
    result does not depend on its batch, so each must match bit for bit (the
    refit within tolerance)."""
    import torch
    xyz, off, _ = synth.config3_clusters_device(device="cuda")
    gp, op = vmmod.segment_params(n_hyp=256, seed=7), orc.make_params(n_hyp=256, seed=7)
    plan = vmmod.FitPlan(off.numel() - 1, xyz.shape[0], gp)
    plan.autotune(xyz, off, reps=1)
    g = plan.run(xyz, off)
    offn = off.cpu().numpy().astype(np.int64)
    sizes = np.diff(offn)
    order = np.argsort(sizes, kind="stable")
    rng = np.random.default_rng(0)
    pick = sorted(set(order[:5].tolist() + order[-5:].tolist() + rng.choice(len(sizes), 10, replace=False).tolist()))
    for c in pick:
        pts = xyz[offn[c]:offn[c + 1]].cpu().numpy()
        o = orc.fit_planes(pts, np.array([0, len(pts)], np.uint32), op, labels=np.array([c], np.uint32))
        compare_planes(_one(g, c), o)
    del xyz, off
    torch.cuda.empty_cache()


def test_map_tuning_changes_nothing_but_speed(orc, vmmod):
    """A map's fit schedule (tile, hypotheses per thread, CTAs per SM, CTA or
    warp per item) and its autotuner leave the segmentation bit for bit."""
    spec, scene = synth.config2_spec(), synth.config2_scene()
    m = vmmod.VoxelMap(spec.dims, spec.origin, spec.voxel_size)
    for f in range(1, 25, 3):
        pts, pose = synth.config2_frame(f, scene, device="cuda")
        m.integrate(pts, pose)
    gp = vmmod.segment_params(n_hyp=100, seed=4)
    ref = m.segment(gp)
    for t in [dict(tile=512, hyp_per_thread=4, ctas_per_sm=4, schedule="cta"),
              dict(tile=256, hyp_per_thread=4, ctas_per_sm=8, schedule="warp"),
              dict(tile=4096, hyp_per_thread=8, ctas_per_sm=2, schedule="cta")]:
        m.set_fit_tuning(t)
        assert m.fit_tuning == t
        _same(m.segment(gp), ref)
    best, ms, n = m.autotune(gp, reps=2)
    assert n >= 10 and ms > 0 and m.fit_tuning == best
    _same(m.segment(gp), ref)
    with pytest.raises(vmmod.VmError):
        m.set_fit_tuning(dict(tile=300, hyp_per_thread=4, ctas_per_sm=4))
