"""Pins of the oracle's ray-cast clearing (Sec. III.B, Eq. 2): a closed-form
axis-aligned ray, the exact set of voxels a segment crosses (rational
arithmetic on the same FP32 end points) for random rays, the walk's
structure, the point's own voxel kept, and a moved object removed."""
from fractions import Fraction

import numpy as np
import pytest

import synth

RES = 0.1


def _full_map(orc, n=12):
    """An n^3 grid at 0.1 m with one point at every voxel centre."""
    m = orc.OracleMap((n, n, n), (0.0, 0.0, 0.0), RES)
    g = (np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3) + 0.5) * RES
    m.integrate(g.astype(np.float32))
    return m, n


def _occupied(m):
    vid, _, _ = m.export_sums()
    return set(vid.tolist())


def _vid(ijk, n):
    """Brick-major voxel id (8^3 bricks, x fastest) of grid coordinates."""
    i, j, k = ijk
    nb = (n + 7) // 8
    b = ((k >> 3) * nb + (j >> 3)) * nb + (i >> 3)
    return b * 512 + (((k & 7) * 8 + (j & 7)) * 8 + (i & 7))


def _pose(t):
    return np.array([1, 0, 0, t[0], 0, 1, 0, t[1], 0, 0, 1, t[2]], np.float32)


def _ray(m, t, p_map):
    """Casts one ray from sensor position t to the map point p_map (given in the
    sensor frame of a translation-only pose); returns the end point in voxel
    units as the oracle forms it and the set of voxels cleared."""
    t = np.asarray(t, np.float32)
    ps = (np.asarray(p_map, np.float32) - t).astype(np.float32).reshape(1, 3)
    w = (ps[0] + t).astype(np.float32)  # fmaf(1, x, t) with zero cross terms: one rounding
    e = w * np.float32(1.0 / RES)
    before = _occupied(m)
    k = m.clear_rays(ps, _pose(t))
    return e, before - _occupied(m), k


def test_axis_aligned_ray_clears_the_voxels_before_the_point(orc):
    m, n = _full_map(orc)
    t = np.float32([0.05, 0.35, 0.65])  # sensor at the centre of voxel (0, 3, 6)
    e, gone, k = _ray(m, t, [1.05, 0.35, 0.65])  # one metre along +x: voxel (10, 3, 6)
    assert k == 10  # voxels x = 0..9; the point's own voxel x = 10 stays
    assert gone == {_vid((x, 3, 6), n) for x in range(10)}


def _exact_crossed(s, e, n):
    """Voxels of the n^3 grid whose interior the segment s -> e crosses
    (positive-length intersection), from exact rationals; and whether some
    pair of boundary crossings is closer than 1e-4 in the ray parameter."""
    S = [Fraction(float(x)) for x in s]
    E = [Fraction(float(x)) for x in e]
    D = [E[a] - S[a] for a in range(3)]
    ts = []
    for a in range(3):
        if D[a] == 0:
            continue
        lo, hi = sorted((S[a], E[a]))
        for b in range(int(np.floor(float(lo))) + 1, int(np.floor(float(hi))) + 1):
            if lo < b < hi:
                ts.append(((b - S[a]) / D[a], a))
    ts.sort()
    near = any(abs(float(ts[i + 1][0] - ts[i][0])) < 1e-4 and ts[i + 1][1] != ts[i][1] for i in range(len(ts) - 1))
    cut = [Fraction(0)] + [t for t, _ in ts] + [Fraction(1)]
    out = set()
    for i in range(len(cut) - 1):
        if cut[i + 1] <= cut[i]:
            continue
        mid = (cut[i] + cut[i + 1]) / 2
        v = tuple(int(np.floor(float(S[a] + mid * D[a]))) for a in range(3))
        if all(0 <= v[a] < n for a in range(3)):
            out.add(v)
    return out, near


def test_random_rays_cross_exactly_the_voxels_of_the_segment(orc):
    rng = np.random.default_rng(3)
    checked = 0
    for trial in range(150):
        m, n = _full_map(orc)
        t = rng.uniform(0.05, 1.15, 3).astype(np.float32)
        p = rng.uniform(-0.1, 1.3, 3)  # may end outside the grid
        s = t * np.float32(1.0 / RES)
        e, gone, _ = _ray(m, t, p)
        exact, near = _exact_crossed(s, e, n)
        exact.discard(tuple(int(np.floor(x)) for x in e))
        if near:
            continue
        assert gone == {_vid(v, n) for v in exact}, (trial, t, p)
        checked += 1
    assert checked > 100


def test_walk_is_a_monotone_path_that_stops_before_the_point(orc):
    rng = np.random.default_rng(11)
    for _ in range(40):
        m, n = _full_map(orc)
        t = rng.uniform(0.05, 1.15, 3).astype(np.float32)
        p = rng.uniform(0.05, 1.15, 3)  # inside: the walk never leaves the grid
        v0 = tuple(int(np.floor(x)) for x in t * np.float32(1 / RES))
        e, gone, k = _ray(m, t, p)
        ve = tuple(int(np.floor(x)) for x in e)
        assert k == sum(abs(a - b) for a, b in zip(v0, ve))  # one voxel a step, the end voxel excluded
        assert _vid(ve, n) not in gone
        if v0 != ve:
            assert _vid(v0, n) in gone


def test_non_finite_points_cast_no_ray(orc):
    m, _ = _full_map(orc)
    p = np.array([[np.nan, 0.5, 0.5], [np.inf, 0.2, 0.2]], np.float32)
    assert m.clear_rays(p, _pose(np.float32([0.05, 0.05, 0.05]))) == 0


def test_a_moved_object_is_cleared(orc):
    """A box seen from a fixed camera, then the same view without it: the box's
    surface voxels lie on rays that now reach the floor behind, and are
    cleared; the floor stays."""
    spec = synth.MapSpec((200, 200, 100), (0.0, 0.0, -0.05), 0.02)
    with_box, without = synth.Scene(), synth.Scene()
    for sc in (with_box, without):
        sc.add(synth._aabb_planes((-50, -50, -1), (50, 50, 0)))
    with_box.add(synth._aabb_planes((1.6, 1.6, 0.0), (2.2, 2.2, 0.5)))
    pose = synth.camera_pose((0.5, 0.5, 1.2), 0.785, 35.0)
    cam = synth.Camera(width=160, height=120)
    a = synth._depth_frame(with_box, cam, pose, seed=1).numpy()
    b = synth._depth_frame(without, cam, pose, seed=2).numpy()
    m = orc.OracleMap(spec.dims, spec.origin, spec.voxel_size)
    m.integrate(a, pose.astype(np.float32).reshape(12))
    vid, S, c = m.export_sums()
    mu = S / c[:, None] / 2**20 + np.array(spec.origin)
    in_box = (mu[:, 0] > 1.58) & (mu[:, 0] < 2.22) & (mu[:, 1] > 1.58) & (mu[:, 1] < 2.22) & (mu[:, 2] > 0.03)
    box_vox = set(vid[in_box].tolist())
    assert len(box_vox) > 100
    m.clear_rays(b, pose.astype(np.float32).reshape(12))
    m.integrate(b, pose.astype(np.float32).reshape(12))
    left = box_vox & set(m.export_sums()[0].tolist())
    assert len(left) <= 0.02 * len(box_vox), len(left)
    floor = (mu[:, 2] < 0.02)
    assert len(set(vid[floor].tolist()) & set(m.export_sums()[0].tolist())) > 0.8 * floor.sum()


def test_clearing_is_the_same_on_all_threads(orc):
    spec, scene = synth.config2_spec(), synth.config2_scene()
    res = []
    for th in (1, 4):
        orc.set_threads(th)
        try:
            m = orc.OracleMap(spec.dims, spec.origin, spec.voxel_size)
            k = 0
            for f in (1, 9, 17):
                pts, pose = synth.config2_frame(f, scene)
                k += m.clear_rays(pts.numpy(), pose)
                m.integrate(pts.numpy(), pose)
            res.append((k, m.export_sums()))
        finally:
            orc.set_threads(1)
    assert res[0][0] == res[1][0]
    for x, y in zip(res[0][1], res[1][1]):
        assert np.array_equal(x, y)


def test_a_sensor_outside_the_grid_casts_no_ray(orc):
    m, _ = _full_map(orc)
    t = np.float32([-0.5, 0.55, 0.55])  # 0.5 m outside the x = 0 face
    e, gone, k = _ray(m, t, [0.95, 0.55, 0.55])
    assert k == 0 and not gone
