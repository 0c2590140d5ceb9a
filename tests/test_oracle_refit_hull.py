"""Pins for the oracle's inlier refit (total least squares, double) and the
boundary polygon (Sec. III.C, boundary polygon generation): the exact integer
monotone-chain hull of the in-plane coordinates quantised to 2^-16 m."""
import itertools
import math

import numpy as np
import pytest
from scipy.spatial import ConvexHull


def _plane_points(rng, n, normal, center, half=0.4, sigma=0.0):
    nrm = np.asarray(normal, float)
    nrm /= np.linalg.norm(nrm)
    a = np.array([1.0, 0, 0]) if abs(nrm[0]) < 0.9 else np.array([0, 1.0, 0])
    u = np.cross(a, nrm); u /= np.linalg.norm(u)
    w = np.cross(nrm, u)
    s = rng.uniform(-half, half, size=(n, 2))
    p = np.asarray(center) + s[:, :1] * u + s[:, 1:] * w + rng.normal(0, sigma, (n, 1)) * nrm if sigma else \
        np.asarray(center) + s[:, :1] * u + s[:, 1:] * w
    return p.astype(np.float32), nrm


@pytest.mark.parametrize("tilt,az", [(0.0, 0.0), (12.0, 40.0), (34.0, 250.0), (70.0, 10.0)])
def test_refit_exact_plane(orc, tilt, az):
    rng = np.random.default_rng(int(tilt * 7 + az))
    t, a = math.radians(tilt), math.radians(az)
    nrm = (math.sin(t) * math.cos(a), math.sin(t) * math.sin(a), math.cos(t))
    pts, n_true = _plane_points(rng, 3000, nrm, (1.5, -2.0, 0.7))
    res = orc.fit_planes(pts, [0, 3000], orc.make_params(n_hyp=32))
    P = res["planes"]
    assert P["inlier_count"][0] == 3000
    ang = math.acos(min(1.0, abs(float(P["refit_n"][0] @ n_true))))
    assert ang < 1e-6
    assert P["refit_n"][0][2] >= 0
    d_true = -float(n_true @ np.array([1.5, -2.0, 0.7])) * np.sign(P["refit_n"][0] @ n_true)
    assert abs(P["refit_d"][0] - d_true) < 1e-6
    assert P["ill_conditioned"][0] == 0


@pytest.mark.parametrize("seed", range(4))
def test_refit_matches_svd(orc, seed):
    rng = np.random.default_rng(seed)
    pts, _ = _plane_points(rng, 5000, rng.normal(size=3) * [0.3, 0.3, 1], rng.uniform(-3, 3, 3), sigma=0.003)
    out = rng.uniform(-4, 4, size=(300, 3)).astype(np.float32)
    allp = np.concatenate([pts, out])
    res = orc.fit_planes(allp, [0, len(allp)], orc.make_params(n_hyp=100, seed=seed))
    P = res["planes"]
    inl = res["inlier"].astype(bool)
    X = allp[inl].astype(np.float64)
    c = X.mean(axis=0)
    _, _, Vt = np.linalg.svd(X - c)
    n = Vt[-1] * np.sign(Vt[-1][2])
    assert abs(float(n @ P["refit_n"][0])) > 1 - 1e-12
    assert abs(P["refit_d"][0] + float(n @ c)) < 1e-9
    # the conditioning the ill-conditioned flag reads: lambda_mid / lambda_min
    # of the centred inlier scatter, from the squared singular values
    sv = np.linalg.svd(X - c, compute_uv=False) ** 2
    assert abs(P["cond"][0] / (sv[1] / sv[2]) - 1) < 1e-8
    assert P["ill_conditioned"][0] == (sv[1] / sv[2] < 10)


def test_refit_flags_ill_conditioned_strip(orc):
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, 2000)
    pts = np.c_[x, rng.uniform(0, 0.001, 2000), rng.normal(0, 0.0005, 2000)].astype(np.float32)
    res = orc.fit_planes(pts, [0, 2000], orc.make_params(n_hyp=64, eps=0.01))
    assert res["planes"]["ill_conditioned"][0] == 1
    X = pts[res["inlier"].astype(bool)].astype(np.float64)
    sv = np.linalg.svd(X - X.mean(axis=0), compute_uv=False) ** 2
    assert res["planes"]["cond"][0] < 10
    assert abs(res["planes"]["cond"][0] / (sv[1] / sv[2]) - 1) < 1e-8


def _brute_hull(P):
    """Hull edges (a, b) with every point left of or on a->b, points on the line
    inside the closed segment; walk them CCW from the lexicographic minimum."""
    P = [tuple(p) for p in np.unique(np.asarray(P, np.int64), axis=0)]
    if len(P) <= 2:
        return sorted(P)
    nxt = {}
    for a, b in itertools.permutations(P, 2):
        ok = True
        for q in P:
            cr = (b[0] - a[0]) * (q[1] - a[1]) - (b[1] - a[1]) * (q[0] - a[0])
            if cr < 0:
                ok = False
                break
            if cr == 0:
                t = (q[0] - a[0]) * (b[0] - a[0]) + (q[1] - a[1]) * (b[1] - a[1])
                if t < 0 or t > (b[0] - a[0]) ** 2 + (b[1] - a[1]) ** 2:
                    ok = False
                    break
        if ok:
            nxt[a] = b
    if not nxt:  # all collinear: the two extreme points
        return [min(P), max(P)]
    start = min(P)
    out = [start]
    while nxt[out[-1]] != start:
        out.append(nxt[out[-1]])
    return out


@pytest.mark.parametrize("seed", range(30))
def test_hull_against_brute_force(orc, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 40))
    span = int(rng.choice([3, 6, 1000, 2 ** 30]))  # small spans force collinear and repeated points
    xy = rng.integers(-span, span + 1, size=(n, 2))
    got = [tuple(p) for p in orc.hull_i32(xy).tolist()]
    assert got == _brute_hull(xy)


def test_hull_special_cases(orc):
    assert orc.hull_i32(np.zeros((0, 2), np.int32)).shape == (0, 2)
    assert orc.hull_i32([[5, 5]]).tolist() == [[5, 5]]
    assert orc.hull_i32([[5, 5], [5, 5], [5, 5]]).tolist() == [[5, 5]]
    assert orc.hull_i32([[3, 1], [1, 1]]).tolist() == [[1, 1], [3, 1]]
    assert orc.hull_i32([[0, 0], [2, 2], [1, 1], [3, 3]]).tolist() == [[0, 0], [3, 3]]
    sq = [[0, 0], [2, 0], [2, 2], [0, 2], [1, 0], [1, 1], [2, 1]]
    assert orc.hull_i32(sq).tolist() == [[0, 0], [2, 0], [2, 2], [0, 2]]


@pytest.mark.parametrize("seed", range(5))
def test_hull_against_qhull(orc, seed):
    rng = np.random.default_rng(seed)
    xy = rng.integers(-2 ** 20, 2 ** 20, size=(3000, 2))
    got = orc.hull_i32(xy)
    qh = ConvexHull(xy.astype(np.float64))
    assert set(map(tuple, got.tolist())) == set(map(tuple, xy[qh.vertices].tolist()))
    # counter-clockwise, strictly convex
    g = got.astype(np.int64)
    a, b, c = g, np.roll(g, -1, 0), np.roll(g, -2, 0)
    cr = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    assert np.all(cr > 0)


def test_plane_hulls_on_config1(orc):
    """Invariants on the config-1 planes: orthonormal right-handed in-plane basis, strictly
    convex CCW hull, every quantised inlier inside or on it, hull vertices are
    quantised inliers, and the projection agrees with float64 to one unit."""
    import synth
    spec, pts, pose = synth.config1()
    m = orc.OracleMap(spec.dims, spec.origin, spec.voxel_size)
    m.integrate(pts, pose)
    res = m.segment(orc.make_params(n_hyp=64))
    P = res["planes"]
    assert len(P["label"]) >= 4
    for k in range(len(P["label"])):
        n = P["ransac_n"][k].astype(np.float64)
        u, v = P["basis_u"][k].astype(np.float64), P["basis_v"][k].astype(np.float64)
        assert abs(u @ n) < 1e-6 and abs(v @ n) < 1e-6 and abs(u @ v) < 1e-6
        assert abs(np.linalg.norm(u) - 1) < 1e-6 and abs(np.linalg.norm(v) - 1) < 1e-6
        # right-handed (u, v, n): counter-clockwise in (X, Y) is counter-clockwise seen from +n
        assert np.linalg.det(np.stack([u, v, n])) > 1 - 1e-6
        # u is e_x x n (no x component) unless n is within 26 deg of e_x, then e_y x n
        assert P["basis_u"][k][0 if abs(n[0]) < 0.9 else 1] == 0.0
        o, cnt = P["point_off"][k], P["n_points"][k]
        cp = res["pts"][o:o + cnt]
        assert np.array_equal(P["origin"][k], cp[0])
        q = cp[res["inlier"][o:o + cnt].astype(bool)].astype(np.float64) - cp[0].astype(np.float64)
        XY = np.rint(np.stack([q @ u, q @ v], 1) * 65536).astype(np.int64)
        H = res["hull"][P["hull_off"][k]:P["hull_off"][k] + P["hull_n"][k]].astype(np.int64)
        assert len(H) >= 3
        # float64 projection vs the quantised hull: every hull vertex is within one unit of an inlier
        d = np.abs(H[:, None, :] - XY[None, :, :]).max(axis=2).min(axis=1)
        assert d.max() <= 1
        a, b = H, np.roll(H, -1, 0)
        c = np.roll(H, -2, 0)
        turn = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
        assert np.all(turn > 0)
        assert tuple(H[0]) == min(map(tuple, H.tolist()))
        # containment with one unit of slack for the float64 re-projection
        ex, ey = b[:, 0] - a[:, 0], b[:, 1] - a[:, 1]
        for p in XY[:: max(1, len(XY) // 400)]:
            cr = ex * (p[1] - a[:, 1]) - ey * (p[0] - a[:, 0])
            assert np.all(cr >= -2 * (np.abs(ex) + np.abs(ey)))


def test_worked_example_two_squares(orc):
    """Two flat 8 x 8-voxel squares (z = 0.125 and z = 0.3125, exact in binary),
    one point at each voxel's centre-ish exact position: closed-form answer."""
    res_m = 0.03125  # 2^-5 m voxels, exact
    pts = []
    for (x0, y0, z) in ((0.0625, 0.0625, 0.125), (0.5, 0.25, 0.3125)):
        for i in range(8):
            for j in range(8):
                pts.append((x0 + (i + 0.5) * res_m, y0 + (j + 0.5) * res_m, z))
    pts = np.array(pts, np.float32)
    m = orc.OracleMap((32, 32, 16), (0, 0, 0), res_m)
    m.integrate(pts)
    out = m.segment(orc.make_params(n_hyp=32, min_cluster=10))
    v, P = out["voxels"], out["planes"]
    assert len(v["vid"]) == 128
    assert np.all(v["n"] == np.float32([0, 0, 1]))
    assert np.all(v["status"] == 2)  # corners have exactly N = 3 neighbours
    assert P["n_points"].tolist() == [64, 64] and P["inlier_count"].tolist() == [64, 64]
    for k, z in enumerate((0.125, 0.3125)):
        assert P["refit_n"][k].tolist() == [0.0, 0.0, 1.0]
        assert P["refit_d"][k] == -z
        assert P["hull_n"][k] == 4
        H = out["hull"][P["hull_off"][k]:P["hull_off"][k] + 4]
        # the four extreme voxel centres, 7 voxels apart: a 7 * 2^-5 m square = 14336 units
        side = 7 * res_m * 65536
        assert sorted(np.abs(H - H.min(axis=0)).max(axis=0).tolist()) == [side, side]
