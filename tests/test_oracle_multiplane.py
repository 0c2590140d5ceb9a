"""Pins of the oracle's sequential multi-plane extraction per cluster
(planes_per_cluster > 1): round q + 1 fits the points of round q that are not
its inliers, with the Philox counter (label, h, q + 1, 0).

* Two separated planted planes in one cluster come out as round 0 and round
  1 with their exact inlier sets and the analytic normals.
* Round 1's selected hypothesis is re-derived from numpy's Philox stream on
  the remaining points, counted in float64 (exact binary32 at the threshold).
* The stopping rules: too few remaining points, too few inliers, no plane.
* A 10 deg ramp joined to a floor (one cluster under Algorithm 1) comes out
  as the cluster's second plane.
* planes_per_cluster = 1 is exactly the single-plane fit; threads change
  nothing."""
import math

import numpy as np

import synth
from test_oracle_ransac import _exact_count, _numpy_philox


def _two_planes(n_a=2000, n_b=1000, seed=0):
    rng = np.random.default_rng(seed)
    a = np.c_[rng.uniform(0, 1, (n_a, 2)), np.zeros(n_a)]                      # z = 0, x in [0, 1]
    xb = rng.uniform(1.5, 2.5, n_b)
    b = np.c_[xb, rng.uniform(0, 1, n_b), 0.2 + 0.1 * xb]                       # z = 0.2 + 0.1 x
    return np.concatenate([a, b]).astype(np.float32)


def _fit(orc, pts, P, n_hyp=100, seed=3, label=7, min_cluster=50):
    off = np.array([0, len(pts)], np.uint32)
    return orc.fit_planes(pts, off, orc.make_params(n_hyp=n_hyp, seed=seed, planes_per_cluster=P,
                                                    min_cluster=min_cluster), labels=np.array([label], np.uint32))


def test_two_planted_planes_come_out_in_two_rounds(orc):
    pts = _two_planes()
    r = _fit(orc, pts, P=3)
    p = r["planes"]
    assert list(p["round"]) == [0, 1] and list(p["label"]) == [7, 7]
    assert list(p["inlier_count"]) == [2000, 1000]
    assert list(p["n_points"]) == [3000, 1000]
    n_b = np.array([-0.1, 0.0, 1.0]) / math.sqrt(1.01)
    assert abs(abs(float(p["refit_n"][0] @ [0, 0, 1.0])) - 1) < 1e-9
    assert abs(abs(float(p["refit_n"][1] @ n_b)) - 1) < 1e-9
    # round 1's hull origin is the first remaining point (the first point of plane b)
    assert np.array_equal(p["origin"][1], pts[2000])


def test_round_one_follows_the_philox_stream_on_the_remaining_points(orc):
    rng = np.random.default_rng(5)
    pts = _two_planes(1500, 900, seed=1)
    pts = (pts + rng.normal(0, 0.002, pts.shape)).astype(np.float32)
    label, seed, eps, H = 11, 99, np.float32(0.01), 64
    r = _fit(orc, pts, P=2, n_hyp=H, seed=seed, label=label)
    p = r["planes"]
    assert list(p["round"]) == [0, 1]
    inl0 = r["inlier"].astype(bool)
    rest = pts[~inl0]
    n = len(rest)
    assert int(p["n_points"][1]) == n
    best, best_cnt = -1, -1
    for h in range(H):
        w = _numpy_philox([label, h, 1, 0], [seed, 0])
        idx = [(int(x) * n) >> 64 for x in w[:3]]
        if len(set(idx)) < 3:
            continue
        p0, p1, p2 = (rest[i].astype(np.float64) for i in idx)
        c = np.cross(p1 - p0, p2 - p0)
        if not np.linalg.norm(c) > 0:
            continue
        nrm = c / np.linalg.norm(c)
        plane = np.r_[nrm, -nrm @ p0].astype(np.float32)
        cnt = _exact_count(rest, plane, eps)
        if cnt > best_cnt:
            best, best_cnt = h, cnt
    assert int(p["best_h"][1]) == best
    # the count is the oracle's exact one; an independent float64 recount can
    # differ only by the rounding of the sampled plane (a point or two)
    assert abs(int(p["inlier_count"][1]) - best_cnt) <= 2


def test_stopping_rules(orc):
    pts = _two_planes(2000, 40)           # 40 points left: fewer than min_cluster = 50
    assert list(_fit(orc, pts, P=3)["planes"]["round"]) == [0]
    pts = _two_planes(2000, 1000)
    assert list(_fit(orc, pts, P=3, min_cluster=2500)["planes"]["round"]) == [0]  # round 0: 2000 < 2500 inliers
    line = np.c_[np.linspace(0, 1, 300), np.zeros(300), np.zeros(300)]
    pts = np.concatenate([_two_planes(2000, 0), line + [0, 5.0, 1.0]]).astype(np.float32)
    r = _fit(orc, pts, P=3)              # the 300 remaining points are collinear: no plane in round 1
    assert list(r["planes"]["round"]) == [0]


def _floor_and_ramp(seed=0, n=20000):
    """A 10 deg ramp rising from a floor (1.2 x 1 m each, joined along x = 1.2):
    normals within 15 deg, so CCL joins them into one cluster (Algorithm 1)."""
    rng = np.random.default_rng(seed)
    half = n // 2
    f = np.c_[rng.uniform(0.0, 1.2, half), rng.uniform(0, 1, half), np.zeros(half)]
    t = rng.uniform(0.0, 1.2, half)
    a = math.radians(10.0)
    r = np.c_[1.2 + t * math.cos(a), rng.uniform(0, 1, half), t * math.sin(a)]
    p = np.concatenate([f, r]) + rng.normal(0, 0.002, (n, 3))
    return synth.MapSpec((130, 60, 20), (0.0, -0.1, -0.05), 0.02), p.astype(np.float32)


def test_a_ramp_merged_with_the_floor_comes_out_as_a_second_plane(orc):
    spec, pts = _floor_and_ramp()
    m = orc.OracleMap(spec.dims, spec.origin, spec.voxel_size)
    m.integrate(pts)
    one = m.segment(orc.make_params(n_hyp=64))
    two = m.segment(orc.make_params(n_hyp=64, planes_per_cluster=2))
    p1, p2 = one["planes"], two["planes"]
    assert len(p1["label"]) == 1  # one cluster: floor and ramp joined
    assert list(p2["round"]) == [0, 1]
    for key in ("best_h", "inlier_count", "hull_n", "refit_n"):  # round 0 is the single-plane fit
        assert np.array_equal(p2[key][:1], p1[key])
    tilts = sorted(math.degrees(math.acos(min(1.0, abs(float(n[2]))))) for n in p2["refit_n"])
    assert tilts[0] < 0.5 and abs(tilts[1] - 10.0) < 0.5, tilts


def test_threads_change_nothing_with_several_rounds(orc):
    spec, pts = _floor_and_ramp(seed=2)
    spec1, pts1, _ = synth.config1()
    out = []
    for th in (1, 4):
        orc.set_threads(th)
        try:
            m = orc.OracleMap(spec.dims, spec.origin, spec.voxel_size)
            m.integrate(pts)
            m.integrate(pts1 + np.float32([0.5, 0.0, 0.0]))  # more clusters beside the floor and ramp
            out.append(m.segment(orc.make_params(n_hyp=64, planes_per_cluster=3)))
        finally:
            orc.set_threads(1)
    assert (out[0]["planes"]["round"] > 0).any()
    for key in ("label", "round", "best_h", "inlier_count", "refit_n", "hull_off", "hull_n"):
        assert np.array_equal(out[0]["planes"][key], out[1]["planes"][key]), key
    assert np.array_equal(out[0]["hull"], out[1]["hull"])
