"""Pins for the oracle's cluster RANSAC (Sec. III.C, stages a-c) and its random
stream (Philox4x64-10 of Salmon et al., SC'11).

* The generator is compared word for word with numpy's independent Philox
  implementation (numpy advances its counter by one before each block).
* Sample indices and hypothesis planes are re-derived from numpy's stream.
* Every hypothesis count is recounted in float64; points within rounding of
  the threshold are decided by exact binary32 evaluation.
* Selection is max count, lowest hypothesis index on ties.
* Exhaustive enumeration of all triples bounds the RANSAC optimum on small
  clusters."""
import itertools
import math

import numpy as np
import pytest

from fp32exact import fmaf, mulf


def _numpy_philox(ctr, key):
    """numpy's Philox block for counter ``ctr``: numpy increments its 256-bit
    counter before generating, so start it one below."""
    v = sum(int(x) << (64 * i) for i, x in enumerate(ctr))
    v = (v - 1) % (1 << 256)
    words = [(v >> (64 * i)) & ((1 << 64) - 1) for i in range(4)]
    # explicit uint64 arrays: a list of large Python ints would pass through float64
    bg = np.random.Philox(counter=np.array(words, dtype=np.uint64),
                          key=np.array([int(key[0]), int(key[1])], dtype=np.uint64))
    return bg.random_raw(4).astype(np.uint64)


@pytest.mark.parametrize("seed", range(4))
def test_philox_matches_numpy(orc, seed):
    rng = np.random.default_rng(seed)
    for _ in range(200):
        ctr = rng.integers(0, 2 ** 63, size=4, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, 4, dtype=np.uint64)
        key = rng.integers(0, 2 ** 63, size=2, dtype=np.uint64)
        assert np.array_equal(orc.philox4x64(ctr, key), _numpy_philox(ctr, key))


def _cluster(seed, n, outliers=0.2, sigma=0.002):
    rng = np.random.default_rng(seed)
    t, a = rng.uniform(0, 0.6), rng.uniform(0, 2 * math.pi)
    nrm = np.array([math.sin(t) * math.cos(a), math.sin(t) * math.sin(a), math.cos(t)])
    u = np.cross([1.0, 0, 0], nrm); u /= np.linalg.norm(u)
    w = np.cross(nrm, u)
    s = rng.uniform(-0.5, 0.5, size=(n, 2))
    p = rng.uniform(-2, 2, 3) + s[:, :1] * u + s[:, 1:] * w + rng.normal(0, sigma, (n, 1)) * nrm
    k = int(outliers * n)
    p[:k] += rng.normal(0, 0.1, size=(k, 3))
    return p[rng.permutation(n)].astype(np.float32)


def _exact_count(pts, plane, eps):
    n = plane[:3].astype(np.float64)
    d = float(plane[3])
    dist = np.abs(pts.astype(np.float64) @ n + d)
    eps = float(np.float32(eps))
    cnt = int((dist <= eps).sum())
    near = np.nonzero(np.abs(dist - eps) < 1e-6)[0]
    for k in near:  # decide by the exact binary32 fma chain
        p = pts[k]
        r = fmaf(plane[2], p[2], fmaf(plane[1], p[1], fmaf(plane[0], p[0], plane[3])))
        exact = abs(float(r)) <= eps
        cnt += int(exact) - int(dist[k] <= eps)
    return cnt


@pytest.mark.parametrize("n,label,seed", [(3, 0, 1), (7, 5, 2), (200, 17, 3), (1500, 123456, 4), (40, 2 ** 31, 5)])
def test_hypotheses_counts_and_selection(orc, n, label, seed):
    pts = _cluster(seed, n)
    H, eps, key_seed = 128, 0.01, 987654321
    counts, planes, best = orc.ransac_counts(pts, label, H, key_seed, eps)
    for h in range(H):
        r = _numpy_philox([label, h, 0, 0], [key_seed, 0])
        idx = [(int(x) * n) >> 64 for x in r[:3]]
        if len(set(idx)) < 3:
            assert counts[h] == -1
            continue
        p0, p1, p2 = (pts[i].astype(np.float64) for i in idx)
        c = np.cross(p1 - p0, p2 - p0)
        if np.linalg.norm(c) == 0:
            assert counts[h] == -1
            continue
        assert counts[h] >= 0
        nr = planes[h, :3].astype(np.float64)
        assert abs(np.linalg.norm(nr) - 1) < 1e-6
        if np.linalg.norm(c) > 1e-4:
            assert abs(abs(nr @ (c / np.linalg.norm(c))) - 1) < 1e-5
        for p in (p0, p1, p2):
            assert abs(nr @ p + planes[h, 3]) < 1e-5
        assert counts[h] == _exact_count(pts, planes[h], eps)
    valid = counts >= 0
    if valid.any():
        assert best == int(np.argmax(np.where(valid, counts, -1)))  # argmax takes the lowest index
        assert counts[best] == counts.max()
    else:
        assert best == -1


def test_degenerate_clusters(orc):
    # two points: every sample repeats an index
    counts, _, best = orc.ransac_counts(np.zeros((2, 3), np.float32), 3, 32, 1, 0.01)
    assert best == -1 and np.all(counts == -1)
    # collinear points: every cross product is zero
    line = np.stack([np.arange(50) * 0.01, np.zeros(50), np.zeros(50)], 1).astype(np.float32)
    counts, _, best = orc.ransac_counts(line, 3, 32, 1, 0.01)
    assert best == -1 and np.all(counts == -1)


def test_planted_plane_every_point_inlier(orc):
    """Points exactly on z = 0.375: a valid sample gives n = (0, 0, +-1) up to
    the one rounding of 1/sqrt, and every point lies within rounding of the plane."""
    rng = np.random.default_rng(9)
    xy = rng.uniform(-1, 1, size=(500, 2))
    pts = np.c_[xy, np.full(500, 0.375)].astype(np.float32)
    counts, planes, best = orc.ransac_counts(pts, 7, 64, 3, 0.01)
    valid = counts >= 0
    assert valid.sum() > 50
    assert np.all(counts[valid] == 500)
    assert np.all(np.abs(np.abs(planes[valid, 2]) - 1) <= 2 ** -23) and np.all(planes[valid, :2] == 0)
    assert best == int(np.argmax(valid))


@pytest.mark.parametrize("seed", range(5))
def test_exhaustive_bound_small_clusters(orc, seed):
    """Best RANSAC count <= the best over all C(n,3) triples (float64 + exact
    tie-breaking); with 60 hypotheses on 12 clustered inliers it reaches it."""
    rng = np.random.default_rng(100 + seed)
    n_in, n_out = 12, 10
    pts_in = np.c_[rng.uniform(0, 0.2, (n_in, 2)), np.full(n_in, 0.5)] + rng.normal(0, 0.001, (n_in, 3))
    pts_out = rng.uniform(0, 0.5, (n_out, 3))
    pts = np.concatenate([pts_in, pts_out])[rng.permutation(n_in + n_out)].astype(np.float32)
    eps = 0.01
    best_all = 0
    for i, j, k in itertools.combinations(range(len(pts)), 3):
        p0, p1, p2 = (pts[x].astype(np.float64) for x in (i, j, k))
        c = np.cross(p1 - p0, p2 - p0)
        nn = np.linalg.norm(c)
        if nn == 0:
            continue
        nrm = c / nn
        d = -nrm @ p0
        best_all = max(best_all, int((np.abs(pts.astype(np.float64) @ nrm + d) <= eps + 1e-6).sum()))
    counts, planes, best = orc.ransac_counts(pts, seed, 60, 11, eps)
    assert counts[best] <= best_all
    assert counts[best] >= n_in


def test_fit_planes_inliers_follow_the_selected_plane(orc):
    pts = np.concatenate([_cluster(1, 300), _cluster(2, 50), _cluster(3, 3)])
    off = np.array([0, 300, 350, 353], np.uint32)
    prm = orc.make_params(n_hyp=64, seed=5)
    res = orc.fit_planes(pts, off, prm, labels=[11, 12, 13])
    P = res["planes"]
    assert P["label"].tolist() == [11, 12, 13]
    for k in range(3):
        o, n = int(off[k]), int(off[k + 1] - off[k])
        counts, planes, best = orc.ransac_counts(pts[o:o + n], 11 + k, 64, 5, 0.01)
        assert best == P["best_h"][k]
        if best < 0:
            continue
        assert np.array_equal(P["ransac_n"][k], planes[best, :3]) and P["ransac_d"][k] == planes[best, 3]
        assert P["inlier_count"][k] == counts[best] == res["inlier"][o:o + n].sum()
