"""Pins for the oracle's voxel update (Sec. III.B, Eq. 1).

The reading under test: p' = R p + t by an fma chain, voxel index
floor((p' - origin) * inv_res), points outside the grid dropped, and per-voxel
exact sums of rint(d * 2^20) plus a count; the mean is the exact integer mean
rounded half up, then mu = origin + M * 2^-20."""
from fractions import Fraction

import numpy as np
import pytest


def _ijk_key(ijk):
    """Brick-major order key: (bz, by, bx, lz, ly, lx)."""
    i, j, k = ijk[..., 0], ijk[..., 1], ijk[..., 2]
    return np.stack([k // 8, j // 8, i // 8, k % 8, j % 8, i % 8], axis=-1)


def _vid_to_ijk(vid, dims):
    nbx = (dims[0] + 7) // 8
    nby = (dims[1] + 7) // 8
    b, l = vid // 512, vid % 512
    return np.stack([(b % nbx) * 8 + l % 8, ((b // nbx) % nby) * 8 + (l // 8) % 8,
                     (b // (nbx * nby)) * 8 + l // 64], axis=-1).astype(np.int64)


def test_exact_binning_and_sums(orc):
    """Offsets that are exact multiples of 2^-20: binning and sums follow in integers."""
    rng = np.random.default_rng(1)
    dims = (16, 16, 16)
    m = orc.OracleMap(dims, (0, 0, 0), 0.02)
    kmax = 16 * 2 ** 20 // 50  # k * 50 < 2^24: the float32 product d * 50 is exact
    K = rng.integers(0, kmax, size=(5000, 3))
    pts = (K.astype(np.float64) * 2.0 ** -20).astype(np.float32)
    assert np.array_equal(pts.astype(np.float64) * 2 ** 20, K)  # the inputs are exact
    m.integrate(pts)
    n_in, n_drop = m.counts()
    assert (n_in, n_drop) == (5000, 0)
    vid, S, c = m.export_sums()
    ijk = _vid_to_ijk(vid.astype(np.int64), dims)
    exp_ijk = (K * 50) // 2 ** 20
    # expected counts and sums by integer arithmetic
    keys, inv = np.unique(exp_ijk, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    cnt = np.bincount(inv)
    sums = np.stack([np.bincount(inv, weights=K[:, a]).astype(np.int64) for a in range(3)], axis=1)
    order = np.lexsort(_ijk_key(keys).T[::-1])
    assert np.array_equal(ijk, keys[order])
    assert np.array_equal(c, cnt[order])
    assert np.array_equal(S, sums[order])


def test_vid_order_is_brick_major(orc):
    rng = np.random.default_rng(2)
    dims = (20, 13, 9)  # ragged bricks on every axis
    m = orc.OracleMap(dims, (0, 0, 0), 0.05)
    ijk = np.stack([rng.integers(0, d, 3000) for d in dims], axis=1)
    pts = ((ijk + 0.5) * 0.05).astype(np.float32)
    m.integrate(pts)
    vid, _, _ = m.export_sums()
    got = _vid_to_ijk(vid.astype(np.int64), dims)
    uniq = np.unique(ijk, axis=0)
    assert got.shape == uniq.shape
    order = np.lexsort(_ijk_key(uniq).T[::-1])
    assert np.array_equal(got, uniq[order])
    assert np.all(np.diff(vid.astype(np.int64)) > 0)


def test_pose_row_major_rotation(orc):
    """A 90-degree yaw with an exactly representable translation: integrating
    with the pose equals integrating the transformed points with identity."""
    rng = np.random.default_rng(3)
    pts = rng.uniform(-0.4, 0.4, size=(4000, 3)).astype(np.float32)
    t = np.float32([0.5, 0.25, 0.125])
    pose = np.array([0, -1, 0, t[0], 1, 0, 0, t[1], 0, 0, 1, t[2]], np.float32)
    a = orc.OracleMap((64, 48, 40), (0, -0.2, -0.3), 0.02)
    a.integrate(pts, pose)
    moved = np.stack([t[0] - pts[:, 1], pts[:, 0] + t[1], pts[:, 2] + t[2]], axis=1).astype(np.float32)
    b = orc.OracleMap((64, 48, 40), (0, -0.2, -0.3), 0.02)
    b.integrate(moved)
    for x, y in zip(a.export_sums(), b.export_sums()):
        assert np.array_equal(x, y)
    assert a.counts() == b.counts()
    # the transposed pose gives a different map: the layout is really row-major
    c = orc.OracleMap((64, 48, 40), (0, -0.2, -0.3), 0.02)
    pose_t = np.array([0, 1, 0, t[0], -1, 0, 0, t[1], 0, 0, 1, t[2]], np.float32)
    c.integrate(pts, pose_t)
    assert c.counts() != a.counts() or not np.array_equal(c.export_sums()[0], a.export_sums()[0])


def test_drops_nan_inf_and_out_of_extent(orc):
    m = orc.OracleMap((10, 10, 10), (0, 0, 0), 0.05)
    good = np.array([[0.01, 0.01, 0.01], [0.49, 0.49, 0.49]], np.float32)
    bad = np.array([[np.nan, 0.1, 0.1], [0.1, np.inf, 0.1], [0.1, 0.1, -np.inf], [-0.001, 0.1, 0.1],
                    [0.5, 0.1, 0.1], [0.1, 0.5, 0.1], [0.1, 0.1, 0.50001], [1e30, 0, 0]], np.float32)
    m.integrate(np.concatenate([good, bad]))
    assert m.counts() == (2, len(bad))
    vid, S, c = m.export_sums()
    assert c.tolist() == [1, 1]


def test_face_rule_floor(orc):
    """A point exactly on a voxel face belongs to the upper voxel (floor)."""
    m = orc.OracleMap((10, 10, 10), (0, 0, 0), 0.05)
    below = np.nextafter(np.float32(0.25), np.float32(0))
    pts = np.array([[0.25, 0.01, 0.01], [below, 0.01, 0.01]], np.float32)
    m.integrate(pts)
    vid, _, _ = m.export_sums()
    ijk = _vid_to_ijk(vid.astype(np.int64), (10, 10, 10))
    assert sorted(ijk[:, 0].tolist()) == [4, 5]


def test_order_independence(orc):
    rng = np.random.default_rng(4)
    pts = rng.uniform(0, 0.6, size=(20000, 3)).astype(np.float32)
    a = orc.OracleMap((32, 32, 32), (0, 0, 0), 0.02)
    a.integrate(pts)
    b = orc.OracleMap((32, 32, 32), (0, 0, 0), 0.02)
    b.integrate(pts[rng.permutation(len(pts))])
    for x, y in zip(a.export_sums(), b.export_sums()):
        assert np.array_equal(x, y)


def test_numpy_histogram_config1(orc):
    """Counts and sums of the config-1 scene against numpy's floor / rint."""
    import synth
    spec, pts, pose = synth.config1()
    m = orc.OracleMap(spec.dims, spec.origin, spec.voxel_size)
    m.integrate(pts, pose)
    d = pts - np.asarray(spec.origin, np.float32)
    f = np.floor(d * np.float32(1 / spec.voxel_size))
    ok = np.all((f >= 0) & (f < np.asarray(spec.dims, np.float32)), axis=1)
    ijk = f[ok].astype(np.int64)
    F = np.rint(d[ok] * np.float32(2 ** 20)).astype(np.int64)
    keys, inv = np.unique(ijk, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    order = np.lexsort(_ijk_key(keys).T[::-1])
    vid, S, c = m.export_sums()
    assert np.array_equal(_vid_to_ijk(vid.astype(np.int64), spec.dims), keys[order])
    assert np.array_equal(c, np.bincount(inv)[order])
    for a in range(3):
        assert np.array_equal(S[:, a], np.bincount(inv, weights=F[:, a]).astype(np.int64)[order])
    assert m.counts() == (int(ok.sum()), int((~ok).sum()))


@pytest.mark.parametrize("ks", [[10, 11], [10, 12], [3, 4, 4], [7], [0, 1, 1, 1]])
def test_mean_rounds_half_up(orc, ks):
    """M = floor(S / c + 1/2) exactly; mu = origin + M * 2^-20 in FP32."""
    origin = np.float32(0.125)
    m = orc.OracleMap((8, 8, 8), (origin, origin, origin), 0.05)
    base = 40000  # inside voxel 0 (0.05 m ~ 52429 units)
    pts = np.array([[(base + k) * 2.0 ** -20 + 0.125] * 3 for k in ks], np.float64).astype(np.float32)
    assert np.array_equal((pts.astype(np.float64) - 0.125) * 2 ** 20, np.array([[base + k] * 3 for k in ks]))
    m.integrate(pts)
    res = m.segment(orc.make_params(min_cluster=1))
    v = res["voxels"]
    S = sum(base + k for k in ks)
    exp_M = int(Fraction(S, len(ks)) + Fraction(1, 2))  # floor for a positive value
    assert v["M"].tolist() == [[exp_M] * 3]
    assert v["mu"][0, 0] == np.float32(origin + np.float32(exp_M * 2.0 ** -20))
