"""Pins of the oracle's robot-centric map (Sec. III.B: the map's centre
follows the robot), read as a window over world-anchored voxel keys moved in
whole bricks:

* a numpy replay, written independently, of keying, window membership,
  eviction and the re-anchored integer sums over a sequence of integrations
  and scrolls matches the oracle's voxel ids, sums and counts exactly;
* a kept voxel's world mean (S / C + A, exact) is unchanged by a scroll;
  scrolling there and back restores every voxel that never left;
* the scroll target puts the centre's key in the middle brick of the window;
* ray-cast clearing (Eq. 2) in a scrolled window clears the voxels that a
  brute-force walk over world keys clears;
* the mean positions of the segmentation follow po + M 2^-20 and agree with
  the unscrolled map's to rounding."""
import numpy as np
import pytest

import synth

N = (48, 40, 24)
ORIGIN = np.float32([0.3, -0.2, 0.1])
RES = 0.02


def _vid(g, n):
    """Brick-major voxel id (8^3 bricks, x fastest) of window coordinates g[..., 3]."""
    nbx, nby = (n[0] + 7) // 8, (n[1] + 7) // 8
    g = np.asarray(g, np.int64)
    b = ((g[..., 2] >> 3) * nby + (g[..., 1] >> 3)) * nbx + (g[..., 0] >> 3)
    return b * 512 + (((g[..., 2] & 7) * 8 + (g[..., 1] & 7)) * 8 + (g[..., 0] & 7))


class Replay:
    """World-keyed voxel sums (rint(d 2^20), int64) with a window of keys."""

    def __init__(self):
        self.inv = np.float32(1.0 / RES)
        self.w = np.zeros(3, np.int64)
        self.vox = {}

    def integrate(self, p):
        d = (p.astype(np.float32) - ORIGIN).astype(np.float32)
        key = np.floor((d * self.inv).astype(np.float32)).astype(np.int64)
        F = np.rint((d * np.float32(1048576.0)).astype(np.float32)).astype(np.int64)
        inside = np.all((key >= self.w) & (key < self.w + np.array(N)), axis=1)
        for k, f in zip(map(tuple, key[inside]), F[inside]):
            s, c = self.vox.get(k, (np.zeros(3, np.int64), 0))
            self.vox[k] = (s + f, c + 1)

    def scroll(self, shift):
        self.w = self.w + 8 * np.asarray(shift, np.int64)
        hi = self.w + np.array(N)
        self.vox = {k: v for k, v in self.vox.items() if np.all((np.array(k) >= self.w) & (np.array(k) < hi))}

    def expected(self):
        A = np.array([int(np.floor(float(w) * 1048576.0 / float(self.inv))) for w in self.w], np.int64)
        keys = np.array(sorted(self.vox), np.int64).reshape(-1, 3)
        vid = _vid(keys - self.w, N)
        S = np.array([self.vox[tuple(k)][0] for k in keys], np.int64).reshape(-1, 3)
        C = np.array([self.vox[tuple(k)][1] for k in keys], np.uint32)
        S = S - C[:, None].astype(np.int64) * A
        o = np.argsort(vid)
        return vid[o].astype(np.uint32), S[o], C[o], A


def _cloud(rng, n, lo, hi):
    return rng.uniform(lo, hi, (n, 3)).astype(np.float32)


def test_replay_of_integrations_and_scrolls(orc):
    rng = np.random.default_rng(0)
    m = orc.OracleMap(N, ORIGIN, RES)
    r = Replay()
    shifts = [(1, 0, 0), (0, -1, 1), (-2, 1, 0), (3, 2, -1), (0, 0, 0), (-1, -1, -1)]
    for sh in [None] + shifts:
        if sh is not None:
            m.scroll(sh)
            r.scroll(sh)
        # points over the current window and 0.1 m beyond it (some are dropped)
        lo = ORIGIN + r.w * RES - 0.1
        p = (lo + rng.uniform(0, 1, (6000, 3)) * (np.array(N) * RES + 0.2)).astype(np.float32)
        m.integrate(p)
        r.integrate(p)
    vid, S, C = m.export_sums()
    evid, eS, eC, A = r.expected()
    assert len(vid) > 5000
    assert np.array_equal(vid, evid) and np.array_equal(C, eC) and np.array_equal(S, eS)
    win = m.window()
    assert np.array_equal(win["offset"], r.w) and np.array_equal(win["anchor"], A)
    assert np.array_equal(win["position_origin"],
                          np.float32([float(o) + a / 1048576.0 for o, a in zip(ORIGIN.astype(np.float64), A)]))


def test_kept_voxels_keep_their_world_means_and_there_and_back_restores(orc):
    rng = np.random.default_rng(1)
    m = orc.OracleMap(N, ORIGIN, RES)
    m.integrate(_cloud(rng, 20000, 0.3, 1.2))
    vid0, S0, C0 = m.export_sums()
    A0 = m.window()["anchor"]
    m.scroll((1, -1, 0))
    vid1, S1, C1 = m.export_sums()
    A1 = m.window()["anchor"]
    assert 0 < len(vid1) < len(vid0)
    # world-anchored sums S + C A: the same multiset of (sum, count) pairs for the kept voxels
    w0 = {(tuple(s + c * A0), c) for s, c in zip(S0.tolist(), C0.tolist())}
    w1 = {(tuple(s + c * A1), c) for s, c in zip(S1.tolist(), C1.tolist())}
    assert w1 <= w0
    m.scroll((-1, 1, 0))
    vid2, S2, C2 = m.export_sums()
    keep = np.isin(vid0, vid2)
    assert keep.sum() == len(vid2) == len(vid1)
    assert np.array_equal(vid0[keep], vid2) and np.array_equal(S0[keep], S2) and np.array_equal(C0[keep], C2)
    assert np.array_equal(m.window()["anchor"], A0) and np.array_equal(m.window()["offset"], [0, 0, 0])
    assert m.window()["voxels_evicted"] == len(vid0) - len(vid1)


def test_scroll_target_centres_the_window(orc):
    rng = np.random.default_rng(2)
    m = orc.OracleMap(N, ORIGIN, RES)
    inv = np.float32(1.0 / RES)
    for _ in range(50):
        c = rng.uniform(-3, 3, 3).astype(np.float32)
        m.scroll_to(c)
        key = np.floor(((c - ORIGIN).astype(np.float32) * inv).astype(np.float32)).astype(np.int64)
        w = m.window()["offset"].astype(np.int64)
        assert np.all(w % 8 == 0)
        assert np.all((key - w >= np.array(N) // 2) & (key - w < np.array(N) // 2 + 8)), (key, w)
        assert np.array_equal(m.scroll_target(c), [0, 0, 0])


def test_clearing_in_a_scrolled_window_follows_world_keys(orc):
    """A point at every voxel centre of the window; after a scroll, axis-aligned
    rays clear exactly the world keys between the sensor's and the point's."""
    n = (24, 24, 24)
    m = orc.OracleMap(n, (0.0, 0.0, 0.0), 0.1)
    m.scroll((1, 2, -1))
    w = m.window()["offset"]
    g = (np.stack(np.meshgrid(*[np.arange(x) for x in n], indexing="ij"), -1).reshape(-1, 3) + w + 0.5) * 0.1
    m.integrate(g.astype(np.float32))
    before = set(m.export_sums()[0].tolist())
    t = ((w + np.array([2, 5, 7]) + 0.5) * 0.1).astype(np.float32)  # sensor in window voxel (2, 5, 7)
    p = (t + np.float32([1.5, 0.0, 0.0])).astype(np.float32)  # 15 voxels along +x
    k = m.clear_rays((p - t).reshape(1, 3), np.array([1, 0, 0, t[0], 0, 1, 0, t[1], 0, 0, 1, t[2]], np.float32))
    gone = before - set(m.export_sums()[0].tolist())
    assert k == 15 and gone == {int(_vid(np.array([x, 5, 7]), n)) for x in range(2, 17)}
    # a sensor whose key lies outside the window casts nothing
    t2 = ((w - 3) * 0.1).astype(np.float32)
    assert m.clear_rays(np.zeros((1, 3), np.float32), np.array([1, 0, 0, t2[0], 0, 1, 0, t2[1], 0, 0, 1, t2[2]],
                                                               np.float32)) == 0


def test_segmentation_positions_follow_the_window_origin(orc):
    _, pts, _ = synth.config1()
    dims, origin = (64, 64, 40), (-0.2, -0.2, -0.2)  # 1.28 x 1.28 x 0.8 m around the stair and ramp
    a = orc.OracleMap(dims, origin, 0.02)
    b = orc.OracleMap(dims, origin, 0.02)
    for m in (a, b):
        m.integrate(pts)
    b.scroll((0, 0, 1))  # up one brick (0.16 m): the scene stays inside
    ra, rb = a.segment(orc.make_params()), b.segment(orc.make_params())
    va, vb = ra["voxels"], rb["voxels"]
    assert len(va["vid"]) == len(vb["vid"]) and b.window()["voxels_evicted"] == 0
    assert np.abs(va["mu"] - vb["mu"]).max() < 2e-7  # po + M 2^-20 rounds differently, by an ulp
    po, A = b.window()["position_origin"], b.window()["anchor"]
    vid, S, C = b.export_sums()
    M = ((2 * S + C[:, None]) // (2 * C[:, None].astype(np.int64))).astype(np.int32)
    assert np.array_equal(vb["mu"], (po + M.astype(np.float32) * np.float32(2.0 ** -20)).astype(np.float32))
    assert len(ra["planes"]["label"]) == len(rb["planes"]["label"])


# Windows whose low face lies far from the base origin (0.01, 0.02 and 0.05 m
# voxels, both signs of the offset): there, FP32 points keyed into the window's
# first voxel row can quantise one 2^-20 m unit below the window's anchor, so
# their sums are negative.
FAR_WINDOWS = [(0.01, (2104, -2072, 2104)), (0.05, (544, -528, -528)), (0.02, (-1040, 1056, -1040))]
FAR_DIMS = (32, 32, 32)


@pytest.mark.parametrize("res,w", FAR_WINDOWS)
def test_far_window_inputs_reach_negative_sums(orc, res, w):
    """The far-window inputs of the GPU test really contain points keyed into
    the window whose quantised offset from the anchor is -1, on every axis,
    in voxels holding many points and in single-point voxels.  Checked two
    ways: the oracle's exported sums, and a direct numpy evaluation of the
    keying and quantisation (FP32 floor of d * inv_res; rint of d * 2^20 less
    the anchor floor(w * 2^20 / inv_res) in double)."""
    m = orc.OracleMap(FAR_DIMS, (0.0, 0.0, 0.0), res)
    m.scroll(np.asarray(w, np.int32) // 8)
    assert np.array_equal(m.window()["offset"], w)
    p = synth.far_window_points(w, FAR_DIMS, res)
    m.integrate(p)
    vid, S, c = m.export_sums()
    inv = np.float32(1.0 / res)
    for a in range(3):
        assert (S[:, a] < 0).any(), f"axis {a}: no negative sum"
        assert ((S[:, a] == -1) & (c == 1)).any(), f"axis {a}: no single-point voxel at -1"
        assert ((S[:, a] < 0) & (c > 1)).any(), f"axis {a}: no negative sum over several points"
        key = np.floor((p[:, a] * inv).astype(np.float32)).astype(np.int64)
        anchor = int(np.floor(w[a] * 1048576.0 / float(inv)))
        F = np.rint((p[:, a] * np.float32(1048576.0)).astype(np.float32)).astype(np.int64) - anchor
        inside = np.ones(len(p), bool)
        for b in range(3):
            kb = np.floor((p[:, b] * inv).astype(np.float32)).astype(np.int64)
            inside &= (kb >= w[b]) & (kb < w[b] + FAR_DIMS[b])
        assert ((key == w[a]) & (F == -1) & inside).any()
