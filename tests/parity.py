"""Comparison helpers for the GPU-vs-oracle parity tests.

Bit-exact: voxel ids, sums and counts; normals, N and status; CCL labels;
cluster point lists; RANSAC hypothesis index, plane, inlier sets; in-plane
basis, origin and quantised hulls.  Tolerance (the refit): normal within
1e-4 rad and offset within 1e-5 m, planes the oracle flags ill-conditioned
excluded; the GPU's ill-conditioned flag equals the oracle's wherever the
oracle's lambda_mid / lambda_min lies outside [9, 11]."""
import math

import numpy as np

REFIT_ANGLE_TOL = 1e-4   # rad
REFIT_OFFSET_TOL = 1e-5  # m


def angle(a, b):
    """Angle between two directions (sign ignored), well conditioned near 0."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    a = a / np.linalg.norm(a)
    b = b / np.linalg.norm(b)
    return math.atan2(float(np.linalg.norm(np.cross(a, b))), abs(float(a @ b)))


def bits(a):
    a = np.ascontiguousarray(a)
    return a.view(np.uint32) if a.dtype == np.float32 else a


def assert_same(a, b, what):
    a, b = np.asarray(a), np.asarray(b)
    assert a.shape == b.shape, f"{what}: shape {a.shape} vs {b.shape}"
    if a.dtype == np.float32 or b.dtype == np.float32:
        ba, bb = bits(a.astype(np.float32)), bits(b.astype(np.float32))
        bad = np.nonzero(ba != bb)
        assert bad[0].size == 0, f"{what}: {bad[0].size} mismatches, first at {bad[0][:5]}: {a[bad][:5]} vs {b[bad][:5]}"
    else:
        bad = np.nonzero(a != b)
        assert bad[0].size == 0, f"{what}: {bad[0].size} mismatches, first at {bad[0][:5]}: {a[bad][:5]} vs {b[bad][:5]}"


def compare_sums(gmap, omap):
    gv, gS, gc = gmap.export_voxels()
    ov, oS, oc = omap.export_sums()
    assert_same(gv, ov, "voxel ids")
    assert_same(gc, oc, "counts")
    assert_same(gS, oS, "sums")
    return len(gv)


def compare_labels(glab, ovox):
    assert_same(glab["vid"], ovox["vid"], "occupied voxel ids")
    assert_same(glab["nbr"], ovox["nbr"], "neighbour counts N")
    assert_same(glab["n"], ovox["n"], "normals")
    assert_same(glab["status"], ovox["status"].astype(np.uint8), "status")
    assert_same(glab["label"], ovox["label"], "CCL labels")


class RefitReport(tuple):
    """(worst angle, worst offset, planes excluded from the refit tolerance,
    planes with a valid hypothesis); unpacks as (worst angle, worst offset)
    for callers that want only those."""

    def __new__(cls, worst_angle, worst_offset, excluded, checked):
        r = super().__new__(cls, (worst_angle, worst_offset))
        r.excluded, r.valid = excluded, checked
        return r


def compare_planes(gres, ores, gclusters=None, check_refit=True):
    """gres: VoxelMap.segment / fit_planes output; ores: oracle result dict.

    Returns a RefitReport.  A plane is excluded from the refit tolerance only
    by the oracle (ill-conditioned in double, or fewer than 3 inliers), never
    by a flag the GPU sets."""
    gp, op = gres["planes"], ores["planes"]
    assert len(gp) == len(op["label"]), f"plane count {len(gp)} vs {len(op['label'])}"
    assert_same(gp["label"], op["label"], "labels")
    assert_same(gp["n_points"], op["n_points"], "cluster sizes")
    assert_same(gp["best_h"], op["best_h"], "selected hypotheses")
    if "round" in op:
        assert_same((gp["flags"] >> 8) & 0xFF, op["round"].astype(np.uint32), "extraction rounds")
    if gclusters is not None:
        assert_same(gclusters["pts"], ores["pts"], "cluster points")
        if ores["pt_vid"] is not None:
            assert_same(gclusters["pt_vid"], ores["pt_vid"], "cluster point voxel ids")
        assert_same(gclusters["inlier"], ores["inlier"], "inlier sets")
    valid = op["best_h"] >= 0
    assert_same(gp["inlier_count"][valid], op["inlier_count"][valid], "inlier counts")
    assert_same(gp["ransac_normal"][valid], op["ransac_n"][valid], "RANSAC normals")
    assert_same(gp["ransac_offset"][valid], op["ransac_d"][valid], "RANSAC offsets")
    assert_same(gp["basis_u"][valid], op["basis_u"][valid], "basis u")
    assert_same(gp["basis_v"][valid], op["basis_v"][valid], "basis v")
    assert_same(gp["hull_origin"][valid], op["origin"][valid], "hull origins")
    assert_same(gp["hull_count"], op["hull_n"], "hull sizes")
    for i in range(len(gp)):
        g = gres["hull_xy"][gp["hull_offset"][i]:gp["hull_offset"][i] + gp["hull_count"][i]]
        o = ores["hull"][op["hull_off"][i]:op["hull_off"][i] + op["hull_n"][i]]
        assert np.array_equal(g, o), f"hull of plane {i} (label {gp['label'][i]}): {g[:6]} vs {o[:6]}"
    worst_a = worst_d = 0.0
    excluded = 0
    if check_refit:
        for i in np.nonzero(valid)[0]:
            if op["inlier_count"][i] < 3:
                excluded += 1
                continue
            # The ill-conditioned flag is checked against the oracle's own
            # lambda_mid / lambda_min wherever that ratio is clear of the
            # threshold 10 (outside [9, 11]); near it, the GPU's FP32 /
            # double-float eigenvalues and the oracle's double Jacobi may
            # round to different sides, and the flag is not compared.
            cond = float(op["cond"][i]) if "cond" in op else float("nan")
            if not (9.0 <= cond <= 11.0) and not math.isnan(cond):
                assert bool(gp["flags"][i] & 1) == bool(op["ill_conditioned"][i]), \
                    f"ill-conditioned flag of plane {i}: GPU {gp['flags'][i] & 1}, oracle " \
                    f"{op['ill_conditioned'][i]} (lambda_mid / lambda_min = {cond:.4g})"
            # Only the oracle's flag excludes a plane from the tolerance.
            if op["ill_conditioned"][i]:
                excluded += 1
                continue
            gn = gp["normal"][i].astype(np.float64)
            on = op["refit_n"][i]
            dot = float(gn @ on)
            s = 1.0 if dot >= 0 else -1.0
            ang = angle(gn, on)
            dd = abs(s * float(gp["offset"][i]) - op["refit_d"][i])
            worst_a, worst_d = max(worst_a, ang), max(worst_d, dd)
            assert ang <= REFIT_ANGLE_TOL, f"refit normal of plane {i}: {ang:.3g} rad"
            assert dd <= REFIT_OFFSET_TOL, f"refit offset of plane {i}: {dd:.3g} m"
    return RefitReport(worst_a, worst_d, excluded, int(valid.sum()))
