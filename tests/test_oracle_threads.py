"""The oracle's all-cores mode (used only to time the CPU baseline on all host
cores) gives exactly the single-thread results: integer sums, normals, labels,
planes and hulls."""
import numpy as np

import synth


def _run(orc, threads):
    orc.set_threads(threads)
    try:
        spec, pts, pose = synth.config1()
        m = orc.OracleMap(spec.dims, spec.origin, spec.voxel_size)
        m.integrate(pts, pose)
        res = m.segment(orc.make_params(n_hyp=64))
        xyz, off, _ = synth.config3_clusters(n_clusters=40, seed=3, size_hi=3000)
        fit = orc.fit_planes(xyz.astype(np.float32), off.astype(np.uint32), orc.make_params(n_hyp=32, seed=2))
        return m.export_sums(), res, fit
    finally:
        orc.set_threads(1)


def test_threads_change_nothing(orc):
    (v1, s1, c1), r1, f1 = _run(orc, 1)
    (v4, s4, c4), r4, f4 = _run(orc, 4)
    assert np.array_equal(v1, v4) and np.array_equal(s1, s4) and np.array_equal(c1, c4)
    for a, b in ((r1, r4), (f1, f4)):
        for key in ("label", "best_h", "inlier_count", "ransac_n", "refit_n", "refit_d", "hull_off", "hull_n"):
            assert np.array_equal(a["planes"][key], b["planes"][key]), key
        assert np.array_equal(a["hull"], b["hull"])
    assert np.array_equal(r1["voxels"]["label"], r4["voxels"]["label"])
    assert np.array_equal(r1["voxels"]["n"], r4["voxels"]["n"])
    assert orc.threads() == 1
