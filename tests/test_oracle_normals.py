"""Pins for the oracle's normal estimation and steppable classification
(Sec. III.C, Eq. 3 and Eq. 4; Jacobi method of Golub & Van Loan Sec. 8.5)."""
import math

import numpy as np
import pytest


def _min_eigvec(A):
    w, V = np.linalg.eigh(A)
    return w, V[:, 0]


@pytest.mark.parametrize("seed", range(6))
def test_jacobi_matches_eigh(orc, seed):
    rng = np.random.default_rng(seed)
    tested = 0
    for _ in range(300):
        B = rng.normal(size=(3, 3)) * rng.uniform(0.01, 100)
        A = (B @ B.T).astype(np.float32).astype(np.float64)
        a6 = np.array([A[0, 0], A[1, 1], A[2, 2], A[0, 1], A[0, 2], A[1, 2]], np.float32)
        n, d, V = orc.jacobi3_f32(a6)
        w, v = _min_eigvec(A)
        assert np.allclose(np.sort(d), w, atol=2e-5 * w[-1])
        # the eigenvectors stay orthonormal
        assert np.allclose(V.T.astype(np.float64) @ V, np.eye(3), atol=2e-6)
        if (w[1] - w[0]) > 1e-2 * w[-1]:
            assert abs(float(np.dot(n, v))) > 1 - 1e-5
            tested += 1
    assert tested > 200


def test_jacobi_special_cases(orc):
    # zero matrix: every pair skipped, V = I, smallest diagonal at index 0
    n, d, V = orc.jacobi3_f32(np.zeros(6, np.float32))
    assert n.tolist() == [1.0, 0.0, 0.0] and np.array_equal(V, np.eye(3, dtype=np.float32))
    # diagonal input with the smallest entry last -> exactly e_z
    n, d, _ = orc.jacobi3_f32(np.array([5, 3, 1, 0, 0, 0], np.float32))
    assert n.tolist() == [0.0, 0.0, 1.0]
    # decoupled z (points on a horizontal plane): exactly e_z
    n, d, _ = orc.jacobi3_f32(np.array([4, 2, 0, 1.5, 0, 0], np.float32))
    assert n.tolist() == [0.0, 0.0, 1.0]
    # orientation: the min eigenvector of diag(1, 0, 1) is e_y with n_z = 0 -> +e_y
    n, _, _ = orc.jacobi3_f32(np.array([1, 0, 1, 0, 0, 0], np.float32))
    assert n.tolist() == [0.0, 1.0, 0.0]


def _sheet(normal, spacing=0.004, extent=0.3, center=(0.25, 0.25, 0.2)):
    n = np.asarray(normal, float)
    n /= np.linalg.norm(n)
    a = np.array([1.0, 0, 0]) if abs(n[0]) < 0.9 else np.array([0, 1.0, 0])
    u = np.cross(a, n); u /= np.linalg.norm(u)
    v = np.cross(n, u)
    s = np.arange(-extent / 2, extent / 2, spacing)
    U, W = np.meshgrid(s, s)
    return (np.asarray(center) + U.reshape(-1, 1) * u + W.reshape(-1, 1) * v).astype(np.float32), n


def test_exact_horizontal_plane_gives_exact_normals(orc):
    """Points all at z = 0.203125 (exact in binary): every normal is exactly (0,0,1)."""
    rng = np.random.default_rng(5)
    xy = rng.uniform(0.05, 0.45, size=(20000, 2))
    pts = np.c_[xy, np.full(len(xy), 0.203125)].astype(np.float32)
    m = orc.OracleMap((25, 25, 25), (0, 0, 0), 0.02)
    m.integrate(pts)
    v = m.segment(orc.make_params(min_cluster=1))["voxels"]
    assert np.all(v["n"] == np.float32([0, 0, 1]))
    interior = v["nbr"] >= 3
    assert np.all(v["status"][interior] == 2) and np.all(v["status"][~interior] == 1)


@pytest.mark.parametrize("tilt_deg,az_deg", [(0, 0), (10, 30), (14, 200), (16, 75), (40, 120), (89, 10)])
def test_tilted_plane_normals_and_classification(orc, tilt_deg, az_deg):
    t, a = math.radians(tilt_deg), math.radians(az_deg)
    pts, n_true = _sheet((math.sin(t) * math.cos(a), math.sin(t) * math.sin(a), math.cos(t)))
    m = orc.OracleMap((25, 25, 25), (0, 0, 0), 0.02)
    m.integrate(pts)
    v = m.segment(orc.make_params(min_cluster=1))["voxels"]
    full = v["nbr"] >= 8  # voxels with a populated window
    ang = np.degrees(np.arccos(np.clip(np.abs(v["n"][full].astype(np.float64) @ n_true), 0, 1)))
    assert ang.max() < 0.05
    assert np.all(v["n"][:, 2] >= 0)
    exp_step = abs(n_true[2]) >= np.float32(math.cos(math.radians(15)))
    assert np.all((v["status"][full] == 2) == exp_step)


def test_window_covariance_against_numpy(orc):
    """Config-1 voxels: N by brute force, the normal against numpy's eigh of the
    window covariance formed independently in float64 from the integer means."""
    import synth
    spec, pts, pose = synth.config1()
    m = orc.OracleMap(spec.dims, spec.origin, spec.voxel_size)
    m.integrate(pts, pose)
    prm = orc.make_params(n_hyp=64)
    v = m.segment(prm)["voxels"]
    index = {tuple(x): i for i, x in enumerate(v["ijk"].tolist())}
    M = v["M"].astype(np.float64)
    checked = 0
    for i, ijk in enumerate(v["ijk"].tolist()):
        nb = [index[(ijk[0] + a, ijk[1] + b, ijk[2] + c)] for a in (-1, 0, 1) for b in (-1, 0, 1)
              for c in (-1, 0, 1) if (ijk[0] + a, ijk[1] + b, ijk[2] + c) in index]
        assert v["nbr"][i] == len(nb) - 1
        P = M[nb]
        C = np.cov(P.T, bias=True) if len(nb) > 1 else np.zeros((3, 3))
        w, e = _min_eigvec(C)
        if len(nb) >= 4 and (w[1] - w[0]) > 0.05 * w[-1]:
            assert abs(float(e @ v["n"][i])) > 1 - 1e-4
            checked += 1
        exp = 2 if (v["nbr"][i] >= 3 and abs(v["n"][i][2]) >= prm.cos_step) else 1
        assert v["status"][i] == exp
    assert checked > 0.8 * len(v["vid"])
