"""Pins for the oracle's clustering of steppable voxels (Sec. III.C, Algorithm 1).

The adjacency is rebuilt here in float64 from the oracle's exported mean
positions and normals; pairs whose float64 test value sits within rounding of a
threshold are decided by exact binary32 evaluation of the reading's fma chain.  The partition is then
checked against scipy's connected components and against a direct run of
Algorithm 1's min-label propagation."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

from fp32exact import fmaf, mulf, subf

OFFS = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1) if (a, b, c) != (0, 0, 0)]


def _adjacency(v, prm, want):
    index = {tuple(x): i for i, x in enumerate(v["ijk"].tolist())}
    mu = v["mu"].astype(np.float64)
    n = v["n"].astype(np.float64)
    d2t, cc = float(prm.d_th2), float(prm.cos_ccl)
    rows, cols, ambiguous = [], [], 0
    for i, ijk in enumerate(v["ijk"].tolist()):
        if v["status"][i] < want:
            continue
        for o in OFFS:
            j = index.get((ijk[0] + o[0], ijk[1] + o[1], ijk[2] + o[2]))
            if j is None or v["status"][j] < want:
                continue
            d2 = float(((mu[i] - mu[j]) ** 2).sum())
            c = abs(float(n[i] @ n[j]))
            if abs(d2 - d2t) < 1e-7 * d2t or abs(c - cc) < 1e-6:
                ambiguous += 1
                dx, dy, dz = (subf(v["mu"][i][a], v["mu"][j][a]) for a in range(3))
                d2 = float(fmaf(dz, dz, fmaf(dy, dy, mulf(dx, dx))))
                ni, nj = v["n"][i], v["n"][j]
                c = abs(float(fmaf(ni[2], nj[2], fmaf(ni[1], nj[1], mulf(ni[0], nj[0])))))
                d2t, cc = np.float32(prm.d_th2), np.float32(prm.cos_ccl)
            if d2 < d2t and c > cc:
                rows.append(i)
                cols.append(j)
    return rows, cols, ambiguous


def _check_partition(v, prm, want):
    rows, cols, amb = _adjacency(v, prm, want)
    assert amb < 0.01 * max(len(rows), 1)
    N = len(v["vid"])
    A = sp.coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(N, N)).tocsr()
    assert (A != A.T).nnz == 0  # the edge test is symmetric
    ncomp, comp = connected_components(A, directed=False)
    member = v["status"] >= want
    lab = v["label"]
    assert np.all(lab[~member] == 0xFFFFFFFF)
    # same partition, and each label is the smallest voxel id of its component
    for cid in np.unique(comp[member]):
        sel = member & (comp == cid)
        assert np.unique(lab[sel]).size == 1
        assert lab[sel][0] == v["vid"][sel].min()
    assert np.unique(lab[member]).size == np.unique(comp[member]).size
    return rows, cols


def _label_propagation(N, rows, cols, member):
    """Algorithm 1: L_i <- i; repeat min-label exchange over edges until stable."""
    L = np.arange(N)
    changed = True
    while changed:
        changed = False
        for i, j in zip(rows, cols):
            if L[i] > L[j]:
                L[i] = L[j]
                changed = True
            elif L[i] < L[j]:
                L[j] = L[i]
                changed = True
    return L


def _random_scene(seed):
    import math
    rng = np.random.default_rng(seed)
    pts = []
    for _ in range(6):
        t = math.radians(rng.uniform(0, 25))
        a = rng.uniform(0, 2 * math.pi)
        n = np.array([math.sin(t) * math.cos(a), math.sin(t) * math.sin(a), math.cos(t)])
        c = rng.uniform([0.05, 0.05, 0.02], [0.45, 0.45, 0.2])
        u = np.cross([1.0, 0, 0], n); u /= np.linalg.norm(u)
        w = np.cross(n, u)
        s = rng.uniform(-0.12, 0.12, size=(1500, 2))
        pts.append(c + s[:, :1] * u + s[:, 1:] * w + rng.normal(0, 0.002, size=(1500, 1)) * n)
    return np.concatenate(pts).astype(np.float32)


@pytest.mark.parametrize("classify", [1, 0])
def test_config1_partition(orc, classify):
    import synth
    spec, pts, pose = synth.config1()
    m = orc.OracleMap(spec.dims, spec.origin, spec.voxel_size)
    m.integrate(pts, pose)
    prm = orc.make_params(n_hyp=8, classify=classify)
    v = m.segment(prm)["voxels"]
    _check_partition(v, prm, 2 if classify else 1)


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("res", [0.01, 0.02, 0.05])
def test_random_planes_partition(orc, seed, res):
    pts = _random_scene(seed)
    dims = (int(round(0.5 / res)),) * 2 + (int(round(0.3 / res)),)
    m = orc.OracleMap(dims, (0, 0, 0), res)
    m.integrate(pts)
    prm = orc.make_params(n_hyp=4, theta_ccl_deg=8.0, d_th=0.05 if res < 0.05 else 0.06)
    v = m.segment(prm)["voxels"]
    rows, cols = _check_partition(v, prm, 2)
    if len(v["vid"]) < 4000:
        L = _label_propagation(len(v["vid"]), rows, cols, v["status"] == 2)
        member = v["status"] == 2
        assert np.array_equal(v["vid"][L[member]], v["label"][member])


def test_clusters_min_size_order_and_points(orc):
    import synth
    spec, pts, pose = synth.config1()
    m = orc.OracleMap(spec.dims, spec.origin, spec.voxel_size)
    m.integrate(pts, pose)
    prm = orc.make_params(n_hyp=8, min_cluster=50)
    res = m.segment(prm)
    v, P = res["voxels"], res["planes"]
    labs, cnts = np.unique(v["label"][v["status"] == 2], return_counts=True)
    keep = cnts >= 50
    assert np.array_equal(P["label"], labs[keep])
    assert np.array_equal(P["n_points"], cnts[keep])
    assert np.all(np.diff(P["label"].astype(np.int64)) > 0)
    vid_to_i = {x: i for i, x in enumerate(v["vid"].tolist())}
    for k in range(len(P["label"])):
        o, n = P["point_off"][k], P["n_points"][k]
        pv = res["pt_vid"][o:o + n]
        assert np.all(np.diff(pv.astype(np.int64)) > 0)  # vid order inside a cluster
        idx = [vid_to_i[x] for x in pv.tolist()]
        assert np.all(v["label"][idx] == P["label"][k])
        assert np.array_equal(res["pts"][o:o + n], v["mu"][idx])
