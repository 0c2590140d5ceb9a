"""Seeded synthetic inputs for the voxel-mapping / plane-segmentation path.

This module generates input data only: scenes, sensor frames, poses and point
clusters.  It holds none of the method's arithmetic (no voxel keying, no
normals, no clustering, no plane fitting), and both the CPU oracle and the CUDA
library consume its outputs.

The paper's inputs came from MuJoCo scenes rendered through a graphics stack
(Sec. IV-A).  None is available here, so every frame is produced by analytic
ray casting against convex polyhedra: stairs, open treads, an overhanging desk,
ramps and boxes.

Workloads:
* ``config1``: 1.0 x 1.0 x 0.5 m map at 0.02 m; floor, a 3-step stair and a 10 deg
  ramp; 20,000 surface points, sigma = 3 mm, seed 0.
* ``config2_*``: 4 x 4 x 2 m map at 0.01 m; a 640 x 480 depth camera (87 x 58 deg,
  range 0.3-4 m, sigma = 1 mm + 0.2 % of range) walking 300 frames over an
  8-step open-tread stair, a desk with a 0.4 m overhang, a 15 deg ramp, floor and
  20 random boxes; frame f uses noise seed f.
* ``config3_clusters``: caller-formed clusters, sizes log-uniform in
  [50, 200000], tilts U[0, 35 deg], 5 % outliers, seed 7
  (``config3_clusters_device``: the same recipe generated on a torch device).
* ``e5_clusters``: the paper's cluster-parallel ablation (1-16 clusters of M in
  [10k, 30k] points).
* ``config4_streams``: serving streams with random extents and resolutions.
* ``config5_*``: the stress workload, a 128-beam spinning LiDAR (1.3 M rays a
  frame) over multi-level floors and 500 boxes and slabs in an 8 x 8 x 3 m map.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = ["MapSpec", "config1", "config2_spec", "config2_scene", "config2_frame", "config2_pose",
           "config3_clusters", "config3_clusters_device", "e5_clusters", "Scene", "Camera", "config4_streams", "config4_scene", "config4_pose", "config4_frame",
           "poisson_arrivals", "identity_pose", "config5_spec", "config5_scene", "config5_pose",
           "config5_frame", "Lidar", "STAGE", "stage_scene", "stage_orbit_frame", "face_values",
           "far_window_points"]


@dataclass
class MapSpec:
    """Grid of ``dims`` voxels of size ``voxel_size`` whose corner is ``origin``."""
    dims: tuple
    origin: tuple
    voxel_size: float

    @property
    def extent(self):
        return tuple(d * self.voxel_size for d in self.dims)


def identity_pose():
    return np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32)


# --------------------------------------------------------------------------
# Config 1: uniform samples over the exposed surfaces of a small stair scene.
# --------------------------------------------------------------------------

def _rect_samples(rng, n, p0, e1, e2):
    a = rng.random(n)
    b = rng.random(n)
    return np.asarray(p0)[None, :] + a[:, None] * np.asarray(e1)[None, :] + b[:, None] * np.asarray(e2)[None, :]


def config1(seed: int = 0, n_points: int = 20000, sigma: float = 0.003):
    """Floor z=0 over [0,1]^2, a 3-step stair (rise 0.15, tread 0.30, width 0.6 m)
    and a 10-degree ramp, sampled uniformly by area, isotropic noise sigma."""
    spec = MapSpec((50, 50, 25), (0.0, 0.0, -0.03), 0.02)
    t10 = math.tan(math.radians(10.0))
    rects = []  # (p0, e1, e2)
    # stair treads x in [0.05, 0.95] in three 0.30 m treads, y in [0, 0.6]
    for k in range(3):
        x0 = 0.05 + 0.30 * k
        h = 0.15 * (k + 1)
        rects.append(((x0, 0.0, h), (0.30, 0, 0), (0, 0.6, 0)))
        # riser at the front of tread k, from the previous height to h
        rects.append(((x0, 0.0, h - 0.15), (0, 0.6, 0), (0, 0, 0.15)))
        # side face at y = 0.6 below tread k
        rects.append(((x0, 0.6, 0.0), (0.30, 0, 0), (0, 0, h)))
    rects.append(((0.95, 0.0, 0.0), (0, 0.6, 0), (0, 0, 0.45)))  # back face
    # ramp x in [0.1, 0.9], y in [0.65, 1.0], rising along +x at 10 degrees
    L = 0.8
    rects.append(((0.1, 0.65, 0.0), (L, 0, L * t10), (0, 0.35, 0)))
    rects.append(((0.9, 0.65, 0.0), (0, 0.35, 0), (0, 0, L * t10)))  # end face
    # floor minus the two footprints, as a set of rectangles
    rects.append(((0.0, 0.0, 0.0), (0.05, 0, 0), (0, 0.65, 0)))
    rects.append(((0.95, 0.0, 0.0), (0.05, 0, 0), (0, 0.65, 0)))
    rects.append(((0.0, 0.6, 0.0), (0.95, 0, 0), (0, 0.05, 0)))
    rects.append(((0.0, 0.65, 0.0), (0.1, 0, 0), (0, 0.35, 0)))
    rects.append(((0.9, 0.65, 0.0), (0.1, 0, 0), (0, 0.35, 0)))
    areas = np.array([np.linalg.norm(np.cross(e1, e2)) for _, e1, e2 in rects])
    rng = np.random.Generator(np.random.PCG64(seed))
    counts = rng.multinomial(n_points, areas / areas.sum())
    pts = [_rect_samples(rng, int(c), p0, e1, e2) for c, (p0, e1, e2) in zip(counts, rects)]
    pts = np.concatenate(pts, axis=0)
    pts = pts + rng.normal(0.0, sigma, size=pts.shape)
    pts = pts[rng.permutation(pts.shape[0])]
    return spec, pts.astype(np.float32), identity_pose()


# --------------------------------------------------------------------------
# Convex-polyhedron scenes and a pinhole depth camera.
# --------------------------------------------------------------------------

def _box_planes(center, half, yaw=0.0, tilt=0.0, tilt_az=0.0):
    """Planes (n, d) with inside = n.x <= d of an oriented box."""
    cy, sy = math.cos(yaw), math.sin(yaw)
    Rz = np.array([[cy, -sy, 0], [sy, cy, 0], [0, 0, 1]])
    ca, sa = math.cos(tilt_az), math.sin(tilt_az)
    axis = np.array([-sa, ca, 0.0])
    ct, st = math.cos(tilt), math.sin(tilt)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    Rt = np.eye(3) + st * K + (1 - ct) * K @ K
    R = Rt @ Rz
    c = np.asarray(center, float)
    planes = []
    for k in range(3):
        a = R[:, k]
        planes.append(np.r_[a, a @ c + half[k]])
        planes.append(np.r_[-a, -a @ c + half[k]])
    return np.array(planes)


def _aabb_planes(lo, hi):
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    return _box_planes((lo + hi) / 2, (hi - lo) / 2)


def _ramp_planes(x0, x1, y0, y1, angle_deg):
    a = math.radians(angle_deg)
    s, c = math.sin(a), math.cos(a)
    return np.array([[-s, 0, c, -x0 * s],   # top: z cos a - (x - x0) sin a <= 0
                     [0, 0, -1, 0.0],        # bottom z >= 0
                     [1, 0, 0, x1],          # end face x <= x1
                     [0, -1, 0, -y0],        # y >= y0
                     [0, 1, 0, y1]])         # y <= y1


@dataclass
class Scene:
    """A union of convex polyhedra, each a (F, 4) array of (n, d), inside n.x <= d."""
    prims: list = field(default_factory=list)

    def add(self, planes):
        self.prims.append(np.asarray(planes, float))


@dataclass
class Camera:
    width: int = 640
    height: int = 480
    fov_h_deg: float = 87.0
    fov_v_deg: float = 58.0
    r_min: float = 0.3
    r_max: float = 4.0
    sigma0: float = 0.001
    sigma_rel: float = 0.002

    def rays(self):
        """Unit ray directions in the camera frame (x right, y down, z forward), row-major pixels."""
        fx = (self.width / 2) / math.tan(math.radians(self.fov_h_deg / 2))
        fy = (self.height / 2) / math.tan(math.radians(self.fov_v_deg / 2))
        u = (np.arange(self.width) + 0.5 - self.width / 2) / fx
        v = (np.arange(self.height) + 0.5 - self.height / 2) / fy
        X, Y = np.meshgrid(u, v)
        d = np.stack([X, Y, np.ones_like(X)], axis=-1).reshape(-1, 3)
        return d / np.linalg.norm(d, axis=1, keepdims=True)


def _prim_sphere(planes):
    """Bounding sphere of a convex polyhedron (vertices from all plane triples)."""
    P = np.asarray(planes, float)
    verts = []
    F = P.shape[0]
    for i in range(F):
        for j in range(i + 1, F):
            for k in range(j + 1, F):
                A = P[[i, j, k], :3]
                if abs(np.linalg.det(A)) < 1e-12:
                    continue
                x = np.linalg.solve(A, P[[i, j, k], 3])
                if np.all(P[:, :3] @ x <= P[:, 3] + 1e-9):
                    verts.append(x)
    V = np.array(verts)
    c = 0.5 * (V.min(axis=0) + V.max(axis=0))
    return c, float(np.linalg.norm(V - c, axis=1).max()) + 1e-6


def raycast(scene: Scene, origin, dirs, device="cpu"):
    """First-hit distance of each ray (inf when nothing is hit); torch on ``device``.

    Each convex polyhedron is first tested against its bounding sphere; only the
    rays that pass are clipped against its planes."""
    import torch
    o_np = np.asarray(origin, np.float64)
    D = torch.as_tensor(np.asarray(dirs), dtype=torch.float32, device=device)
    best = torch.full((D.shape[0],), float("inf"), dtype=torch.float32, device=device)
    for planes in scene.prims:
        if not hasattr(scene, "_spheres"):
            scene._spheres = {}
        key = id(planes)
        if key not in scene._spheres:
            scene._spheres[key] = _prim_sphere(planes)
        c, rad = scene._spheres[key]
        oc = torch.as_tensor(c - o_np, dtype=torch.float32, device=device)
        tc = D @ oc
        d2 = float(oc @ oc) - tc * tc
        inside = float(np.dot(c - o_np, c - o_np)) <= rad * rad
        cand = (d2 <= rad * rad) & ((tc > 0) | inside)
        idx = torch.nonzero(cand).flatten()
        if idx.numel() == 0:
            continue
        d = D[idx]
        P = torch.as_tensor(planes, dtype=torch.float32, device=device)
        n = P[:, :3]
        num = P[:, 3] - n @ torch.as_tensor(o_np, dtype=torch.float32, device=device)
        den = d @ n.T
        t = num[None] / den
        inf = torch.tensor(float("inf"), device=device)
        te = torch.where(den < 0, t, -inf).max(dim=1).values
        tx = torch.where(den > 0, t, inf).min(dim=1).values
        par_miss = ((den == 0) & (num[None] < 0)).any(dim=1)
        hit = (te <= tx) & (te > 0) & ~par_miss
        th = torch.where(hit, te, inf)
        best[idx] = torch.minimum(best[idx], th)
    return best


def _rot_z(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])


def _rot_y(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])


# camera axes (x right, y down, z forward) -> body axes (x forward, y left, z up)
_CAM_TO_BODY = np.array([[0, 0, 1.0], [-1, 0, 0], [0, -1, 0]])


def camera_pose(position, yaw, pitch_down_deg):
    R = _rot_z(yaw) @ _rot_y(math.radians(pitch_down_deg)) @ _CAM_TO_BODY
    return np.concatenate([R, np.asarray(position, float)[:, None]], axis=1)


def _depth_frame(scene, cam, pose34, seed, device="cpu"):
    """Points in the camera frame (NaN where the ray returns nothing), float32[H*W, 3]."""
    import torch
    dirs = cam.rays()
    R = pose34[:, :3]
    t = pose34[:, 3]
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = rng.standard_normal(dirs.shape[0]).astype(np.float32)
    r = raycast(scene, t, dirs @ R.T, device=device)
    nz = torch.as_tensor(noise, device=device)
    valid = (r >= cam.r_min) & (r <= cam.r_max)
    r_noisy = r + nz * (cam.sigma0 + cam.sigma_rel * r)
    d = torch.as_tensor(dirs, dtype=torch.float32, device=device)
    pts = d * r_noisy[:, None]
    pts = torch.where(valid[:, None], pts, torch.full_like(pts, float("nan")))
    return pts


# --------------------------------------------------------------------------
# Config 2: the paper-scale trajectory.
# --------------------------------------------------------------------------

def config2_spec():
    return MapSpec((400, 400, 200), (0.0, 0.0, -0.05), 0.01)


STAIR_X0, STAIR_Y = 1.0, (0.4, 1.2)


def config2_scene(seed: int = 0, n_boxes: int = 20):
    sc = Scene()
    sc.add(_aabb_planes((-50, -50, -1), (50, 50, 0)))  # floor
    for k in range(1, 9):  # 8-step open-tread stair: rise 0.15, run 0.30, 0.03 thick, 0.8 wide
        x0 = STAIR_X0 + 0.30 * (k - 1)
        sc.add(_aabb_planes((x0, STAIR_Y[0], 0.15 * k - 0.03), (x0 + 0.30, STAIR_Y[1], 0.15 * k)))
    # desk: top at 0.72 m, 0.03 m thick, overhanging its legs by 0.4 m along +x
    sc.add(_aabb_planes((1.8, 2.2, 0.69), (3.0, 3.0, 0.72)))
    for lx in (1.8, 2.56):
        for ly in (2.2, 2.96):
            sc.add(_aabb_planes((lx, ly, 0.0), (lx + 0.04, ly + 0.04, 0.69)))
    sc.add(_ramp_planes(0.3, 1.7, 1.4, 2.0, 15.0))  # 15-degree ramp
    rng = np.random.Generator(np.random.PCG64(seed))
    keep_out = [(0.9, 3.5, 0.3, 1.3), (1.7, 3.1, 2.1, 3.1), (0.2, 1.8, 1.3, 2.1)]
    placed = 0
    while placed < n_boxes:
        sx, sy = rng.uniform(0.1, 0.5, 2)
        h = rng.uniform(0.05, 0.4)
        cx, cy = rng.uniform(0.3, 3.7, 2)
        yaw = rng.uniform(0, math.pi / 2)
        r = 0.5 * math.hypot(sx, sy)
        box = (cx - r, cx + r, cy - r, cy + r)
        if any(not (box[1] < a or box[0] > b or box[3] < c or box[2] > d) for a, b, c, d in keep_out):
            continue
        keep_out.append(box)
        sc.add(_box_planes((cx, cy, h / 2), (sx / 2, sy / 2, h / 2), yaw=yaw))
        placed += 1
    return sc


def _terrain_height(x, y):
    if STAIR_Y[0] <= y <= STAIR_Y[1] and STAIR_X0 <= x < STAIR_X0 + 2.4:
        return 0.15 * (int((x - STAIR_X0) / 0.30) + 1)
    return 0.0


def config2_pose(frame: int):
    """Sensor->map pose of frame ``frame`` (1..300), 30 Hz, walking +x over the stair."""
    t = (frame - 1) / 30.0
    x = 0.3 + 0.3 * t
    y = 0.8 + 0.15 * math.sin(0.6 * t)
    yaw = 0.35 * math.sin(0.5 * t)
    z = _terrain_height(x, y) + 0.45
    return camera_pose((x, y, z), yaw, 25.0)


def config2_frame(frame: int, scene: Scene | None = None, device="cpu"):
    """(points float32[307200, 3] in the camera frame, pose float32[12]) of one frame."""
    scene = scene or config2_scene()
    pose = config2_pose(frame)
    pts = _depth_frame(scene, Camera(), pose, seed=frame, device=device)
    return pts, pose.astype(np.float32).reshape(12)


# --------------------------------------------------------------------------
# Config 3 / E5: caller-formed clusters for the batched plane fit.
# --------------------------------------------------------------------------

def _patch(rng, size, tilt, az, center, lattice=0.01, jitter=0.003, sigma=0.001, outlier_frac=0.05):
    side = int(math.ceil(math.sqrt(size)))
    idx = np.arange(size)
    u = (idx % side - (side - 1) / 2) * lattice + rng.uniform(-jitter, jitter, size)
    v = (idx // side - (side - 1) / 2) * lattice + rng.uniform(-jitter, jitter, size)
    w = rng.normal(0.0, sigma, size)
    n = np.array([math.sin(tilt) * math.cos(az), math.sin(tilt) * math.sin(az), math.cos(tilt)])
    a = np.array([1.0, 0, 0]) if abs(n[0]) < 0.9 else np.array([0, 1.0, 0])
    e1 = np.cross(a, n)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    p = center[None, :] + u[:, None] * e1 + v[:, None] * e2 + w[:, None] * n
    n_out = int(round(outlier_frac * size))
    if n_out:
        lo = p.min(axis=0) - 0.05
        hi = p.max(axis=0) + 0.05
        sel = rng.choice(size, n_out, replace=False)
        p[sel] = rng.uniform(lo, hi, size=(n_out, 3))
    return p, n


def config3_clusters(n_clusters: int = 2000, seed: int = 7, size_lo: int = 50, size_hi: int = 200000,
                     max_tilt_deg: float = 35.0, outlier_frac: float = 0.05):
    """(xyz float32[sum, 3], off uint32[k+1], true normals float64[k, 3])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.exp(rng.uniform(math.log(size_lo), math.log(size_hi), n_clusters)).astype(np.int64)
    sizes = np.clip(sizes, size_lo, size_hi)
    off = np.zeros(n_clusters + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    xyz = np.empty((int(off[-1]), 3), np.float32)
    normals = np.zeros((n_clusters, 3))
    for k in range(n_clusters):
        tilt = math.radians(rng.uniform(0, max_tilt_deg))
        az = rng.uniform(0, 2 * math.pi)
        center = rng.uniform(-8, 8, 3) * np.array([1, 1, 0.1])
        p, n = _patch(rng, int(sizes[k]), tilt, az, center, outlier_frac=outlier_frac)
        xyz[off[k]:off[k + 1]] = p
        normals[k] = n
    return xyz, off.astype(np.uint32), normals


def config3_clusters_device(n_clusters: int = 2000, seed: int = 7, size_lo: int = 50, size_hi: int = 200000,
                            max_tilt_deg: float = 35.0, outlier_frac: float = 0.05, device="cuda"):
    """The config-3 recipe generated on a torch device (the 48 M-point batch
    takes about 30 s in numpy): per-cluster sizes, tilts, azimuths and centres
    from numpy's PCG64(seed) as in ``config3_clusters``; lattice jitter, normal
    noise and outliers from a torch generator seeded with ``seed``, each point
    an outlier with probability ``outlier_frac`` (uniform in its cluster's
    box padded by 0.05 m).  Returns xyz float32[sum, 3] and off int32[k+1] (the
    same bits as uint32: every offset is below 2^31) as torch tensors on
    ``device``, and the true normals float64[k, 3] on the host."""
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.exp(rng.uniform(math.log(size_lo), math.log(size_hi), n_clusters)).astype(np.int64)
    sizes = np.clip(sizes, size_lo, size_hi)
    tilt = np.radians(rng.uniform(0, max_tilt_deg, n_clusters))
    az = rng.uniform(0, 2 * math.pi, n_clusters)
    center = rng.uniform(-8, 8, (n_clusters, 3)) * np.array([1, 1, 0.1])
    n = np.stack([np.sin(tilt) * np.cos(az), np.sin(tilt) * np.sin(az), np.cos(tilt)], 1)
    a = np.where(np.abs(n[:, :1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
    e1 = np.cross(a, n)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(n, e1)
    off = np.zeros(n_clusters + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    f64 = dict(dtype=torch.float64, device=device)
    cid = torch.repeat_interleave(torch.arange(n_clusters, device=device), torch.as_tensor(sizes, device=device))
    idx = torch.arange(int(off[-1]), device=device) - torch.as_tensor(off[:-1], device=device)[cid]
    side = torch.as_tensor(np.ceil(np.sqrt(sizes)), **f64)[cid]
    jit = 0.003
    u = (torch.remainder(idx, side) - (side - 1) / 2) * 0.01 + (torch.rand(idx.shape, generator=g, **f64) * 2 - 1) * jit
    v = (torch.div(idx, side, rounding_mode="floor") - (side - 1) / 2) * 0.01 \
        + (torch.rand(idx.shape, generator=g, **f64) * 2 - 1) * jit
    w = torch.randn(idx.shape, generator=g, **f64) * 0.001
    C_, N_ = torch.as_tensor(center, **f64), torch.as_tensor(n, **f64)
    E1, E2 = torch.as_tensor(e1, **f64), torch.as_tensor(e2, **f64)
    p = C_[cid] + u[:, None] * E1[cid] + v[:, None] * E2[cid] + w[:, None] * N_[cid]
    lo = torch.full((n_clusters, 3), float("inf"), **f64).scatter_reduce(0, cid[:, None].expand(-1, 3), p, "amin")
    hi = torch.full((n_clusters, 3), float("-inf"), **f64).scatter_reduce(0, cid[:, None].expand(-1, 3), p, "amax")
    lo, hi = lo - 0.05, hi + 0.05
    out = torch.rand(idx.shape, generator=g, **f64) < outlier_frac
    r = torch.rand((int(off[-1]), 3), generator=g, **f64)
    q = lo[cid] + r * (hi - lo)[cid]
    p = torch.where(out[:, None], q, p)
    assert off[-1] < 2**31
    return (p.to(torch.float32).contiguous(), torch.as_tensor(off.astype(np.int32), device=device), n)


def e5_clusters(n_clusters: int, seed: int, m_lo: int = 10000, m_hi: int = 30000):
    """The paper's cluster-parallel ablation input: n_clusters clusters of exactly M
    random points each, M ~ U[m_lo, m_hi] per trial, noisy planar patches."""
    rng = np.random.Generator(np.random.PCG64(seed))
    M = int(rng.integers(m_lo, m_hi + 1))
    off = np.arange(n_clusters + 1, dtype=np.int64) * M
    xyz = np.empty((n_clusters * M, 3), np.float32)
    for k in range(n_clusters):
        tilt = math.radians(rng.uniform(0, 30))
        az = rng.uniform(0, 2 * math.pi)
        center = rng.uniform(-3, 3, 3) * np.array([1, 1, 0.2])
        p, _ = _patch(rng, M, tilt, az, center, outlier_frac=0.1)
        xyz[k * M:(k + 1) * M] = p
    return xyz, off.astype(np.uint32)


# --------------------------------------------------------------------------
# Config 4: serving streams.
# --------------------------------------------------------------------------

@dataclass
class StreamSpec:
    stream_id: int
    spec: MapSpec
    scene_seed: int
    rate_hz: float
    arrival_seed: int


def config4_streams(n_streams: int = 16, seed: int = 11, rate_hz: float = 30.0):
    """Stream descriptions: extent U[2, 6] m per side x 2 m, resolution in {0.01, 0.02, 0.05}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for s in range(n_streams):
        ex, ey = rng.uniform(2.0, 6.0, 2)
        res = float(rng.choice([0.01, 0.02, 0.05]))
        dims = (int(round(ex / res)), int(round(ey / res)), int(round(2.0 / res)))
        out.append(StreamSpec(s, MapSpec(dims, (0.0, 0.0, -0.05), res), 1000 + s, rate_hz, 5000 + s))
    return out


def config4_scene(st: StreamSpec) -> Scene:
    """An independently seeded stair / desk / ramp scene inside a stream's map
    extent: floor, an open-tread stair (4-8 steps, rise 0.15 m, run 0.30 m,
    treads 0.03 m thick, 0.8 m wide), a desk (top 0.72 m, 0.03 m thick, legs
    set back 0.4 m from one edge), a 15 deg ramp and 10 boxes, placed with
    PCG64(scene_seed)."""
    rng = np.random.Generator(np.random.PCG64(st.scene_seed))
    ex = st.spec.dims[0] * st.spec.voxel_size
    ey = st.spec.dims[1] * st.spec.voxel_size
    sc = Scene()
    sc.add(_aabb_planes((-50, -50, -1), (50, 50, 0)))
    n_steps = int(rng.integers(4, 9))
    x0 = rng.uniform(0.1, max(0.2, ex - 0.3 * n_steps - 0.1))
    y0 = rng.uniform(0.1, max(0.2, ey - 0.9))
    for k in range(1, n_steps + 1):
        xa = x0 + 0.30 * (k - 1)
        sc.add(_aabb_planes((xa, y0, 0.15 * k - 0.03), (xa + 0.30, y0 + 0.8, 0.15 * k)))
    dx, dy = rng.uniform(0.1, max(0.2, ex - 1.3)), rng.uniform(0.1, max(0.2, ey - 0.9))
    sc.add(_aabb_planes((dx, dy, 0.69), (dx + 1.2, dy + 0.8, 0.72)))
    for lx in (dx, dx + 0.76):
        for ly in (dy, dy + 0.76):
            sc.add(_aabb_planes((lx, ly, 0.0), (lx + 0.04, ly + 0.04, 0.69)))
    rx, ry = rng.uniform(0.1, max(0.2, ex - 1.5)), rng.uniform(0.1, max(0.2, ey - 0.7))
    sc.add(_ramp_planes(rx, rx + 1.4, ry, ry + 0.6, 15.0))
    for _ in range(10):
        sx, sy = rng.uniform(0.1, 0.5, 2)
        h = rng.uniform(0.05, 0.4)
        cx, cy = rng.uniform(0.2, ex - 0.2), rng.uniform(0.2, ey - 0.2)
        sc.add(_box_planes((cx, cy, h / 2), (sx / 2, sy / 2, h / 2), yaw=rng.uniform(0, math.pi / 2)))
    return sc


def config4_pose(st: StreamSpec, frame: int):
    """Sensor->map pose of a stream's frame ``frame`` (30 Hz): an ellipse around
    the extent's centre (radii 0.3 x the extent, one lap in 20 s), 0.45 m above
    the floor, facing along the path, pitched down 25 deg."""
    ex = st.spec.dims[0] * st.spec.voxel_size
    ey = st.spec.dims[1] * st.spec.voxel_size
    w = 2 * math.pi / 20.0
    t = frame / 30.0 + (st.scene_seed % 97) * 0.37  # streams start at different phases
    x = ex / 2 + 0.3 * ex * math.cos(w * t)
    y = ey / 2 + 0.3 * ey * math.sin(w * t)
    yaw = math.atan2(0.3 * ey * math.cos(w * t), -0.3 * ex * math.sin(w * t))
    return camera_pose((x, y, 0.45), yaw, 25.0)


def config4_frame(st: StreamSpec, scene: Scene, frame: int, device="cpu"):
    """(points float32[307200, 3] in the camera frame, pose float32[12]) of a
    stream's frame; noise seed = scene_seed * 100003 + frame."""
    pose = config4_pose(st, frame)
    pts = _depth_frame(scene, Camera(), pose, seed=st.scene_seed * 100003 + frame, device=device)
    return pts, pose.astype(np.float32).reshape(12)


# --------------------------------------------------------------------------
# Config 5: the stress workload (spinning LiDAR over a cluttered multi-level
# scene).
# --------------------------------------------------------------------------

def config5_spec():
    """8 x 8 x 3 m map at 0.01 m (800 x 800 x 300 voxels)."""
    return MapSpec((800, 800, 300), (0.0, 0.0, -0.05), 0.01)


@dataclass
class Lidar:
    """A 128-beam spinning LiDAR: beams evenly spaced over a vertical field of
    view of +-22.5 deg (the builder's choice where the workload gives none),
    10,160 azimuth steps per revolution (1,300,480 rays a frame), range
    0.5-20 m, sigma 5 mm along the ray, 20 Hz."""
    beams: int = 128
    steps: int = 10160
    vfov_deg: float = 22.5
    r_min: float = 0.5
    r_max: float = 20.0
    sigma: float = 0.005

    def rays(self):
        """Unit ray directions in the sensor frame (z up), beam-major."""
        el = np.radians(np.linspace(-self.vfov_deg, self.vfov_deg, self.beams))
        az = np.arange(self.steps) * (2 * math.pi / self.steps)
        E, A = np.meshgrid(el, az, indexing="ij")
        return np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], axis=-1).reshape(-1, 3)


def config5_scene(seed: int = 5, n_objects: int = 500) -> Scene:
    """Multi-level floors with overhangs and 500 boxes and slabs: a ground floor,
    a mezzanine slab at 1.2 m over y in [5, 8] m and a gallery slab at 2.2 m
    over x in [0, 2.5] m (both 0.05 m thick, open underneath), and 500 objects
    with sizes log-uniform in [0.1, 2] m, tilts up to 30 deg and random yaw;
    a third of them are slabs (0.02-0.08 m thick); objects rest on the level
    under them.  PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sc = Scene()
    sc.add(_aabb_planes((-50, -50, -1), (50, 50, 0)))
    sc.add(_aabb_planes((0.0, 5.0, 1.15), (8.0, 8.0, 1.2)))
    sc.add(_aabb_planes((0.0, 0.0, 2.15), (2.5, 8.0, 2.2)))
    for i in range(n_objects):
        sx, sy = np.exp(rng.uniform(math.log(0.1), math.log(2.0), 2))
        slab = i % 3 == 0
        sz = rng.uniform(0.02, 0.08) if slab else float(np.exp(rng.uniform(math.log(0.1), math.log(1.0))))
        cx, cy = rng.uniform(0.2, 7.8, 2)
        base = 0.0
        if cy >= 5.0 and rng.uniform() < 0.5:
            base = 1.2
        elif cx <= 2.5 and rng.uniform() < 0.3:
            base = 2.2
        tilt = math.radians(rng.uniform(0, 30))
        sc.add(_box_planes((cx, cy, base + sz / 2), (sx / 2, sy / 2, sz / 2), yaw=rng.uniform(0, math.pi),
                           tilt=tilt, tilt_az=rng.uniform(0, 2 * math.pi)))
    return sc


def config5_pose(frame: int):
    """Sensor->map pose of frame ``frame`` (20 Hz): a circle of radius 2.5 m
    about the room's centre at 0.5 m/s, 0.6 m above the ground floor, the
    sensor level (z up)."""
    t = frame / 20.0
    w = 0.5 / 2.5
    x, y = 4.0 + 2.5 * math.cos(w * t), 4.0 + 2.5 * math.sin(w * t)
    R = _rot_z(w * t + math.pi / 2)
    return np.concatenate([R, np.array([[x], [y], [0.6]])], axis=1)


def config5_frame(frame: int, scene: Scene, device="cpu", lidar: Lidar | None = None):
    """(points float32[1,300,480, 3] in the sensor frame, NaN without a return
    in range; pose float32[12]).  Noise seed = 500,000 + frame."""
    import torch
    lidar = lidar or Lidar()
    pose = config5_pose(frame)
    dirs = lidar.rays()
    R, t = pose[:, :3], pose[:, 3]
    rng = np.random.Generator(np.random.PCG64(500000 + frame))
    noise = rng.standard_normal(dirs.shape[0]).astype(np.float32)
    r = raycast(scene, t, dirs @ R.T, device=device)
    nz = torch.as_tensor(noise, device=device)
    valid = (r >= lidar.r_min) & (r <= lidar.r_max)
    rn = r + nz * lidar.sigma
    d = torch.as_tensor(dirs, dtype=torch.float32, device=device)
    pts = d * rn[:, None]
    pts = torch.where(valid[:, None], pts, torch.full_like(pts, float("nan")))
    return pts, pose.astype(np.float32).reshape(12)


# --------------------------------------------------------------------------
# The single-stage scene for the plane IoU evaluation.
# --------------------------------------------------------------------------

STAGE = ((1.2, 1.4), (2.8, 2.6), 0.25)  # (x0, y0), (x1, y1), height: the stage top's ground truth


def stage_scene() -> Scene:
    """Floor and one stage (a 1.6 x 1.2 m box, 0.25 m high, centred at (2, 2)):
    its top is a plane whose region is known exactly."""
    sc = Scene()
    sc.add(_aabb_planes((-50, -50, -1), (50, 50, 0)))
    (x0, y0), (x1, y1), h = STAGE
    sc.add(_aabb_planes((x0, y0, 0.0), (x1, y1, h)))
    return sc


def stage_orbit_frame(k: int, n: int, scene: Scene, device="cpu"):
    """Frame k of n from the config-2 camera on a 1.9 m circle about the stage,
    1.1 m up, facing its centre, pitched down 35 deg; noise seed 700,000 + k."""
    a = 2 * math.pi * k / n
    pos = (2.0 + 1.9 * math.cos(a), 2.0 + 1.9 * math.sin(a), 1.1)
    pose = camera_pose(pos, a + math.pi, 35.0)
    pts = _depth_frame(scene, Camera(), pose, seed=700000 + k, device=device)
    return pts, pose.astype(np.float32).reshape(12)


def poisson_arrivals(rate_hz: float, duration_s: float, seed: int):
    rng = np.random.Generator(np.random.PCG64(seed))
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            return np.array(out)
        out.append(t)


def face_values(corner: float, n_ulps: int = 8):
    """The FP32 values within n_ulps units in the last place of fl32(corner),
    on both sides of it, ascending (2 n_ulps + 1 values)."""
    c = np.float32(corner)
    vals, up, dn = [c], c, c
    for _ in range(n_ulps):
        up = np.nextafter(up, np.float32(np.inf))
        dn = np.nextafter(dn, np.float32(-np.inf))
        vals += [up, dn]
    return np.sort(np.array(vals, np.float32))


def far_window_points(w, dims, voxel_size, per_cell: int = 12, n_ulps: int = 8, seed: int = 0):
    """Points around the low faces of a map window far from the base origin.

    The map's base origin is (0, 0, 0) and its window covers voxels
    w .. w + dims - 1 per axis, so its low face on axis a lies at
    w[a] * voxel_size.  For each axis a:
    * a plane over the lower half of the window in the two other axes:
      per voxel column of that half, per_cell points jittered by up to 0.4
      voxel about the column's centre, all with the same coordinate a, taken
      in turn from face_values(w[a] * voxel_size, n_ulps) (the FP32 values
      just below and above the face);
    * single points, one per voxel: coordinate a again from those face values
      (each value twice), the other two at voxel centres of the window's upper
      half in both of them, so no other point shares their voxels.
    Identity pose; float32 [n, 3]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = np.asarray(w, np.int64)
    dims = np.asarray(dims, np.int64)
    res = float(voxel_size)
    out = []
    for a in range(3):
        fv = face_values(float(w[a]) * res, n_ulps)
        b, c = (a + 1) % 3, (a + 2) % 3
        hb, hc = dims[b] // 2, dims[c] // 2
        ib, ic = np.meshgrid(np.arange(hb), np.arange(hc), indexing="ij")
        col = np.repeat(np.arange(hb * hc), per_cell)
        p = np.zeros((len(col), 3), np.float64)
        p[:, a] = fv[col % len(fv)]
        p[:, b] = (w[b] + ib.reshape(-1)[col] + 0.5 + rng.uniform(-0.4, 0.4, len(col))) * res
        p[:, c] = (w[c] + ic.reshape(-1)[col] + 0.5 + rng.uniform(-0.4, 0.4, len(col))) * res
        out.append(p.astype(np.float32))
        # singles: voxel centres of the upper half in b and c, one point each
        cells = [(i, j) for i in range(hb, dims[b]) for j in range(hc, dims[c])]
        n_single = min(2 * len(fv), len(cells))
        q = np.zeros((n_single, 3), np.float64)
        q[:, a] = np.concatenate([fv, fv])[:n_single]
        for k in range(n_single):
            i, j = cells[(k * 7) % len(cells)]
            q[k, b] = (w[b] + i + 0.5) * res
            q[k, c] = (w[c] + j + 0.5) * res
        out.append(q.astype(np.float32))
    return np.concatenate(out)
