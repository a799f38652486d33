"""Seeded synthetic point clouds shaped like the workloads of LSG-CPD's experiments.

This module only samples geometry: surfaces, analytic ray casting, noise,
outliers and ground-truth rigid motions.  It holds none of the registration
method's arithmetic, so both the CUDA path and the FP64 oracle can take their
inputs from here without sharing any of the method.

Every generator is deterministic in its seed (numpy ``PCG64``), works in FP64
and returns FP32-rounded clouds; both implementations consume the same rounded
values.  A returned pair maps the source onto the target with the ground-truth
rigid motion ``(R_gt, t_gt)``: ``y ~ R_gt @ x + t_gt`` on overlapping parts.

Workload shapes (stand-ins for the paper's datasets, which are not available):
  * ``sphere_plane_pair`` -- range-scanner object (Sec. 4.1, Stanford Bunny
    stand-in): unit sphere plus an off-centre plane patch.
  * ``rgbd_room_pair``   -- RGBD frames (Sec. 4.3, Stanford Lounge stand-in):
    a room of 6 walls, 3 boxes and 2 spheres, ray cast from a pinhole camera.
  * ``lidar_pair``       -- LiDAR scans (Sec. 4.4, KITTI stand-in): 64 rings
    over a ground plane with boxes, cylinders and a far wall.
  * ``batch_pairs``      -- many independent uneven pairs.
  * ``superquadric_pair``-- a large range scan from a union of superquadrics.
  * ``estep_case``       -- unstructured random clouds with random normals and
    penalties, for E-step unit tests.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 20210000


def make_rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def random_unit_vector(rng: np.random.Generator) -> np.ndarray:
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


def axis_angle_matrix(axis: np.ndarray, angle: float) -> np.ndarray:
    """Rotation matrix of ``angle`` radians about the unit ``axis`` (Rodrigues)."""
    k = np.asarray(axis, dtype=np.float64)
    k = k / np.linalg.norm(k)
    K = np.array([[0.0, -k[2], k[1]], [k[2], 0.0, -k[0]], [-k[1], k[0], 0.0]])
    return np.eye(3) + math.sin(angle) * K + (1.0 - math.cos(angle)) * (K @ K)


def random_rotation(rng: np.random.Generator, angle_rad: float) -> np.ndarray:
    return axis_angle_matrix(random_unit_vector(rng), angle_rad)


def _f32(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


def _pair(target: np.ndarray, source_world: np.ndarray, R_p: np.ndarray, t_p: np.ndarray,
          centre: np.ndarray, **meta) -> dict:
    """Build a pair whose source is ``R_p (p - centre) + centre + t_p``.

    The ground truth maps the moved source back: ``p = R_p^T (x - centre - t_p) + centre``.
    """
    src = (source_world - centre) @ R_p.T + centre + t_p
    R_gt = R_p.T
    t_gt = centre - R_p.T @ (centre + t_p)
    out = dict(X=_f32(src), Y=_f32(target), R_gt=R_gt, t_gt=t_gt)
    out.update(meta)
    return out


# ---------------------------------------------------------------------------
# Surface samplers
# ---------------------------------------------------------------------------

def sample_sphere(rng, n, centre=(0.0, 0.0, 0.0), radius=1.0):
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return np.asarray(centre) + radius * v


def sample_rect(rng, n, origin, u, v):
    """Uniform samples of the parallelogram ``origin + a u + b v``, a, b in [0, 1]."""
    a = rng.random((n, 1))
    b = rng.random((n, 1))
    return np.asarray(origin) + a * np.asarray(u) + b * np.asarray(v)


def sample_box_surface(rng, n, lo, hi, skip_bottom=False):
    """Area-weighted uniform samples of the surface of the axis-aligned box [lo, hi]."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    s = hi - lo
    faces = []
    for ax in range(3):
        a1, a2 = [a for a in range(3) if a != ax]
        for side in (0, 1):
            if skip_bottom and ax == 2 and side == 0:
                continue
            o = lo.copy()
            o[ax] = lo[ax] if side == 0 else hi[ax]
            u = np.zeros(3)
            u[a1] = s[a1]
            v = np.zeros(3)
            v[a2] = s[a2]
            faces.append((o, u, v, s[a1] * s[a2]))
    areas = np.array([f[3] for f in faces])
    counts = rng.multinomial(n, areas / areas.sum())
    pts = [sample_rect(rng, c, f[0], f[1], f[2]) for f, c in zip(faces, counts) if c > 0]
    p = np.concatenate(pts, axis=0)
    return p[rng.permutation(len(p))]


def sphere_plane_cloud(rng, n, noise):
    """Half on the unit sphere, half on the off-centre patch z=-1.25, x in [-0.2, 0.8], y in [-0.5, 0.5]."""
    n_s = n // 2
    n_p = n - n_s
    s = sample_sphere(rng, n_s)
    p = sample_rect(rng, n_p, (-0.2, -0.5, -1.25), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0))
    pts = np.concatenate([s, p], axis=0)
    pts = pts + noise * rng.standard_normal(pts.shape)
    return pts[rng.permutation(n)]


def _replace_outliers(rng, pts, ratio):
    n = len(pts)
    k = int(round(ratio * n))
    if k == 0:
        return pts, np.zeros(0, dtype=np.int64)
    lo = pts.min(axis=0)
    hi = pts.max(axis=0)
    idx = rng.choice(n, size=k, replace=False)
    out = pts.copy()
    out[idx] = lo + rng.random((k, 3)) * (hi - lo)
    return out, np.sort(idx)


# ---------------------------------------------------------------------------
# Workload 1: plain single pair, sphere + plane
# ---------------------------------------------------------------------------

def sphere_plane_pair(seed=SEED_BASE + 1, n=1000, m=1000, noise=0.005, angle_deg=30.0,
                      trans_norm=0.1):
    """Target and source sampled independently from the sphere + plane shape.

    The source is rotated by exactly ``angle_deg`` about a random axis (through the
    origin) and translated by a random direction scaled to ``trans_norm``.
    """
    rng = make_rng(seed)
    Y = sphere_plane_cloud(rng, m, noise)
    P = sphere_plane_cloud(rng, n, noise)
    R_p = random_rotation(rng, math.radians(angle_deg))
    t_p = trans_norm * random_unit_vector(rng)
    return _pair(Y, P, R_p, t_p, np.zeros(3), name="sphere_plane", seed=seed, w=0.1,
                 knn_k=10, max_iters=50)


# ---------------------------------------------------------------------------
# Analytic ray casting (no graphics API): planes of a closed box seen from the
# inside, solid axis-aligned boxes, spheres and vertical cylinders.
# ---------------------------------------------------------------------------

_EPS = 1e-9


def _ray_room_exit(o, d, lo, hi):
    """Distance to the inside walls of the axis-aligned box [lo, hi] (o inside)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(d > 0, (hi - o) / d, np.where(d < 0, (lo - o) / d, np.inf))
    return t.min(axis=1)


def _ray_box(o, d, lo, hi):
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        t1 = (lo - o) * inv
        t2 = (hi - o) * inv
    tn = np.nanmax(np.minimum(t1, t2), axis=1)
    tf = np.nanmin(np.maximum(t1, t2), axis=1)
    hit = (tn <= tf) & (tn > _EPS)
    return np.where(hit, tn, np.inf)


def _ray_sphere(o, d, c, r):
    oc = o - c
    b = np.einsum("ij,ij->i", d, oc)
    cc = np.einsum("ij,ij->i", oc, oc) - r * r
    disc = b * b - cc
    with np.errstate(invalid="ignore"):
        t = -b - np.sqrt(disc)
    return np.where((disc >= 0) & (t > _EPS), t, np.inf)


def _ray_vcyl(o, d, cx, cy, r, z0, z1):
    """Solid vertical cylinder (side and top caps) with axis (cx, cy), z in [z0, z1]."""
    ox = o[:, 0] - cx
    oy = o[:, 1] - cy
    a = d[:, 0] ** 2 + d[:, 1] ** 2
    b = ox * d[:, 0] + oy * d[:, 1]
    c = ox * ox + oy * oy - r * r
    disc = b * b - a * c
    with np.errstate(invalid="ignore", divide="ignore"):
        t_side = (-b - np.sqrt(disc)) / a
    z = o[:, 2] + t_side * d[:, 2]
    side_ok = (disc >= 0) & (a > 1e-12) & (t_side > _EPS) & (z >= z0) & (z <= z1)
    t = np.where(side_ok, t_side, np.inf)
    with np.errstate(divide="ignore", invalid="ignore"):
        t_top = (z1 - o[:, 2]) / d[:, 2]
    xt = ox + t_top * d[:, 0]
    yt = oy + t_top * d[:, 1]
    top_ok = (t_top > _EPS) & (xt * xt + yt * yt <= r * r) & (o[:, 2] > z1)
    return np.minimum(t, np.where(top_ok, t_top, np.inf))


def _cast(o, d, scene):
    t = np.full(len(d), np.inf)
    for kind, prm in scene:
        if kind == "room":
            t = np.minimum(t, _ray_room_exit(o, d, *prm))
        elif kind == "box":
            t = np.minimum(t, _ray_box(o, d, *prm))
        elif kind == "sphere":
            t = np.minimum(t, _ray_sphere(o, d, *prm))
        elif kind == "vcyl":
            t = np.minimum(t, _ray_vcyl(o, d, *prm))
        elif kind == "ground":
            with np.errstate(divide="ignore", invalid="ignore"):
                tg = (prm - o[:, 2]) / d[:, 2]
            t = np.minimum(t, np.where(tg > _EPS, tg, np.inf))
        elif kind == "farwall":
            cx, cy, r = prm
            t = np.minimum(t, _ray_vcyl_inside(o, d, cx, cy, r))
    return t


def _ray_vcyl_inside(o, d, cx, cy, r):
    ox = o[:, 0] - cx
    oy = o[:, 1] - cy
    a = d[:, 0] ** 2 + d[:, 1] ** 2
    b = ox * d[:, 0] + oy * d[:, 1]
    c = ox * ox + oy * oy - r * r
    with np.errstate(invalid="ignore", divide="ignore"):
        t = (-b + np.sqrt(b * b - a * c)) / a
    return np.where(a > 1e-12, t, np.inf)


def _look_rotation(forward, up=(0.0, 0.0, 1.0)):
    """Camera-to-world rotation for a camera with x right, y down, z forward."""
    f = np.asarray(forward, dtype=np.float64)
    f = f / np.linalg.norm(f)
    r = np.cross(f, np.asarray(up))
    r = r / np.linalg.norm(r)
    dn = np.cross(f, r)
    return np.stack([r, dn, f], axis=1)


# ---------------------------------------------------------------------------
# Workload 2: RGBD-shaped pair (room scene, pinhole camera 160 x 125)
# ---------------------------------------------------------------------------

ROOM_HI = np.array([5.0, 4.0, 2.6])
CAM_W, CAM_H, CAM_F = 160, 125, 138.6


def _room_scene(rng):
    scene = [("room", (np.zeros(3), ROOM_HI.copy()))]
    solids = []
    for _ in range(3):
        s = rng.uniform(0.3, 0.9, size=3)
        x = rng.uniform(0.4, ROOM_HI[0] - 0.4 - s[0])
        y = rng.uniform(0.4, ROOM_HI[1] - 0.4 - s[1])
        lo = np.array([x, y, 0.0])
        scene.append(("box", (lo, lo + s)))
        solids.append(("box", lo, lo + s))
    for _ in range(2):
        r = rng.uniform(0.2, 0.4)
        c = np.array([rng.uniform(r + 0.3, ROOM_HI[0] - r - 0.3),
                      rng.uniform(r + 0.3, ROOM_HI[1] - r - 0.3),
                      rng.uniform(r, ROOM_HI[2] - r - 0.2)])
        scene.append(("sphere", (c, r)))
        solids.append(("sphere", c, r))
    return scene, solids


def _inside_solid(p, solids, margin=0.15):
    for s in solids:
        if s[0] == "box" and np.all(p > s[1] - margin) and np.all(p < s[2] + margin):
            return True
        if s[0] == "sphere" and np.linalg.norm(p - s[1]) < s[2] + margin:
            return True
    return False


def _pixel_rays():
    u = (np.arange(CAM_W) + 0.5) - CAM_W / 2.0
    v = (np.arange(CAM_H) + 0.5) - CAM_H / 2.0
    uu, vv = np.meshgrid(u, v)
    d = np.stack([uu.ravel() / CAM_F, vv.ravel() / CAM_F, np.ones(uu.size)], axis=1)
    return d


def _render(scene, c, R_wc):
    dc = _pixel_rays()
    dw = dc @ R_wc.T
    dw /= np.linalg.norm(dw, axis=1, keepdims=True)
    o = np.broadcast_to(c, dw.shape)
    t = _cast(o, dw, scene)
    depth = (t[:, None] * dw) @ R_wc[:, 2]
    return c + t[:, None] * dw, dw, t, depth


def _visible_fraction(scene, pts, c2, R_wc2):
    pc = (pts - c2) @ R_wc2
    z = pc[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        u = CAM_F * pc[:, 0] / z + CAM_W / 2.0
        v = CAM_F * pc[:, 1] / z + CAM_H / 2.0
    infr = (z > 0.05) & (u >= 0) & (u < CAM_W) & (v >= 0) & (v < CAM_H)
    dist = np.linalg.norm(pts - c2, axis=1)
    d = (pts - c2) / dist[:, None]
    t = _cast(np.broadcast_to(c2, d.shape), d, scene)
    unocc = t >= dist * (1.0 - 1e-6) - 1e-6
    return float(np.mean(infr & unocc))


def rgbd_room_pair(seed=SEED_BASE + 2, overlap=0.70, overlap_tol=0.03, max_angle_deg=45.0,
                   max_trans=0.3, outlier_ratio=0.05, depth_noise=0.002):
    """Two 160x125 depth views of a synthetic room (20,000 points each).

    View 1 is the target.  View 2 is chosen so that ``overlap`` +- ``overlap_tol`` of
    view-1 points lie in view-2's frustum and are unoccluded; it becomes the source
    after a rigid perturbation (angle U[0, max_angle], |t| U[0, max_trans]) about its
    centroid.  Depth noise along each ray has std ``depth_noise * depth^2``; a fraction
    ``outlier_ratio`` of each view is replaced by uniform points in that view's AABB.
    """
    rng = make_rng(seed)
    for _attempt in range(200):
        scene, solids = _room_scene(rng)
        c1 = np.array([rng.uniform(0.5, 1.2), rng.uniform(0.8, 3.2), rng.uniform(1.1, 1.6)])
        if _inside_solid(c1, solids):
            continue
        look = np.array([rng.uniform(3.0, 4.5), rng.uniform(1.2, 2.8), rng.uniform(0.6, 1.2)])
        R1 = _look_rotation(look - c1)
        pts1, _, _, _ = _render(scene, c1, R1)
        ok = False
        for _k in range(60):
            yaw = math.radians(rng.uniform(8.0, 30.0)) * (1 if rng.random() < 0.5 else -1)
            Rz = axis_angle_matrix(np.array([0.0, 0.0, 1.0]), yaw)
            c2 = c1 + rng.uniform(-0.3, 0.3, size=3) * np.array([1.0, 1.0, 0.3])
            if _inside_solid(c2, solids):
                continue
            R2 = Rz @ R1
            frac = _visible_fraction(scene, pts1, c2, R2)
            if abs(frac - overlap) <= overlap_tol:
                ok = True
                break
        if ok:
            break
    else:  # pragma: no cover - the search above always succeeds for the default seeds
        raise RuntimeError("could not place the second camera")

    def noisy_view(c, R):
        p, dw, t, depth = _render(scene, c, R)
        eps = rng.standard_normal(len(t)) * depth_noise * depth ** 2
        p = c + (t * (depth + eps) / depth)[:, None] * dw
        p, _ = _replace_outliers(rng, p, outlier_ratio)
        return p

    Y = noisy_view(c1, R1)
    P = noisy_view(c2, R2)
    R_p = random_rotation(rng, math.radians(rng.uniform(0.0, max_angle_deg)))
    t_p = rng.uniform(0.0, max_trans) * random_unit_vector(rng)
    centre = P.mean(axis=0)
    cam_source = R_p @ (c2 - centre) + centre + t_p  # the source camera moves with its view
    return _pair(Y, P, R_p, t_p, centre, name="rgbd_room", seed=seed, w=0.1, knn_k=10,
                 max_iters=50, overlap=frac, cam_target=c1, cam_source=cam_source)


def depth_confidence(points, camera, near=None):
    """Measurement confidence phi = e_min / e(x) for a depth sensor whose error
    grows with the squared depth, e(x) = k max(|x - camera|, near)^2 (k cancels),
    e_min = k near^2 the error at the sensor's near limit (default: the 5th
    percentile of the view's depths).  float32 in (0, 1]."""
    d = np.sqrt(((np.asarray(points, dtype=np.float64) - np.asarray(camera)) ** 2).sum(axis=1))
    near = float(np.percentile(d, 5.0)) if near is None else float(near)
    return np.minimum(1.0, (near / np.maximum(d, 1e-12)) ** 2).astype(np.float32)


# ---------------------------------------------------------------------------
# Workload 3: LiDAR-shaped pair (64 rings x 1563 azimuths)
# ---------------------------------------------------------------------------

def _lidar_scene(rng):
    scene = [("ground", 0.0)]
    for _ in range(20):
        while True:
            c = rng.uniform(-40.0, 40.0, size=2)
            if np.linalg.norm(c) > 4.0:
                break
        s = np.array([rng.uniform(1.0, 4.0), rng.uniform(1.0, 4.0), rng.uniform(1.0, 3.0)])
        lo = np.array([c[0] - s[0] / 2, c[1] - s[1] / 2, 0.0])
        scene.append(("box", (lo, lo + s)))
    for _ in range(10):
        while True:
            c = rng.uniform(-40.0, 40.0, size=2)
            if np.linalg.norm(c) > 4.0:
                break
        scene.append(("vcyl", (c[0], c[1], rng.uniform(0.2, 0.5), 0.0, rng.uniform(2.0, 5.0))))
    scene.append(("farwall", (0.0, 0.0, 80.0)))
    return scene


def _lidar_scan(rng, scene, origin, yaw, rings, azimuths, range_noise):
    el = np.radians(np.linspace(2.0, -24.8, rings))
    az = yaw + 2.0 * np.pi * np.arange(azimuths) / azimuths
    ee, aa = np.meshgrid(el, az, indexing="ij")
    d = np.stack([np.cos(ee) * np.cos(aa), np.cos(ee) * np.sin(aa), np.sin(ee)], axis=-1).reshape(-1, 3)
    o = np.broadcast_to(origin, d.shape)
    t = _cast(o, d, scene)
    t = t + range_noise * rng.standard_normal(len(t))
    return origin + t[:, None] * d


def lidar_pair(seed=SEED_BASE + 3, rings=64, azimuths=1563, range_noise=0.02, outlier_ratio=0.05,
               step=1.0, yaw_deg=10.0):
    """Two spinning-LiDAR scans (``rings * azimuths`` points) of a street-like scene.

    The sensor sits 1.73 m above the ground; the source scan is taken from a pose
    ``step`` metres away with a ``yaw_deg`` heading change.  Both scans are expressed
    in their own sensor frames, so the ground truth is that relative pose.
    """
    rng = make_rng(seed)
    scene = _lidar_scene(rng)
    h = 1.73
    o1 = np.array([0.0, 0.0, h])
    heading = rng.uniform(0.0, 2.0 * np.pi)
    o2 = o1 + step * np.array([math.cos(heading), math.sin(heading), 0.0])
    yaw = math.radians(yaw_deg)
    Y = _lidar_scan(rng, scene, o1, 0.0, rings, azimuths, range_noise)
    Pw = _lidar_scan(rng, scene, o2, yaw, rings, azimuths, range_noise)
    Y, _ = _replace_outliers(rng, Y, outlier_ratio)
    Pw, _ = _replace_outliers(rng, Pw, outlier_ratio)
    # express each scan in its sensor frame: p_s = Rz(yaw_s)^T (p_w - o_s)
    Rz2 = axis_angle_matrix(np.array([0.0, 0.0, 1.0]), yaw)
    Yl = Y - o1
    X = (Pw - o2) @ Rz2
    R_gt = Rz2
    t_gt = o2 - o1
    return dict(X=_f32(X), Y=_f32(Yl), R_gt=R_gt, t_gt=t_gt, name="lidar", seed=seed, w=0.1,
                knn_k=10, max_iters=50)


# ---------------------------------------------------------------------------
# Workload 4: a batch of independent uneven pairs
# ---------------------------------------------------------------------------

def _shape_cloud(rng, kind, n, noise, box_sides, ground):
    if kind == 0:
        return sphere_plane_cloud(rng, n, noise)
    if kind == 1:
        p = sample_box_surface(rng, n, -box_sides / 2, box_sides / 2)
    else:
        n_g = n // 2
        g = sample_rect(rng, n_g, (-1.5, -1.5, 0.0), (3.0, 0.0, 0.0), (0.0, 3.0, 0.0))
        b = sample_box_surface(rng, n - n_g, ground[0], ground[1], skip_bottom=True)
        p = np.concatenate([g, b], axis=0)[rng.permutation(n)]
    return p + noise * rng.standard_normal(p.shape)


def batch_pairs(seed=SEED_BASE + 4, num_pairs=256, n_lo=500, n_hi=20000, max_angle_deg=90.0,
                noise_rel=0.005):
    """``num_pairs`` independent pairs with N, M log-uniform integers in [n_lo, n_hi]."""
    rng = make_rng(seed)
    pairs = []
    for i in range(num_pairs):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        m = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        kind = int(rng.integers(0, 3))
        box_sides = rng.uniform(0.5, 1.5, size=3)
        lo = np.array([rng.uniform(-0.8, 0.2), rng.uniform(-0.8, 0.2), 0.0])
        ground = (lo, lo + rng.uniform(0.4, 0.9, size=3))
        scale = {0: 2.0, 1: float(np.linalg.norm(box_sides)), 2: 3.0}[kind]
        Y = _shape_cloud(rng, kind, m, noise_rel * scale, box_sides, ground)
        P = _shape_cloud(rng, kind, n, noise_rel * scale, box_sides, ground)
        diag = float(np.linalg.norm(Y.max(axis=0) - Y.min(axis=0)))
        R_p = random_rotation(rng, math.radians(rng.uniform(0.0, max_angle_deg)))
        t_p = rng.uniform(0.0, 0.1 * diag) * random_unit_vector(rng)
        pairs.append(_pair(Y, P, R_p, t_p, P.mean(axis=0), name=f"batch{i}", kind=kind))
    return pairs


# ---------------------------------------------------------------------------
# Workload 5: large range-scan pair from a union of superquadrics
# ---------------------------------------------------------------------------

def _sq_sign_pow(c, e):
    return np.sign(c) * np.abs(c) ** e


def _superquadric_points(rng, n, a, e1, e2, R, c):
    """Area-weighted samples of a superellipsoid surface (parametric grid + rejection)."""
    out = []
    need = n
    while need > 0:
        m = max(4 * need, 1024)
        eta = rng.uniform(-np.pi / 2, np.pi / 2, m)
        om = rng.uniform(-np.pi, np.pi, m)
        h = 1e-4

        def pt(et, o):
            ce, se = np.cos(et), np.sin(et)
            co, so = np.cos(o), np.sin(o)
            return np.stack([a[0] * _sq_sign_pow(ce, e1) * _sq_sign_pow(co, e2),
                             a[1] * _sq_sign_pow(ce, e1) * _sq_sign_pow(so, e2),
                             a[2] * _sq_sign_pow(se, e1)], axis=1)

        p0 = pt(eta, om)
        d_eta = (pt(eta + h, om) - p0) / h
        d_om = (pt(eta, om + h) - p0) / h
        dens = np.linalg.norm(np.cross(d_eta, d_om), axis=1)
        cap = np.quantile(dens, 0.995) + 1e-12
        keep = rng.random(m) * cap < np.minimum(dens, cap)
        sel = p0[keep][:need]
        out.append(sel)
        need -= len(sel)
    p = np.concatenate(out, axis=0)
    return p @ R.T + c


def superquadric_pair(seed=SEED_BASE + 5, n=500000, m=500000, num_shapes=8, noise_rel=0.002,
                      outlier_ratio=0.10, max_angle_deg=60.0):
    rng = make_rng(seed)
    shapes = []
    for _ in range(num_shapes):
        shapes.append(dict(a=rng.uniform(0.1, 0.4, 3), e1=rng.uniform(0.3, 1.5), e2=rng.uniform(0.3, 1.5),
                           R=random_rotation(rng, rng.uniform(0.0, np.pi)), c=rng.uniform(0.0, 1.0, 3)))
    weights = np.array([np.prod(s["a"]) ** (2.0 / 3.0) for s in shapes])

    def cloud(k):
        cnt = rng.multinomial(k, weights / weights.sum())
        pts = [_superquadric_points(rng, int(ci), s["a"], s["e1"], s["e2"], s["R"], s["c"])
               for s, ci in zip(shapes, cnt) if ci > 0]
        p = np.concatenate(pts, axis=0)[rng.permutation(k)]
        return p

    Y = cloud(m)
    diag = float(np.linalg.norm(Y.max(axis=0) - Y.min(axis=0)))
    P = cloud(n)
    Y = Y + noise_rel * diag * rng.standard_normal(Y.shape)
    P = P + noise_rel * diag * rng.standard_normal(P.shape)
    Y, _ = _replace_outliers(rng, Y, outlier_ratio)
    P, _ = _replace_outliers(rng, P, outlier_ratio)
    R_p = random_rotation(rng, math.radians(rng.uniform(0.0, max_angle_deg)))
    t_p = rng.uniform(0.0, 0.1 * diag) * random_unit_vector(rng)
    return _pair(Y, P, R_p, t_p, P.mean(axis=0), name="superquadrics", seed=seed, w=0.1, knn_k=10,
                 max_iters=50)


# ---------------------------------------------------------------------------
# Unstructured inputs for E-step unit tests
# ---------------------------------------------------------------------------

def estep_case(seed, n, m, alpha_max=2.0, spread=1.0, sigma2=None, angle_deg=20.0, trans=0.1,
               offset=(0.0, 0.0, 0.0)):
    """Random clouds in a cube of side ``spread`` (shifted by ``offset``), random unit
    normals, penalties uniform in [0, alpha_max], a random pose and a variance.

    ``sigma2`` defaults to a value that gives each source a few effective neighbours.
    """
    rng = make_rng(seed)
    off = np.asarray(offset, dtype=np.float64)
    Y = off + spread * rng.random((m, 3))
    X = off + spread * rng.random((n, 3))
    nrm = rng.standard_normal((m, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    alpha = alpha_max * rng.random(m)
    R = random_rotation(rng, math.radians(angle_deg))
    t = trans * random_unit_vector(rng)
    if sigma2 is None:
        sigma2 = (spread / max(m, 1) ** (1.0 / 3.0)) ** 2 * 2.0
    return dict(X=_f32(X), Y=_f32(Y), normals=_f32(nrm), alpha=_f32(alpha), R=R, t=t,
                sigma2=float(sigma2))
