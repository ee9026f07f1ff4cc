"""Seeded scene generators: raw point clouds, depth frames and agent sets.

Everything here is input data.  Randomness comes from numpy's PCG64 generator
seeded per call, so the same seed gives the same bytes on every run of this
image.  Values are produced in float64 and rounded to float32 once, which is
the precision the planner receives from a sensor.

The scene shapes follow the tabletop manipulation workloads of the paper's
evaluation (Sec. VI, Fig. 4 scenes: a table with boxes and cylinders; Sec. VI-C
real-world setup with a depth camera), which are not published as data.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


# ---------------------------------------------------------------------------
# Sphere-surface cloud (the single-obstacle workload)
# ---------------------------------------------------------------------------

def sphere_cloud(n: int, seed: int, radius: float = 0.10,
                 centre=(0.5, 0.0, 0.4), jitter: float = 0.002) -> np.ndarray:
    """``n`` points uniform on a sphere surface plus isotropic Gaussian jitter.

    Directions are normalised standard-normal vectors (uniform on the sphere).
    Returns float32 ``[n, 3]`` (AoS xyz, metres).
    """
    g = _rng(seed)
    d = g.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pts = np.asarray(centre, dtype=np.float64) + radius * d
    pts += g.normal(0.0, jitter, size=(n, 3))
    return np.ascontiguousarray(pts.astype(np.float32))


# ---------------------------------------------------------------------------
# Tabletop scene and depth-camera rendering by analytic ray casting
# ---------------------------------------------------------------------------

@dataclass
class TabletopScene:
    """A table plane z=0 with axis-aligned boxes, vertical cylinders and spheres."""

    boxes: list = field(default_factory=list)      # (xmin, ymin, zmin, xmax, ymax, zmax)
    cylinders: list = field(default_factory=list)  # (cx, cy, r, h)
    spheres: list = field(default_factory=list)    # (cx, cy, cz, r)


def tabletop_scene(seed: int, n_boxes: int = 3, n_cyl: int = 2) -> TabletopScene:
    """Table + ``n_boxes`` boxes (sides U[5,20] cm) + ``n_cyl`` cylinders
    (radius U[3,8] cm, height U[10,30] cm), all resting on the table, with
    centres drawn in x in [0.25, 0.75], y in [-0.3, 0.3]."""
    g = _rng(seed)
    sc = TabletopScene()
    for _ in range(n_boxes):
        sx, sy, sz = g.uniform(0.05, 0.20, size=3)
        cx, cy = g.uniform(0.25, 0.75), g.uniform(-0.3, 0.3)
        sc.boxes.append((cx - sx / 2, cy - sy / 2, 0.0, cx + sx / 2, cy + sy / 2, sz))
    for _ in range(n_cyl):
        r = g.uniform(0.03, 0.08)
        h = g.uniform(0.10, 0.30)
        cx, cy = g.uniform(0.25, 0.75), g.uniform(-0.3, 0.3)
        sc.cylinders.append((cx, cy, r, h))
    return sc


def camera_pose(position=(0.5, -0.4, 1.2), target=(0.5, 0.0, 0.0)):
    """World-from-camera rotation (columns = camera x right, y down, z forward)
    and the camera position, for a pinhole camera looking at ``target``."""
    pos = np.asarray(position, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - pos
    fwd /= np.linalg.norm(fwd)
    up = np.array([0.0, 0.0, 1.0])
    xc = np.cross(fwd, up)
    xc /= np.linalg.norm(xc)
    yc = np.cross(fwd, xc)
    R = np.stack([xc, yc, fwd], axis=1)
    return R, pos


def _hit_plane_z0(o, d):
    t = np.full(d.shape[0], np.inf)
    m = d[:, 2] < 0
    t[m] = -o[2] / d[m, 2]
    return t


def _hit_box(o, d, box):
    lo = np.asarray(box[:3])
    hi = np.asarray(box[3:])
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        t1 = (lo - o) * inv
        t2 = (hi - o) * inv
    tmin = np.nanmax(np.minimum(t1, t2), axis=1)
    tmax = np.nanmin(np.maximum(t1, t2), axis=1)
    hit = (tmax >= tmin) & (tmax > 0)
    t = np.where(tmin > 0, tmin, tmax)
    return np.where(hit, t, np.inf)


def _hit_cylinder(o, d, cyl):
    cx, cy, r, h = cyl
    ox, oy = o[0] - cx, o[1] - cy
    a = d[:, 0] ** 2 + d[:, 1] ** 2
    b = 2.0 * (ox * d[:, 0] + oy * d[:, 1])
    c = ox * ox + oy * oy - r * r
    disc = b * b - 4 * a * c
    t_side = np.full(d.shape[0], np.inf)
    ok = (disc >= 0) & (a > 0)
    sq = np.sqrt(np.where(ok, disc, 0.0))
    with np.errstate(divide="ignore", invalid="ignore"):
        t0 = (-b - sq) / (2 * a)
    z0 = o[2] + t0 * d[:, 2]
    good = ok & (t0 > 0) & (z0 >= 0) & (z0 <= h)
    t_side[good] = t0[good]
    # top cap
    t_cap = np.full(d.shape[0], np.inf)
    m = d[:, 2] < 0
    tc = (h - o[2]) / np.where(m, d[:, 2], -1.0)
    px = ox + tc * d[:, 0]
    py = oy + tc * d[:, 1]
    capok = m & (tc > 0) & (px * px + py * py <= r * r)
    t_cap[capok] = tc[capok]
    return np.minimum(t_side, t_cap)


def _hit_sphere(o, d, sph):
    c = np.asarray(sph[:3])
    r = sph[3]
    oc = o - c
    a = np.einsum("ij,ij->i", d, d)
    b = 2.0 * (d @ oc)
    cc = oc @ oc - r * r
    disc = b * b - 4 * a * cc
    ok = disc >= 0
    sq = np.sqrt(np.where(ok, disc, 0.0))
    t0 = (-b - sq) / (2 * a)
    return np.where(ok & (t0 > 0), t0, np.inf)


def render_depth_frame(scene: TabletopScene, seed: int, width: int = 640,
                       height: int = 480, fx: float = 525.0, fy: float = 525.0,
                       cx: float = 319.5, cy: float = 239.5,
                       cam_position=(0.5, -0.4, 1.2), cam_target=(0.5, 0.0, 0.0),
                       depth_noise: float = 0.002, nan_frac: float = 0.05,
                       n_points: int | None = None):
    """Render an organised depth cloud of ``scene`` in the camera frame.

    Each pixel's ray is intersected analytically with the table plane, boxes,
    cylinders and spheres; the nearest hit's camera-frame depth gets
    N(0, depth_noise) noise along the ray; a Bernoulli(nan_frac) dropout and
    rays that miss everything give NaN rows.  With ``n_points`` a seeded subset
    of pixels (without replacement, in pixel order) is returned instead of the
    full frame.

    Returns ``(xyz_cam float32 [N,3], T_cam_to_world float32 [12])`` where the
    transform is row-major 3x4 ``[R | t]`` mapping camera to world.
    """
    g = _rng(seed)
    R, pos = camera_pose(cam_position, cam_target)
    u, v = np.meshgrid(np.arange(width, dtype=np.float64),
                       np.arange(height, dtype=np.float64))
    u = u.reshape(-1)
    v = v.reshape(-1)
    if n_points is not None:
        sel = np.sort(g.choice(width * height, size=n_points, replace=False))
        u, v = u[sel], v[sel]
    dcam = np.stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u)], axis=1)
    dworld = dcam @ R.T
    t = _hit_plane_z0(pos, dworld)
    for b in scene.boxes:
        t = np.minimum(t, _hit_box(pos, dworld, b))
    for c in scene.cylinders:
        t = np.minimum(t, _hit_cylinder(pos, dworld, c))
    for s in scene.spheres:
        t = np.minimum(t, _hit_sphere(pos, dworld, s))
    # dcam has unit z, so the ray parameter t is the camera-frame depth.
    depth = t + g.normal(0.0, depth_noise, size=t.shape)
    drop = g.random(t.shape) < nan_frac
    depth[drop | ~np.isfinite(t)] = np.nan
    xyz = dcam * depth[:, None]
    T = np.concatenate([R, pos[:, None]], axis=1).reshape(-1)
    return (np.ascontiguousarray(xyz.astype(np.float32)),
            np.ascontiguousarray(T.astype(np.float32)))


# ---------------------------------------------------------------------------
# Agents
# ---------------------------------------------------------------------------

def agent_set(n: int, seed: int, start, goal, speed: float = 1.0,
              speed_noise: float = 0.1, k_r_range=(0.5, 2.0), k_a: float = 1.0,
              r_d: float = 0.05, r_a: float = 0.0) -> dict:
    """Point-mass planning agents (Sec. IV-A, agent set and its heuristic parameters).

    All start at ``start``.  Initial velocity = ``speed`` toward the goal plus
    N(0, speed_noise) per axis; current vector c = a normalised standard-normal
    vector; field gain k_r ~ U[k_r_range]; attractive gain k_a, detection
    radius r_d and agent radius r_a are constant.

    Returns float32 SoA arrays: ``p0, v0, c`` of shape ``[3, n]`` and
    ``k_r, k_a, r_d, r_a`` of shape ``[n]``.
    """
    g = _rng(seed)
    start = np.asarray(start, dtype=np.float64)
    goal = np.asarray(goal, dtype=np.float64)
    u = (goal - start) / np.linalg.norm(goal - start)
    v0 = speed * u[None, :] + g.normal(0.0, speed_noise, size=(n, 3))
    c = g.standard_normal((n, 3))
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    k_r = g.uniform(k_r_range[0], k_r_range[1], size=n)
    f32 = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.float32))  # noqa: E731
    return {
        "p0": f32(np.repeat(start[:, None], n, axis=1)),
        "v0": f32(v0.T),
        "c": f32(c.T),
        "k_r": f32(k_r),
        "k_a": f32(np.full(n, k_a)),
        "r_d": f32(np.full(n, r_d)),
        "r_a": f32(np.full(n, r_a)),
    }


def moving_spheres(seed: int, n: int = 4):
    """Sphere obstacles on sinusoidal paths: radius U[4,10] cm, amplitude
    0.2 m, frequency U[0.2,1] Hz, seeded phase and unit axis; returns a
    function of time giving ``[(cx, cy, cz, r), ...]``."""
    g = _rng(seed)
    p0 = np.stack([g.uniform(0.3, 0.7, n), g.uniform(-0.25, 0.25, n),
                   g.uniform(0.15, 0.45, n)], axis=1)
    r = g.uniform(0.04, 0.10, n)
    f = g.uniform(0.2, 1.0, n)
    phi = g.uniform(0.0, 2 * math.pi, n)
    ax = g.standard_normal((n, 3))
    ax /= np.linalg.norm(ax, axis=1, keepdims=True)

    def at(t: float):
        c = p0 + 0.2 * np.sin(2 * math.pi * f * t + phi)[:, None] * ax
        return [(float(c[i, 0]), float(c[i, 1]), float(c[i, 2]), float(r[i]))
                for i in range(n)]

    return at
