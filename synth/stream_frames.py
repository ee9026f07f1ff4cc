"""The served request stream's depth frames, rendered many at a time.

The served control loop takes a request every millisecond for 10 s, each
with its own 200,000-point frame of the tabletop scene with four spheres on
sinusoidal paths, seen at the request's arrival time.  Ten thousand such
frames take minutes to ray-cast one by one on the host, so this module casts
them in torch, on any device, a chunk of frames at a time: the rays of the
static scene (table, boxes, cylinders) are intersected once, on the host,
by the same analytic ray caster as ``scenes.render_depth_frame``; each frame
then draws its pixel subset, intersects the selected rays with the four
spheres at its time, and adds its depth noise and dropouts.

Frames are seeded per chunk of ``CHUNK`` frames (a torch generator on the
rendering device), so the same stream is drawn on every run of one device
type; they follow the recipe of ``render_depth_frame`` (pixel subset without
replacement in pixel order, N(0, 2 mm) noise along the ray, 5% Bernoulli
dropouts, NaN where a ray misses everything) but are not bit-identical to it:
its generator is numpy's.  Input generation only: none of the planning
method's arithmetic is here.
"""

from __future__ import annotations

import numpy as np

from .scenes import (_hit_box, _hit_cylinder, _hit_plane_z0, camera_pose, moving_spheres,
                     tabletop_scene)

CHUNK = 64


class StreamFrames:
    """Renderer of the stream's frames: ``render(times, first)`` returns the
    frames of requests first .. first+len(times)-1 (arrival times ``times``)
    as a float32 tensor [F, n_points, 3] on ``device``, camera frame; ``T``
    is the shared camera-to-world transform."""

    def __init__(self, seed: int = 1005, n_points: int = 200000, width: int = 640,
                 height: int = 480, fx: float = 525.0, fy: float = 525.0, cx: float = 319.5,
                 cy: float = 239.5, cam_position=(0.5, -0.4, 1.2), cam_target=(0.5, 0.0, 0.0),
                 depth_noise: float = 0.002, nan_frac: float = 0.05, device="cpu"):
        import torch
        self.seed, self.n_points = int(seed), int(n_points)
        self.depth_noise, self.nan_frac = float(depth_noise), float(nan_frac)
        self.device = torch.device(device)
        scene = tabletop_scene(seed)
        self.spheres_at = moving_spheres(seed)
        R, pos = camera_pose(cam_position, cam_target)
        u, v = np.meshgrid(np.arange(width, dtype=np.float64), np.arange(height, dtype=np.float64))
        u, v = u.reshape(-1), v.reshape(-1)
        dcam = np.stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u)], axis=1)
        dworld = dcam @ R.T
        t = _hit_plane_z0(pos, dworld)
        for b in scene.boxes:
            t = np.minimum(t, _hit_box(pos, dworld, b))
        for c in scene.cylinders:
            t = np.minimum(t, _hit_cylinder(pos, dworld, c))
        f64 = dict(dtype=torch.float64, device=self.device)
        self.n_pix = width * height
        self.dcam = torch.as_tensor(dcam, **f64)
        self.dworld = torch.as_tensor(dworld, **f64)
        self.t_static = torch.as_tensor(t, **f64)
        self.pos = torch.as_tensor(pos, **f64)
        self.T = np.ascontiguousarray(np.concatenate([R, pos[:, None]], axis=1).reshape(-1)
                                      .astype(np.float32))

    def render(self, times, first: int, noise: bool = True):
        """Frames of requests first .. first + len(times) - 1; ``first`` must
        be a multiple of CHUNK when len(times) > CHUNK (chunks are seeded by
        index).  ``noise=False`` renders exact depths of every pixel in
        pixel order (no subset, noise or dropouts)."""
        import torch
        times = np.asarray(times, dtype=np.float64)
        out = []
        for c0 in range(0, times.size, CHUNK):
            out.append(self._chunk(times[c0:c0 + CHUNK], first + c0, noise))
        return torch.cat(out, dim=0)

    def _chunk(self, times, first, noise):
        import torch
        F = times.size
        g = torch.Generator(device=self.device)
        g.manual_seed(self.seed * 1_000_003 + first // CHUNK)
        if noise:
            keys = torch.rand(F, self.n_pix, generator=g, device=self.device)
            sel = keys.argsort(dim=1)[:, :self.n_points].sort(dim=1).values
        else:
            sel = torch.arange(self.n_pix, device=self.device).expand(F, -1)
        n = sel.shape[1]
        d = self.dworld[sel]                               # [F, n, 3]
        t = self.t_static[sel].clone()                     # [F, n]
        sph = torch.as_tensor(np.array([self.spheres_at(float(tt)) for tt in times]),
                              dtype=torch.float64, device=self.device)  # [F, 4, (cx, cy, cz, r)]
        a = (d * d).sum(-1)
        for s in range(sph.shape[1]):
            oc = self.pos[None, :] - sph[:, s, :3]        # [F, 3]
            b = 2.0 * (d * oc[:, None, :]).sum(-1)
            cc = (oc * oc).sum(-1) - sph[:, s, 3] ** 2     # [F]
            disc = b * b - 4.0 * a * cc[:, None]
            ok = disc >= 0
            sq = torch.sqrt(torch.where(ok, disc, torch.zeros_like(disc)))
            t0 = (-b - sq) / (2.0 * a)
            hit = ok & (t0 > 0)
            t = torch.minimum(t, torch.where(hit, t0, torch.full_like(t0, float("inf"))))
        depth = t
        if noise:
            depth = t + self.depth_noise * torch.randn(F, n, generator=g, dtype=torch.float64,
                                                       device=self.device)
            drop = torch.rand(F, n, generator=g, device=self.device) < self.nan_frac
            depth = torch.where(drop | ~torch.isfinite(t), torch.full_like(t, float("nan")), depth)
        else:
            depth = torch.where(torch.isfinite(t), t, torch.full_like(t, float("nan")))
        xyz = self.dcam[sel] * depth[..., None]
        return xyz.to(torch.float32)
