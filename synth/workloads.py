"""The five synthetic workloads: seeds, shapes and the physical constants.

A workload is plain data: a raw cloud (or an obstacle set), a camera
transform, a voxel workspace, an agent set and the rollout/cost constants.
The constants the paper leaves open (inertia, damping, repulsive scale,
initial speed, detection radius, clamp) are fixed here once, and both the
CUDA path and the oracle read them from here.

Seeds: ``1000 + workload id``; per-scene sub-seeds come from numpy's
SeedSequence spawned from that seed.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

from .scenes import (sphere_cloud, tabletop_scene, render_depth_frame,
                     agent_set, moving_spheres, _rng)

IDENTITY_T = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], dtype=np.float32)


@dataclass
class Workspace:
    """Voxel grid of the workspace: lower corner ``lo`` (m), edge ``voxel``
    (m, = 2 r_O), cell counts ``dims``; the upper corner is lo + dims*voxel.
    Voxels with fewer than ``min_pts`` points are dropped."""

    lo: tuple
    voxel: float
    dims: tuple
    min_pts: int = 1

    @property
    def r_O(self) -> float:
        return float(np.float32(self.voxel) * np.float32(0.5))


@dataclass
class PhysicsParams:
    """Rollout and cost constants (Sec. IV-A agent model, Eq. for F, f_a, the
    velocity and pose updates; Sec. IV-A cost)."""

    goal: tuple = (0.8, 0.0, 0.4)
    dt: float = 1e-3            # delta_t (s)
    n_steps: int = 200          # N_k
    damping: float = 2.0 * math.sqrt(2.0)   # D = d I_3, critical for k_a = 1
    inv_mass: float = 1.0       # inertia tensor = inv_mass I_3
    rho: float = 1e-2           # repulsive scale: k_f = rho * k_r
    eps: float = 1e-3           # minimum acceptable distance (clamp)
    vel_half: float = 0.5       # the 1/2 in the velocity update
    clear_margin: float = 0.03  # clearance-penalty margin (m)
    clear_beta: float = 100.0   # softplus sharpness (1/m)
    ckpt_every: int = 50        # adjoint checkpoint interval
    w_path: float = 1.0
    w_goal: float = 10.0
    w_clear: float = 0.0
    # four-term cost (Eq. cost_function): weights of the goal, obstacle, path
    # and smoothness terms, the radius r_c of the goal/obstacle terms and the
    # acceleration bound a_max normalising the jerk
    w4: tuple = (1.0, 1.0, 1.0, 1.0)
    cost_radius: float = 0.05
    a_max: float = 50.0

    def as_dict(self) -> dict:
        return asdict(self)


def _sub_seeds(seed: int, n: int):
    return [int(s.generate_state(1)[0]) for s in np.random.SeedSequence(seed).spawn(n)]


SPHERE_WS = Workspace(lo=(0.0, -0.5, 0.0), voxel=0.01, dims=(100, 100, 80))
TABLE_WS = Workspace(lo=(0.0, -0.5, -0.02), voxel=0.005, dims=(200, 200, 160))
SPHERE_START, SPHERE_GOAL = (0.2, 0.0, 0.4), (0.8, 0.0, 0.4)
TABLE_START, TABLE_GOAL = (0.15, 0.0, 0.10), (0.85, 0.0, 0.10)

# Repulsive scales chosen so that the largest per-step turn of the velocity,
# 1/2 dt rho k_r W, stays at or below about 0.1 rad on each workload's densest
# approach.  W grows with the number of obstacle primitives per unit of
# surface, i.e. as 1/voxel^2, so the scale is quoted at a reference voxel and
# multiplied by (voxel / reference)^2.
RHO_SPHERE = 5e-2       # at 1 cm voxels
RHO_TABLE = 3e-3        # at 5 mm voxels
RHO_DENSE = 1e-4        # raw 50k-point cloud, no detection gate
INITIAL_SPEED = 1.0


def sphere_workload(seed: int = 1001, n_raw: int = 20000, voxel: float = 0.01,
                    n_agents: int = 8, n_steps: int = 200) -> dict:
    """Single query on a sphere-surface cloud: 20,000 points, radius 0.10 m,
    centre (0.5, 0, 0.4), 2 mm jitter, voxel 1 cm; 8 agents, 200 steps."""
    s_cloud, s_agents = _sub_seeds(seed, 2)
    xyz = sphere_cloud(n_raw, s_cloud)
    extent = (1.0, 1.0, 0.8)
    dims = tuple(int(math.ceil(e / voxel - 1e-9)) for e in extent)
    ws = Workspace(lo=SPHERE_WS.lo, voxel=voxel, dims=dims)
    agents = agent_set(n_agents, s_agents, SPHERE_START, SPHERE_GOAL, speed=INITIAL_SPEED)
    prm = PhysicsParams(goal=SPHERE_GOAL, n_steps=n_steps,
                        rho=RHO_SPHERE * (voxel / 0.01) ** 2)
    return {"name": f"sphere{n_raw}_v{voxel*1000:g}mm_na{n_agents}_nk{n_steps}",
            "xyz": xyz, "T": IDENTITY_T.copy(), "workspace": ws,
            "agents": agents, "params": prm}


def tabletop_workload(seed: int = 1002, n_agents: int = 256, n_steps: int = 500,
                      n_points: int | None = None, voxel: float = 0.005,
                      spheres_at: float | None = None, sphere_seed: int | None = None,
                      scene_seed: int | None = None, frame_seed: int | None = None) -> dict:
    """Tabletop depth frame: 640x480 render of a table, 3 boxes and 2
    cylinders, 2 mm depth noise, 5% NaN dropouts; workspace 1 x 1 x 0.8 m at
    5 mm voxels; 256 agents, 500 steps."""
    s_scene, s_frame, s_agents = _sub_seeds(seed, 3)
    scene = tabletop_scene(s_scene if scene_seed is None else scene_seed)
    if spheres_at is not None:
        scene.spheres = moving_spheres(sphere_seed if sphere_seed is not None else seed)(spheres_at)
    xyz, T = render_depth_frame(scene, s_frame if frame_seed is None else frame_seed,
                                n_points=n_points)
    extent = (1.0, 1.0, 0.8)
    dims = tuple(int(math.ceil(e / voxel - 1e-9)) for e in extent)
    ws = Workspace(lo=TABLE_WS.lo, voxel=voxel, dims=dims)
    agents = agent_set(n_agents, s_agents, TABLE_START, TABLE_GOAL, speed=INITIAL_SPEED)
    prm = PhysicsParams(goal=TABLE_GOAL, n_steps=n_steps,
                        rho=RHO_TABLE * (voxel / 0.005) ** 2)
    return {"name": f"tabletop640x480_v{voxel*1000:g}mm_na{n_agents}_nk{n_steps}",
            "xyz": xyz, "T": T, "workspace": ws, "agents": agents, "params": prm,
            "scene": scene}


# Heterogeneous ensemble (the paper's multi-agent runs: two agents per
# heuristic, one with a large and one with a small detection radius).  The
# APF term grows as |d|^-3 where the MFI weight grows as 1/|d|, so APF gains
# are scaled down to give forces of the same order near the obstacles.
APF_GAIN = 1e-3
R_D_SMALL, R_D_LARGE = 0.05, 0.10


def ensemble_agents(agents: dict, n_apf: int, apf_gain: float = APF_GAIN,
                    r_d=(R_D_SMALL, R_D_LARGE)) -> dict:
    """An agent set turned into a heterogeneous ensemble: the last ``n_apf``
    agents are the APF ones (gains k_r scaled by ``apf_gain``), the others
    MFI; within each heuristic the detection radius alternates small, large."""
    ag = {k: np.array(v, copy=True) for k, v in agents.items()}
    n = ag["k_r"].size
    nm = n - n_apf
    idx = np.arange(n)
    local = np.where(idx < nm, idx, idx - nm)
    ag["r_d"] = np.where(local % 2 == 0, r_d[0], r_d[1]).astype(np.float32)
    ag["k_r"][nm:] = (ag["k_r"][nm:].astype(np.float64) * apf_gain).astype(np.float32)
    return ag


# Depth cameras of the multi-sensor frames (the paper's real-world runs use
# two RealSense cameras at 848x480); all look at the table centre.
SENSOR_POSITIONS = ((0.5, -0.4, 1.2), (0.5, 0.45, 1.1), (-0.3, 0.0, 1.0))


def multi_sensor_frames(seed: int = 1006, n_sensors: int = 2, width: int = 848,
                        height: int = 480, fx: float = 425.0, n_points: int | None = None) -> dict:
    """The tabletop scene seen by ``n_sensors`` depth cameras at once: one
    organised cloud per sensor in its own camera frame with its
    camera-to-world transform, 2 mm depth noise and 5% dropouts each."""
    subs = _sub_seeds(seed, 1 + n_sensors)
    scene = tabletop_scene(subs[0])
    clouds = []
    for s in range(n_sensors):
        xyz, T = render_depth_frame(scene, subs[1 + s], width=width, height=height, fx=fx, fy=fx,
                                    cx=(width - 1) / 2.0, cy=(height - 1) / 2.0,
                                    cam_position=SENSOR_POSITIONS[s % len(SENSOR_POSITIONS)],
                                    n_points=n_points)
        clouds.append((xyz, T))
    return {"clouds": clouds, "workspace": TABLE_WS, "scene": scene}


def batch_workloads(seed: int = 1003, n_scenes: int = 64) -> list:
    """64 uneven sphere-cloud queries: raw points log-uniform in [5k, 300k],
    voxel U[4, 10] mm, agents log-uniform in {32..1024}, steps U{100..1000}."""
    g = _rng(seed)
    out = []
    subs = _sub_seeds(seed, n_scenes)
    for q in range(n_scenes):
        n_raw = int(round(math.exp(g.uniform(math.log(5e3), math.log(3e5)))))
        voxel = float(np.float32(g.uniform(0.004, 0.010)))
        n_agents = int(round(math.exp(g.uniform(math.log(32), math.log(1024)))))
        n_steps = int(g.integers(100, 1001))
        out.append(sphere_workload(seed=subs[q], n_raw=n_raw, voxel=voxel,
                                   n_agents=n_agents, n_steps=n_steps))
    return out


def adjoint_workload(seed: int = 1004, n_obs: int = 50000, n_agents: int = 512,
                     n_steps: int = 1000) -> dict:
    """Differentiable rollout: 50,000 sphere-cloud points used directly as
    obstacles (r_O = 5 mm), no detection gate, 512 agents, 1000 steps; cost =
    path length + 10 goal distance + softplus clearance penalty (3 cm)."""
    s_cloud, s_agents = _sub_seeds(seed, 2)
    obs = sphere_cloud(n_obs, s_cloud)
    agents = agent_set(n_agents, s_agents, SPHERE_START, SPHERE_GOAL,
                       speed=INITIAL_SPEED, r_d=math.inf)
    prm = PhysicsParams(goal=SPHERE_GOAL, n_steps=n_steps, rho=RHO_DENSE,
                        w_clear=1.0)
    return {"name": f"dense{n_obs}_na{n_agents}_nk{n_steps}",
            "obstacles": np.ascontiguousarray(obs.T), "r_O": 0.005,
            "agents": agents, "params": prm}


def serve_stream(seed: int = 1005, n_requests: int = 10000, rate_hz: float = 1000.0,
                 n_points: int = 200000, n_steps: int = 300):
    """Control-rate request stream: arrivals every 1/rate_hz s (open loop);
    request r carries a 200k-point frame of the tabletop scene plus 4 moving
    spheres at its arrival time, and asks for N_a in {64, 256, 1024} agents
    with 300 steps.  Returns (arrival times, a function r -> workload)."""
    g = _rng(seed)
    na_choice = g.choice(np.array([64, 256, 1024]), size=n_requests)
    arrivals = np.arange(n_requests, dtype=np.float64) / rate_hz
    subs = _sub_seeds(seed, n_requests)

    def request(r: int) -> dict:
        return tabletop_workload(seed=subs[r], n_agents=int(na_choice[r]), n_steps=n_steps,
                                 n_points=n_points, voxel=0.01, spheres_at=float(arrivals[r]),
                                 sphere_seed=seed, scene_seed=seed)

    return arrivals, na_choice, request
