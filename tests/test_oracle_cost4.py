"""Pins for the oracle's four-term cost (Eq. cost_function with Eqs.
cost_goal, cost_obs, cost_path, cost_smooth) on hand-built trajectories
whose terms are known in closed form: straight lines at constant speed and
constant acceleration (no jerk), a cubic (constant third difference), goal
and obstacle distances inside and outside the radius, both branches of the
path cost and their meeting point, and the saturation of the smoothness
term."""

import math

import numpy as np
import pytest

import oracle

DT = 1e-3


def _traj(fn, nk):
    """[1, nk + 1, 3] trajectory p_k = fn(k) (p_0 .. p_nk)."""
    return np.array([[fn(k) for k in range(nk + 1)]], dtype=np.float64)


def _costs(traj, m=None, goal=(0.0, 0.0, 0.0), r_c=0.05, a_max=10.0, w=(1, 1, 1, 1)):
    nk = traj.shape[1] - 1
    if m is None:
        m = np.full((1, nk), np.inf)
    return oracle.four_term_costs(traj, m, goal, DT, r_c, a_max, w)


def test_straight_line_constant_speed():
    # start 0.3 m from the goal, 1 mm per step toward it for N_k = 100 steps:
    # the candidate trajectory p_0 .. p_99 covers 99 mm of the 300 mm
    nk = 100
    tr = _traj(lambda k: (0.3 - 1e-3 * k, 0.0, 0.0), nk)
    c = _costs(tr)
    assert c["d1"][0] == pytest.approx(0.3, abs=1e-15)
    assert c["L"][0] == pytest.approx(0.099, rel=1e-12)
    assert c["path"][0] == pytest.approx(1.0 - 0.099 / 0.3, rel=1e-12)   # shorter branch
    assert c["J"][0] == pytest.approx(0.0, abs=1e-24)
    assert c["smooth"][0] == pytest.approx(0.0, abs=1e-15)
    assert c["goal"][0] == 1.0          # always beyond r_c = 5 cm
    assert c["obs"][0] == 0.0           # no obstacles: clearance inf


def test_path_cost_branches_meet_at_the_start_distance():
    nk = 50
    d1 = 0.2
    exact = _traj(lambda k: (d1 - d1 / (nk - 1) * k, 0.0, 0.0), nk)   # xi^N_k reaches the goal
    assert _costs(exact)["path"][0] == pytest.approx(0.0, abs=1e-12)
    # a detour of twice the length (its corner on a sample, k = 25 of 0 .. 50):
    # 1 - d1 / (2 d1) = 1/2
    nd = 51

    def detour(k):
        s = 2 * d1 * k / (nd - 1)              # arc length so far
        return (d1 - s, 0.0, 0.0) if s <= d1 else (0.0, s - d1, 0.0)
    c = _costs(_traj(detour, nd))
    assert c["L"][0] == pytest.approx(2 * d1, rel=1e-12)
    assert c["path"][0] == pytest.approx(0.5, rel=1e-12)
    # half the length, short branch: 1 - (d1 / 2) / d1 = 1/2
    half = _traj(lambda k: (d1 - 0.5 * d1 * k / (nk - 1), 0.0, 0.0), nk)
    assert _costs(half)["path"][0] == pytest.approx(0.5, rel=1e-12)
    # standing still at the goal
    assert _costs(_traj(lambda k: (0.0, 0.0, 0.0), nk))["path"][0] == 0.0


def test_constant_acceleration_has_no_jerk_and_a_cubic_has_a_known_one():
    nk = 80
    quad = _traj(lambda k: (0.5 + 0.3 * (k * DT) ** 2, 0.1, 0.2), nk)
    assert _costs(quad)["J"][0] == pytest.approx(0.0, abs=1e-22)
    c3 = 4.0
    cub = _traj(lambda k: (0.5, c3 * (k * DT) ** 3, 0.0), nk)
    c = _costs(cub, a_max=1.0)
    # third difference of c t^3 on a grid of step dt is 6 c dt^3, at the
    # N_k - 3 indices k = 4 .. N_k of the candidate trajectory
    J = (nk - 3) * (6 * c3 * DT ** 3) ** 2
    assert c["J"][0] == pytest.approx(J, rel=1e-6)
    assert c["smooth"][0] == pytest.approx(J / (nk * DT ** 4 * 1.0), rel=1e-6)
    # saturation at 1
    big = _traj(lambda k: (0.5, 1e4 * (k * DT) ** 3, 0.0), nk)
    assert _costs(big, a_max=1.0)["smooth"][0] == 1.0


def test_goal_and_obstacle_terms():
    nk = 40
    r_c = 0.05
    # first half of the candidate states at the goal, second half 2 r_c away
    tr = _traj(lambda k: (0.0, 0.0, 0.0) if k < nk // 2 else (2 * r_c, 0.0, 0.0), nk)
    assert _costs(tr, r_c=r_c)["goal"][0] == pytest.approx(0.5, rel=1e-15)
    # a quarter of the way inside: distance r_c / 4 everywhere -> 1/4
    inside = _traj(lambda k: (0.0, r_c / 4, 0.0), nk)
    assert _costs(inside, r_c=r_c)["goal"][0] == pytest.approx(0.25, rel=1e-14)
    # obstacle term: clearance >= r_c -> 0, clearance 0 -> 1, r_c / 2 -> 1/2,
    # penetration (negative clearance) -> above 1, as printed
    m = np.array([[r_c] * 10 + [0.0] * 10 + [r_c / 2] * 10 + [2 * r_c] * 10])
    c = _costs(tr, m=m, r_c=r_c)
    assert c["obs"][0] == pytest.approx((0 + 10 + 5 + 0) / 40, rel=1e-14)
    pen = _costs(tr, m=np.full((1, nk), -r_c / 2), r_c=r_c)
    assert pen["obs"][0] == pytest.approx(1.5, rel=1e-14)


def test_weights_combine_linearly():
    nk = 60
    tr = _traj(lambda k: (0.3 - 1e-3 * k, 2e3 * (k * DT) ** 3, 0.0), nk)
    m = np.linspace(0.0, 0.1, nk)[None, :]
    parts = _costs(tr, m=m, a_max=2.0)
    w = (0.7, 1.3, 2.0, 0.25)
    tot = _costs(tr, m=m, a_max=2.0, w=w)["C"][0]
    want = sum(wj * parts[k][0] for wj, k in zip(w, ("goal", "obs", "path", "smooth")))
    assert tot == pytest.approx(want, rel=1e-14)
    assert math.isfinite(tot)


def test_on_an_oracle_rollout():
    """The candidate path length is the rollout's path length without its
    last segment, d1 is the start's distance to the goal, and the obstacle
    term follows the rollout's clearance trace."""
    import synth
    w = synth.sphere_workload(n_agents=4, n_steps=120)
    f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    obs = np.stack([f["x"], f["y"], f["z"]])
    prm = w["params"]
    ro = oracle.rollout(obs, f["r_O"], w["agents"], prm, want_trace=True)
    c = oracle.four_term_costs(ro["traj"], ro["m_trace"], prm.goal, prm.dt, 0.1, 10.0)
    last = np.sqrt(((ro["traj"][:, -1] - ro["traj"][:, -2]) ** 2).sum(axis=1))
    assert np.allclose(c["L"] + last, ro["path_len"], rtol=1e-12, atol=0)
    start = np.asarray(w["agents"]["p0"], np.float64).T
    assert np.allclose(c["d1"], np.linalg.norm(start - np.asarray(prm.goal), axis=1), rtol=1e-12)
    assert np.all((c["obs"] >= 0) & (c["obs"] <= 1.5)) and np.any(c["obs"] > 0)
