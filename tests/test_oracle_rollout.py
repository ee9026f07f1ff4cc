"""Pins for the oracle's rollout (Sec. IV-A: F = f_a + f_r, vdot = I F,
v_k = v_(k-1) + 1/2 dt vdot, p_(k+1) = p_k + dt v_k) and its cost sums.

Closed forms and invariants, none of which re-types the stepping code:
  * pure circular field: the per-step identity |v_k|^2 - |v_(k-1)|^2 =
    |v_k - v_(k-1)|^2 (the force is orthogonal to the velocity it is
    evaluated with), and speed drift -> 0 at first order as dt -> 0 (the swirl
    leaves the energy unchanged, Sec. III);
  * analytic deflection: with every obstacle clamped and no gate, W is
    constant and the heading turns toward c with tan(theta/2) =
    tan(theta0/2) exp(-a t), a = 1/2 rho k_r W inv_mass, in the plane of (v0, c);
  * no obstacles: the critically damped ODE solution e(t) = (e0 + (e0' + w e0) t)
    exp(-w t), w = sqrt(k_a inv_mass / 2), is approached at first order, and
    the agent converges to the goal;
  * straight-line motion past one obstacle: path length and the clearance
    sequence follow from the geometry.
"""

import dataclasses
import math

import numpy as np
import pytest

import oracle
from synth.workloads import PhysicsParams


def _one_agent(p0, v0, c, k_r=1.0, k_a=1.0, r_d=0.05, r_a=0.0):
    col = lambda x: np.asarray(x, np.float64).reshape(3, 1)  # noqa: E731
    return {"p0": col(p0), "v0": col(v0), "c": col(c), "k_r": np.array([k_r]),
            "k_a": np.array([k_a]), "r_d": np.array([r_d]), "r_a": np.array([r_a])}


def _velocities(traj, dt):
    return np.diff(traj, axis=1) / dt


def test_pure_cf_speed_identity_and_convergence():
    g = np.random.Generator(np.random.PCG64(3))
    obs = np.stack([0.3 + 0.05 * g.standard_normal(400), 0.02 * g.standard_normal(400),
                    0.02 * g.standard_normal(400)])
    ag = _one_agent((0.0, 0.0, 0.0), (1.0, 0.05, 0.0), (0.0, 0.0, 1.0), k_r=1.0, k_a=0.0,
                    r_d=0.05)
    drifts = []
    for N, dt in ((400, 1e-3), (800, 5e-4), (1600, 2.5e-4)):
        prm = PhysicsParams(goal=(0.6, 0, 0), dt=dt, n_steps=N, damping=0.0, rho=0.05)
        ro = oracle.rollout(obs, 0.005, ag, prm)
        vel = _velocities(ro["traj"], dt)[0]
        v_all = np.vstack([ag["v0"].T, vel])           # v_(-1) = v0, v_0 .. v_(N-1)
        sq = (v_all ** 2).sum(axis=1)
        dv2 = (np.diff(v_all, axis=0) ** 2).sum(axis=1)
        assert np.allclose(np.diff(sq), dv2, rtol=1e-6, atol=1e-10)
        assert np.max(dv2) > 0                        # the field was active
        drifts.append(math.sqrt(sq[-1]) - math.sqrt(sq[0]))
    assert drifts[0] > 0
    assert 1.7 < drifts[0] / drifts[1] < 2.3 and 1.7 < drifts[1] / drifts[2] < 2.3


def _theta(v, c):
    return math.acos(np.clip(np.dot(v, c) / np.linalg.norm(v) / np.linalg.norm(c), -1, 1))


def test_analytic_deflection():
    obs = np.array([[0.01, -0.01, 0.0, 0.02], [0.0, 0.01, -0.01, 0.0], [0.0, 0.0, 0.01, -0.02]])
    n_obs = obs.shape[1]
    eps, rho, k_r, T_end = 10.0, 10.0, 1.0, 0.5
    W = n_obs / eps
    a = 0.5 * rho * k_r * W * 1.0
    v0 = np.array([1.0, 0.0, 0.0])
    c = np.array([math.cos(2.0), math.sin(2.0), 0.0])   # theta0 = 2 rad
    th0 = _theta(v0, c)
    exact = 2 * math.atan(math.tan(th0 / 2) * math.exp(-a * T_end))
    errs = []
    for N in (500, 1000, 2000):
        dt = T_end / N
        prm = PhysicsParams(goal=(0, 0, 0), dt=dt, n_steps=N, damping=0.0, rho=rho, eps=eps)
        ag = _one_agent((0, 0, 0), v0, c, k_r=k_r, k_a=0.0, r_d=math.inf)
        ro = oracle.rollout(obs, 0.005, ag, prm, want_traj=False, want_trace=True)
        assert np.allclose(ro["w_trace"], W, rtol=1e-14)
        vf = ro["v_final"][:, 0]
        assert abs(vf[2]) < 1e-12                      # stays in span(v0, c)
        errs.append(abs(_theta(vf, c) - exact))
    assert errs[0] < 0.02
    assert 1.7 < errs[0] / errs[1] < 2.3 and 1.7 < errs[1] / errs[2] < 2.3


def test_no_obstacles_critically_damped_ode():
    empty = np.zeros((3, 0))
    goal = np.array([0.8, 0.1, -0.2])
    p0, v0 = np.array([0.2, 0.0, 0.4]), np.array([0.3, -0.2, 0.1])
    k_a = 1.0
    w = math.sqrt(k_a / 2)
    T_end = 2.0
    e0, de0 = p0 - goal, v0
    exact = goal + (e0 + (de0 + w * e0) * T_end) * math.exp(-w * T_end)
    errs = []
    for N in (200, 400, 800):
        prm = PhysicsParams(goal=tuple(goal), dt=T_end / N, n_steps=N,
                            damping=2 * math.sqrt(2 * k_a), rho=0.05)
        ro = oracle.rollout(empty, 0.005, _one_agent(p0, v0, (0, 0, 1), k_a=k_a), prm)
        errs.append(np.linalg.norm(ro["p_final"][:, 0] - exact))
        assert ro["clear_pen"][0] == 0.0 and math.isinf(ro["min_clear"][0])
    assert 1.7 < errs[0] / errs[1] < 2.3 and 1.7 < errs[1] / errs[2] < 2.3
    prm = PhysicsParams(goal=tuple(goal), dt=1e-2, n_steps=6000, damping=2 * math.sqrt(2), rho=0.05)
    ro = oracle.rollout(empty, 0.005, _one_agent(p0, v0, (0, 0, 1)), prm, want_traj=False)
    assert np.linalg.norm(ro["p_final"][:, 0] - goal) < 1e-6 * np.linalg.norm(e0)


def test_straight_line_path_and_clearance():
    obs = np.array([[0.5], [0.02], [0.0]])
    r_O, dt, N = 0.005, 1e-3, 1000
    prm = PhysicsParams(goal=(0, 0, 0), dt=dt, n_steps=N, damping=0.0, rho=0.05,
                        clear_margin=0.03, clear_beta=100.0)
    ag = _one_agent((0, 0, 0), (1.0, 0, 0), (0, 0, 1), k_r=0.0, k_a=0.0)
    ro = oracle.rollout(obs, r_O, ag, prm, want_trace=True)
    assert ro["path_len"][0] == pytest.approx(N * dt * 1.0, rel=1e-12)
    x = np.arange(N) * dt
    m = np.sqrt((x - 0.5) ** 2 + 0.02 ** 2) - r_O
    assert np.allclose(ro["m_trace"][0], m, rtol=0, atol=1e-12)
    assert ro["min_clear"][0] == pytest.approx(0.015, abs=1e-12)
    bx = 100.0 * (0.03 - m)
    sp = np.where(bx > 0, bx + np.log1p(np.exp(-np.abs(bx))), np.log1p(np.exp(bx))) / 100.0
    assert ro["clear_pen"][0] == pytest.approx(sp.sum(), rel=1e-12)
    assert np.allclose(ro["traj"][0, -1], ro["p_final"][:, 0])
    assert np.allclose(ro["traj"][0, 0], 0.0)


def test_agents_independent():
    """Each agent's result does not depend on which other agents share the
    call (the basis of batching and serving)."""
    g = np.random.Generator(np.random.PCG64(11))
    obs = g.uniform(0.3, 0.5, (3, 300))
    n = 6
    ag = {"p0": np.tile([[0.2], [0.0], [0.4]], (1, n)), "v0": g.normal(0, 1, (3, n)),
          "c": g.normal(0, 1, (3, n)), "k_r": g.uniform(0.5, 2, n), "k_a": np.ones(n),
          "r_d": np.full(n, 0.05), "r_a": np.zeros(n)}
    prm = PhysicsParams(n_steps=150, rho=0.05)
    full = oracle.rollout(obs, 0.005, ag, prm)
    sub = {k: v[..., [4, 1]] for k, v in ag.items()}
    part = oracle.rollout(obs, 0.005, sub, prm)
    assert np.array_equal(part["traj"], full["traj"][[4, 1]])
    assert np.array_equal(part["path_len"], full["path_len"][[4, 1]])
