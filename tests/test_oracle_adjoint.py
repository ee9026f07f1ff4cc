"""Pins for the oracle's discrete adjoint of the rollout cost.

  * FP64 central finite differences (h = 1e-6) of the cost, on samples whose
    branch signature (clamped pairs, gated-in pairs, nearest obstacle per
    step) does not change within +-h;
  * a closed form: with no field (k_r = 0), no attractor and no damping the
    agent moves in a straight line, p_N = p_0 + N dt v0 and L = N dt |v0|,
    so dC/dv0 = N dt (w_path v0/|v0| + w_goal (p_N - g)/|p_N - g|);
  * the adjoint's cost equals the rollout's cost.
"""

import dataclasses
import math

import numpy as np
import pytest

import oracle
import synth
from synth.workloads import PhysicsParams


def _check_fd(obs, r_O, agents, prm, ids, tol=1e-6, min_valid=0.75):
    adj = oracle.adjoint(obs, r_O, agents, prm)
    fd = oracle.fd_gradient(obs, r_O, agents, prm, ids)
    n_valid = n_total = 0
    for i, (g, ok) in fd.items():
        a = oracle.grad_vector(adj, i)
        scale = np.abs(g).max()
        assert scale > 0
        err = np.abs(a - g)[ok]
        assert np.all(err <= tol * scale + 1e-10), (i, err.max() / scale)
        n_valid += ok.sum()
        n_total += ok.size
    assert n_valid >= min_valid * n_total, f"only {n_valid}/{n_total} FD samples without a kink"


def test_dense_no_gate_with_clearance_penalty():
    w = synth.adjoint_workload(n_obs=3000, n_agents=6, n_steps=200)
    _check_fd(w["obstacles"], w["r_O"], w["agents"], w["params"], range(6))


def test_gated_sphere_workload():
    w = synth.sphere_workload(n_agents=6, n_steps=200)
    f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    obs = np.stack([f["x"], f["y"], f["z"]])
    prm = dataclasses.replace(w["params"], w_clear=1.0)
    _check_fd(obs, f["r_O"], w["agents"], prm, range(6))


def test_straight_line_closed_form():
    obs = np.array([[0.5], [0.3], [0.0]])
    N, dt = 300, 1e-3
    prm = PhysicsParams(goal=(0.4, 0.1, -0.1), dt=dt, n_steps=N, damping=0.0, rho=0.05,
                        w_path=1.3, w_goal=10.0, w_clear=0.0)
    v0 = np.array([0.7, -0.2, 0.4])
    ag = {"p0": np.zeros((3, 1)), "v0": v0.reshape(3, 1), "c": np.array([[0.0], [0.0], [1.0]]),
          "k_r": np.zeros(1), "k_a": np.zeros(1), "r_d": np.full(1, 0.05), "r_a": np.zeros(1)}
    adj = oracle.adjoint(obs, 0.005, ag, prm)
    pN = N * dt * v0
    e = pN - np.asarray(prm.goal)
    expect = N * dt * (prm.w_path * v0 / np.linalg.norm(v0) + prm.w_goal * e / np.linalg.norm(e))
    assert np.allclose(adj["g_v0"][:, 0], expect, rtol=1e-10, atol=1e-12)
    assert adj["cost"][0] == pytest.approx(prm.w_path * N * dt * np.linalg.norm(v0)
                                           + prm.w_goal * np.linalg.norm(e), rel=1e-12)


def test_cost_matches_rollout():
    w = synth.adjoint_workload(n_obs=2000, n_agents=5, n_steps=150)
    adj = oracle.adjoint(w["obstacles"], w["r_O"], w["agents"], w["params"])
    ro = oracle.rollout(w["obstacles"], w["r_O"], w["agents"], w["params"], want_traj=False)
    assert np.allclose(adj["cost"], oracle.costs(ro, w["params"]), rtol=1e-13, atol=0)
    assert np.all(np.isfinite(adj["g_c"])) and np.all(np.isfinite(adj["g_v0"]))
