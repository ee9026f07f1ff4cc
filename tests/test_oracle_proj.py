"""Pins for the oracle's MFI with the per-obstacle projected current (Eq.
mfi with c_j = d' - n_j (n_j . d'), the equation after it; static obstacles,
d' = -v), written out in the oracle with the two cross products.

Closed forms: for v = v0 x_hat and the normal n = (cos t, sin t, 0) the term
is (0, v0^2 sin t cos t, 0) / s, so it vanishes head-on (t = 0: the
projected current is zero) and side-on (t = 90 deg); every term is
orthogonal to v; the term is even in the normal, so two obstacles mirrored
through the agent add instead of cancelling; the gate and clamp of Alg. 1;
the reduced form used by the CUDA kernel,
    f = (|v|^2 sum_j a_j d_j - v sum_j a_j (d_j . v)) / |v|,
    a_j = w_j (d_j . v) / |d_j|^2,  w_j = [s_j <= r_d] / s_j,
equals the cross-product form; a pure projected-current rollout keeps the
discrete speed identity |v_k|^2 - |v_{k-1}|^2 = |v_k - v_{k-1}|^2; the
ensemble keeps agents independent.
"""

import dataclasses
import math

import numpy as np
import pytest

import oracle
import synth


def _ag(k_r=1.0, r_d=0.05, r_a=0.0, n=1):
    return {"k_r": np.full(n, k_r, np.float64), "r_d": np.full(n, r_d, np.float64),
            "r_a": np.full(n, r_a, np.float64)}


def _f(obs, r_O, p, v, ag, rho=1.0, eps=1e-3):
    return oracle.proj_eval(np.asarray(obs, np.float64).reshape(3, -1), r_O,
                            np.asarray(p, np.float64).reshape(3, -1),
                            np.asarray(v, np.float64).reshape(3, -1), ag, rho, eps)


def test_single_obstacle_closed_form():
    v0, t, dn, R = 2.0, math.radians(30.0), 0.03, 0.005
    p = np.array([0.4, -0.1, 0.2])
    obs = p - dn * np.array([math.cos(t), math.sin(t), 0.0])
    out = _f(obs, R, p, [v0, 0.0, 0.0], _ag())
    s = dn - R
    want = np.array([0.0, v0 ** 2 * math.sin(t) * math.cos(t) / s, 0.0])
    assert np.allclose(out["f_r"][:, 0], want, rtol=1e-13, atol=1e-12)
    assert want[1] == pytest.approx(69.28203230275509, rel=1e-13)
    assert out["m"][0] == pytest.approx(s, abs=1e-15)


@pytest.mark.parametrize("t_deg", [0.0, 90.0, 180.0])
def test_head_on_and_side_on_vanish(t_deg):
    t = math.radians(t_deg)
    p = np.zeros(3)
    obs = p - 0.02 * np.array([math.cos(t), math.sin(t), 0.0])
    f = _f(obs, 0.0, p, [1.5, 0.0, 0.0], _ag())["f_r"][:, 0]
    assert np.abs(f).max() <= 1e-12


def test_orthogonal_to_velocity_and_even_in_the_normal():
    g = np.random.Generator(np.random.PCG64(11))
    p = np.array([0.3, 0.0, 0.4])
    v = g.normal(size=3)
    off = g.normal(0.0, 0.02, (3, 50))
    one = _f(p[:, None] + off, 0.004, p, v, _ag(r_d=0.2))["f_r"][:, 0]
    assert abs(one @ v) <= 1e-12 * np.linalg.norm(one) * np.linalg.norm(v)
    both = _f(np.concatenate([p[:, None] + off, p[:, None] - off], axis=1), 0.004, p, v,
              _ag(r_d=0.2))["f_r"][:, 0]
    assert np.allclose(both, 2.0 * one, rtol=1e-12, atol=0)


def test_gate_clamp_and_zero_velocity():
    p = np.zeros(3)
    v = [1.0, 0.0, 0.0]
    t = math.radians(45.0)
    u = np.array([math.cos(t), math.sin(t), 0.0])
    # R = 0.25, r_d = 0.5: s = 0.5 exactly at |d| = 0.75 still counts (<=), beyond not
    at = _f(p - 0.75 * u, 0.25, p, v, _ag(r_d=0.5))["f_r"][:, 0]
    out = _f(p - 0.7500001 * u, 0.25, p, v, _ag(r_d=0.5))["f_r"][:, 0]
    assert at[1] == pytest.approx(0.5 / 0.5, rel=1e-12)   # v0^2 sin t cos t / s
    assert np.all(out == 0.0)
    # penetration: s clamped at eps, direction from the normal
    pen = _f(p - 0.1 * u, 0.25, p, v, _ag(r_d=0.5), eps=1e-3)["f_r"][:, 0]
    assert pen[1] == pytest.approx(0.5 / 1e-3, rel=1e-12)
    assert np.all(_f(p - 0.3 * u, 0.25, p, [0.0, 0.0, 0.0], _ag(r_d=0.5))["f_r"] == 0.0)
    assert np.all(_f(p, 0.25, p, v, _ag(r_d=0.5))["f_r"] == 0.0)     # d = 0: no normal


def test_reduced_form_matches_cross_products():
    g = np.random.Generator(np.random.PCG64(5))
    p = np.array([0.5, 0.1, 0.3])
    obs = p[:, None] + g.normal(0.0, 0.03, (3, 300))
    R, eps, r_d = 0.005, 1e-3, 0.05
    for _ in range(5):
        v = g.normal(size=3)
        f = _f(obs, R, p, v, _ag(r_d=r_d), eps=eps)["f_r"][:, 0]
        d = p[:, None] - obs
        dn = np.linalg.norm(d, axis=0)
        s = np.maximum(dn - R, eps)
        w = np.where(s <= r_d, 1.0 / s, 0.0)
        t = v @ d
        a = w * t / dn ** 2
        red = (v @ v * (d @ a) - v * (a @ t)) / np.linalg.norm(v)
        assert np.allclose(f, red, rtol=1e-11, atol=1e-12)


def test_pure_projected_rollout_keeps_the_speed_identity():
    w = synth.sphere_workload(n_agents=4, n_steps=150)
    f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    obs = np.stack([f["x"], f["y"], f["z"]])
    ag = dict(w["agents"])
    ag["k_a"] = np.zeros(4, np.float32)
    prm = dataclasses.replace(w["params"], damping=0.0)
    ro = oracle.rollout(obs, f["r_O"], ag, prm, n_proj=4, want_trace=True)
    vk = np.diff(ro["traj"], axis=1) / prm.dt            # v_0 .. v_{N_k - 1}
    dv = np.diff(vk, axis=1)
    lhs = (vk[:, 1:] ** 2).sum(axis=2) - (vk[:, :-1] ** 2).sum(axis=2)
    rhs = (dv ** 2).sum(axis=2)
    assert np.allclose(lhs, rhs, rtol=1e-6, atol=1e-9)
    assert ro["w_trace"].max() > 0                        # the field was active


def test_ensemble_with_projected_agents_is_partitioned():
    w = synth.sphere_workload(n_agents=9, n_steps=120)
    f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    obs = np.stack([f["x"], f["y"], f["z"]])
    ag = synth.ensemble_agents(w["agents"], 3)
    mixed = oracle.rollout(obs, f["r_O"], ag, w["params"], n_apf=3, n_proj=3)
    sub = lambda lo, hi: {k: v[..., lo:hi] for k, v in ag.items()}   # noqa: E731
    assert np.array_equal(mixed["traj"][:3], oracle.rollout(obs, f["r_O"], sub(0, 3),
                                                             w["params"])["traj"])
    assert np.array_equal(mixed["traj"][3:6], oracle.rollout(obs, f["r_O"], sub(3, 6),
                                                              w["params"], n_proj=3)["traj"])
    assert np.array_equal(mixed["traj"][6:], oracle.rollout(obs, f["r_O"], sub(6, 9),
                                                             w["params"], n_apf=3)["traj"])
