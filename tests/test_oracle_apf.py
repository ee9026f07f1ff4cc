"""Pins for the oracle's APF heuristic (Eq. apf) and the heterogeneous
ensemble rollout (the last n_apf agents on APF).

The APF force is the negative gradient of Khatib's potential
U(r) = 1/2 k_f (1/r - 1/r_d)^2 in the centre distance r, so it is pinned by
a central finite difference of U written here independently; plus the strict
gate d_O < r_d on exactly representable distances, the inverse-cube scaling
without a gate, symmetry (two mirrored obstacles cancel), the Alg. 1 clamp
for a penetrating agent, energy conservation of an undamped head-on
encounter, and the ensemble's partition invariance.
"""

import numpy as np
import pytest

import oracle
import synth


def _ag(k_r, r_d, r_a=0.0, n=1):
    return {"k_r": np.full(n, k_r, np.float64), "r_d": np.full(n, r_d, np.float64),
            "r_a": np.full(n, r_a, np.float64)}


def _f(obs, r_O, p, ag, rho=1.0, eps=1e-3):
    return oracle.apf_eval(np.asarray(obs, np.float64).reshape(3, -1), r_O,
                           np.asarray(p, np.float64).reshape(3, -1), ag, rho, eps)


@pytest.mark.parametrize("r", [0.03, 0.05, 0.07, 0.11])
def test_force_is_minus_gradient_of_khatib_potential(r):
    k_f, r_d, r_O = 2.5, 0.12, 0.01   # the gate d_O = r - r_O < r_d holds for all r
    u = np.array([0.36, -0.48, 0.8])  # unit direction
    U = lambda x: 0.5 * k_f * (1.0 / x - 1.0 / r_d) ** 2  # noqa: E731
    h = 1e-7
    dU = (U(r + h) - U(r - h)) / (2 * h)
    out = _f([0.0, 0.0, 0.0], r_O, r * u, _ag(1.0, r_d), rho=k_f)
    assert np.allclose(out["f_r"][:, 0], -dU * u, rtol=1e-7, atol=1e-9)
    assert out["m"][0] == pytest.approx(r - r_O, abs=1e-15)


def test_gate_is_strict():
    # R = 0.25, r_d = 0.5: exactly at d_O = r_d (r = 0.75) nothing, just inside something
    at = _f([0, 0, 0], 0.25, [0.75, 0, 0], _ag(1.0, 0.5))
    inside = _f([0, 0, 0], 0.25, [0.7421875, 0, 0], _ag(1.0, 0.5))
    assert np.all(at["f_r"] == 0.0)
    assert inside["f_r"][0, 0] != 0.0
    # between r = r_d and r = r_d + R the printed coefficient (1/r - 1/r_d) is
    # negative: the term pulls toward the obstacle (taken as printed)
    assert inside["f_r"][0, 0] < 0.0


def test_inverse_cube_without_gate():
    a = _f([0, 0, 0], 0.0, [0.05, 0, 0], _ag(1.0, np.inf))["f_r"][0, 0]
    b = _f([0, 0, 0], 0.0, [0.10, 0, 0], _ag(1.0, np.inf))["f_r"][0, 0]
    assert a > 0 and b > 0
    assert a / b == pytest.approx(8.0, rel=1e-13)


def test_mirrored_obstacles_cancel_and_permutation():
    g = np.random.Generator(np.random.PCG64(3))
    p = np.array([0.1, -0.2, 0.3])
    off = g.normal(0, 0.02, (3, 40))
    obs = np.concatenate([p[:, None] + off, p[:, None] - off], axis=1)
    out = _f(obs, 0.005, p, _ag(1.0, 0.06))
    single = _f(obs[:, :40], 0.005, p, _ag(1.0, 0.06))
    assert np.abs(out["f_r"]).max() <= 1e-12 * np.abs(single["f_r"]).max()
    # the term-magnitude sum does not cancel: it doubles, and for one
    # obstacle it equals the force magnitude
    assert out["f_abs"][0] == pytest.approx(2.0 * single["f_abs"][0], rel=1e-13)
    one = _f(obs[:, :1], 0.005, p, _ag(1.0, np.inf), rho=3.0)
    assert one["f_abs"][0] == pytest.approx(np.linalg.norm(one["f_r"][:, 0]), rel=1e-14)
    assert single["f_abs"][0] >= np.linalg.norm(single["f_r"][:, 0])
    perm = g.permutation(40)
    a = _f(obs[:, :40], 0.005, p, _ag(1.0, 0.06))["f_r"]
    b = _f(obs[:, :40][:, perm], 0.005, p, _ag(1.0, 0.06))["f_r"]
    assert np.allclose(a, b, rtol=1e-13, atol=0)


def test_penetration_clamped_by_alg1():
    # R = 0.01, eps = 1e-3: any centre distance below R + eps gives the force
    # magnitude at R + eps, along the same direction
    ref = _f([0, 0, 0], 0.01, [0.011, 0, 0], _ag(1.0, 0.05))["f_r"][0, 0]
    for r in (0.0105, 0.005, 1e-6):
        got = _f([0, 0, 0], 0.01, [r, 0, 0], _ag(1.0, 0.05))["f_r"][0, 0]
        assert got == pytest.approx(ref, rel=1e-12)
    assert np.all(_f([0, 0, 0], 0.01, [0, 0, 0], _ag(1.0, 0.05))["f_r"] == 0.0)


def test_undamped_head_on_encounter_conserves_energy():
    """k_a = 0, D = 0: the update v += 1/2 dt F, p += dt v is symplectic
    Euler for p'' = F / 2, so E = |v|^2 / 2 + U / 2 stays constant up to
    O(dt), and the agent turns back where U / 2 has used up its kinetic
    energy."""
    k_f, r_d = 2e-6, 0.1
    obs = np.zeros((3, 1))
    prm = synth.PhysicsParams(goal=(0.0, 0.0, 0.0), dt=1e-4, n_steps=6000, damping=0.0,
                              rho=1.0, w_clear=0.0)
    ag = {"p0": np.array([[0.12], [0.0], [0.0]]), "v0": np.array([[-0.5], [0.0], [0.0]]),
          "c": np.array([[0.0], [0.0], [1.0]]), "k_r": np.array([k_f]), "k_a": np.array([0.0]),
          "r_d": np.array([r_d]), "r_a": np.array([0.0])}
    ro = oracle.rollout(obs, 0.0, ag, prm, n_apf=1)
    x = ro["traj"][0, :, 0]
    U = np.where(x < r_d, 0.5 * k_f * (1.0 / np.maximum(x, 1e-3) - 1.0 / r_d) ** 2, 0.0)
    v = np.diff(x) / prm.dt                    # v_k between p_k and p_k+1
    E = 0.5 * v ** 2 + 0.5 * U[1:]
    # turning point: U(r*) / 2 = v0^2 / 2 with U = k_f / 2 (1/r - 1/r_d)^2, so
    # 1/r* = 1/r_d + v0 sqrt(2 / k_f) = 10 + 500
    assert x.min() == pytest.approx(1.0 / 510.0, rel=0.02)
    assert x[-1] > x.min() + 0.01 and v[-1] > 0
    # O(dt) excursion inside the steep field, and the same energy once the
    # agent has left it again (symplectic: no secular drift)
    assert np.abs(E - E[0]).max() <= 1.5e-2 * E[0]
    assert abs(E[-1] - E[0]) <= 1e-9 * E[0]


def test_ensemble_partition_invariance():
    w = synth.sphere_workload(n_agents=10, n_steps=150)
    f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    obs = np.stack([f["x"], f["y"], f["z"]])
    ag = dict(w["agents"])
    ag["k_r"] = ag["k_r"].copy()
    ag["k_r"][6:] *= 1e-3    # APF gains, scaled to the inverse-cube field
    mixed = oracle.rollout(obs, f["r_O"], ag, w["params"], n_apf=4)
    cf = oracle.rollout(obs, f["r_O"], {k: v[..., :6] for k, v in ag.items()}, w["params"])
    apf = oracle.rollout(obs, f["r_O"], {k: v[..., 6:] for k, v in ag.items()}, w["params"],
                         n_apf=4)
    assert np.array_equal(mixed["traj"][:6], cf["traj"])
    assert np.array_equal(mixed["traj"][6:], apf["traj"])
    none = oracle.rollout(obs, f["r_O"], ag, w["params"], n_apf=0)
    assert not np.array_equal(none["traj"][6:], mixed["traj"][6:])
    # with every obstacle out of reach both heuristics reduce to the attractor
    far = obs + 10.0
    a = oracle.rollout(far, f["r_O"], ag, w["params"], n_apf=10)
    b = oracle.rollout(far, f["r_O"], ag, w["params"], n_apf=0)
    assert np.array_equal(a["traj"], b["traj"])
