"""Pins for the oracle's circular-field force (Eq. mfi, Alg. 1).

Hand-derived single-obstacle values (golden fixture), the orthogonality of
the CF force to the velocity (it only turns the velocity: Sec. III, the swirl
that leaves the energy unchanged), obstacle-permutation invariance, the
linearity in the gain, and the zero-velocity guard.
"""

import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _agents(c, k_r, r_d, r_a, n=1):
    return {"c": np.asarray(c, np.float64).reshape(3, n), "k_r": np.full(n, k_r),
            "r_d": np.full(n, r_d), "r_a": np.full(n, r_a)}


@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLD, "force_single_obstacle.json")))["cases"],
                         ids=lambda c: c["name"])
def test_golden_single_obstacle(case):
    obs = np.asarray(case["obstacles"], np.float64).T
    out = oracle.cf_eval(obs, case["r_O"], np.reshape(case["p"], (3, 1)),
                         np.reshape(case["v"], (3, 1)),
                         _agents(case["c"], case["k_r"], case["r_d"], case["r_a"]),
                         case["rho"], case["eps"])
    assert out["W"][0] == pytest.approx(case["W"], rel=1e-12, abs=1e-12)
    assert out["m"][0] == pytest.approx(case["m"], rel=1e-12, abs=1e-15)
    assert np.allclose(out["f_r"][:, 0], case["f_r"], rtol=1e-12, atol=1e-12)


def _scene(seed=7, n_obs=500, n_ag=16):
    g = np.random.Generator(np.random.PCG64(seed))
    obs = g.uniform(-0.1, 0.1, (3, n_obs))
    p = g.uniform(-0.05, 0.05, (3, n_ag))
    v = g.normal(0, 1, (3, n_ag))
    c = g.normal(0, 1, (3, n_ag))
    c /= np.linalg.norm(c, axis=0)
    ag = {"c": c, "k_r": g.uniform(0.5, 2, n_ag), "r_d": np.full(n_ag, 0.05),
          "r_a": np.zeros(n_ag)}
    return obs, p, v, ag


def test_orthogonal_to_velocity():
    obs, p, v, ag = _scene()
    f = oracle.cf_eval(obs, 0.005, p, v, ag, 0.01, 1e-3)["f_r"]
    dots = np.abs((f * v).sum(axis=0))
    scale = np.linalg.norm(f, axis=0) * np.linalg.norm(v, axis=0)
    assert np.all(dots <= 1e-13 * scale + 1e-300)
    assert np.all(np.linalg.norm(f, axis=0) > 0)


def test_obstacle_permutation_invariance():
    obs, p, v, ag = _scene()
    a = oracle.cf_eval(obs, 0.005, p, v, ag, 0.01, 1e-3)
    perm = np.random.Generator(np.random.PCG64(1)).permutation(obs.shape[1])
    b = oracle.cf_eval(obs[:, perm], 0.005, p, v, ag, 0.01, 1e-3)
    assert np.allclose(a["W"], b["W"], rtol=1e-12)
    assert np.array_equal(a["m"], b["m"])


def test_linear_in_gain_and_zero_velocity():
    obs, p, v, ag = _scene()
    a = oracle.cf_eval(obs, 0.005, p, v, ag, 0.01, 1e-3)
    ag2 = dict(ag, k_r=2 * ag["k_r"])
    b = oracle.cf_eval(obs, 0.005, p, v, ag2, 0.01, 1e-3)
    assert np.allclose(b["f_r"], 2 * a["f_r"], rtol=1e-13, atol=0)
    z = oracle.cf_eval(obs, 0.005, p, np.zeros_like(v), ag, 0.01, 1e-3)
    assert np.all(z["f_r"] == 0.0)
    assert np.array_equal(z["W"], a["W"])


def test_sum_equals_brute_force_pairs():
    """W for a real obstacle set equals the pairwise sum taken one obstacle at
    a time (the force is additive over S_W, Alg. 1)."""
    w = synth.sphere_workload()
    f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    obs = np.stack([f["x"], f["y"], f["z"]]).astype(np.float64)
    p = np.array([[0.36], [0.01], [0.41]])
    v = np.array([[1.0], [0.0], [0.0]])
    ag = {k: np.asarray(w["agents"][k][:1], np.float64) for k in ("k_r", "r_d", "r_a")}
    ag["c"] = np.asarray(w["agents"]["c"][:, :1], np.float64)
    full = oracle.cf_eval(obs, f["r_O"], p, v, ag, 0.05, 1e-3)
    parts = [oracle.cf_eval(obs[:, j:j + 1], f["r_O"], p, v, ag, 0.05, 1e-3)["W"][0]
             for j in range(obs.shape[1])]
    assert full["W"][0] == pytest.approx(sum(parts), rel=1e-12)
    assert full["W"][0] > 0
