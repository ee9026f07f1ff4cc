"""GPU four-term cost (Eq. cost_function: goal, obstacle, path, smoothness
terms of Sec. IV-A "Cost Functions") and the selection with hysteresis
("Selection Mechanism") vs the oracle.

The rollout accumulates the sums of the terms over the candidate trajectory
(the N_k evaluated states p_0 .. p_{N_k-1}); score_and_select4 combines them.
Tolerances follow from the rollout's own parity: each goal / obstacle term
is a 1/r_c-Lipschitz function of a position or clearance, so it may differ
from the oracle's by the measured trajectory error / r_c (plus FP32 sums);
the path length like the rollout's path length (1e-3 m); the jerk sum is
accumulated from FP32 force differences (relative error ~1e-6 |F| / |dF|
per step), checked to 1e-2 relative.  Selection: the GPU's i* equals the
oracle's unless their oracle costs differ by less than 1e-6, and the
device-resident C_best follows the alpha rule across re-planning ticks.
"""

import dataclasses
import math

import numpy as np
import pytest

import oracle
import synth

from _helpers import to_dev_agents

pytestmark = pytest.mark.gpu
POS_TOL = 1e-3


@pytest.fixture(scope="module")
def gm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2606_12579_b300 as gm
    gm.context()
    return gm


def _filtered(w):
    ref = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    return np.stack([ref["x"], ref["y"], ref["z"]]), ref["r_O"]


def _gpu_obstacles(gm, obs, r_O, cap=None):
    import torch
    return gm.Obstacles.from_points(torch.from_numpy(np.ascontiguousarray(obs, np.float32)), r_O,
                                    cap=cap)


def _terms_vs_oracle(gm, gpu, ref, prm):
    """Compare the GPU's per-term costs (from cost_terms and from the
    scorer with one-hot weights) with the oracle's four_term_costs."""
    traj = gpu["traj"].cpu().numpy().astype(np.float64)
    terr = np.abs(traj - ref["traj"]).max()
    assert terr <= POS_TOL
    rc = prm.cost_radius
    want = oracle.four_term_costs(ref["traj"], ref["m_trace"], prm.goal, prm.dt, rc, prm.a_max,
                                  prm.w4)
    ct = gpu["cost_terms"].cpu().numpy().astype(np.float64)
    nk = prm.n_steps
    tol_pos = terr / rc + 1e-5
    assert np.abs(ct[0] / nk - want["goal"]).max() <= tol_pos
    assert np.abs(ct[1] / nk - want["obs"]).max() <= tol_pos
    assert np.abs(ct[2] - want["L"]).max() <= POS_TOL
    assert np.abs(ct[4] - want["d1"]).max() <= 1e-6
    assert np.allclose(ct[3], want["J"], rtol=1e-2, atol=1e-12)
    # the scorer combines the GPU's own sums exactly as Eq. (cost_function)
    # says (FP32 rounding only), one term at a time and weighted
    L, d1 = ct[2], ct[4]
    gpu_terms = {"goal": ct[0] / nk, "obs": ct[1] / nk,
                 "path": np.where(L >= d1, np.where(L > 0, 1 - d1 / np.maximum(L, 1e-300), 0.0),
                                  1 - L / np.maximum(d1, 1e-300)),
                 "smooth": np.minimum(1.0, ct[3] / (nk * prm.dt ** 4 * prm.a_max ** 2))}
    for j, name in enumerate(("goal", "obs", "path", "smooth")):
        w1 = tuple(1.0 if i == j else 0.0 for i in range(4))
        sel = gm.score_and_select4(gpu, dataclasses.replace(prm, w4=w1))
        gm.sync()
        c = sel["costs"].cpu().numpy().astype(np.float64)
        assert np.allclose(c, gpu_terms[name], rtol=1e-5, atol=1e-6), name
    # and the terms themselves agree with the oracle's (path via L above)
    assert np.allclose(gpu_terms["smooth"], want["smooth"], rtol=1e-2, atol=1e-9)
    sel = gm.score_and_select4(gpu, prm)
    gm.sync()
    C = sel["costs"].cpu().numpy().astype(np.float64)
    Cg = sum(wj * gpu_terms[k] for wj, k in zip(prm.w4, ("goal", "obs", "path", "smooth")))
    assert np.allclose(C, Cg, rtol=1e-5, atol=1e-6)
    gi, oi = int(sel["best"].item()), oracle.select(want["C"])
    assert gi == oi or abs(want["C"][gi] - want["C"][oi]) < 1e-6
    return want


def _sphere(n_agents=8, n_steps=200):
    w = synth.sphere_workload(n_agents=n_agents, n_steps=n_steps)
    w["params"] = dataclasses.replace(w["params"], cost_radius=0.1, a_max=50.0,
                                      w4=(1.0, 2.0, 1.0, 0.5))
    return w


@pytest.mark.parametrize("shape", [None, (2, 4, 256, 0), (3, 3, 128, 1)],
                         ids=["auto", "cluster", "grid"])
def test_four_term_costs_sphere(gm, shape):
    w = _sphere()
    obs, r_O = _filtered(w)
    prm = w["params"]
    ref = oracle.rollout(obs, r_O, w["agents"], prm, want_trace=True)
    out = gm.alloc_rollout_out(8, prm.n_steps, want_cost4=True)
    gm.rollout_agents(_gpu_obstacles(gm, obs, r_O), to_dev_agents(w["agents"]), prm, out=out,
                      tuning=shape)
    gm.sync()
    want = _terms_vs_oracle(gm, out, ref, prm)
    assert np.all(want["obs"] > 0) and np.all(want["smooth"] > 0)   # every term active


def test_four_term_costs_tabletop_sample(gm):
    """256 agents x 500 steps on the tabletop frame; 12 agents checked."""
    import torch
    w = synth.tabletop_workload()
    prm = dataclasses.replace(w["params"], cost_radius=0.05, a_max=50.0)
    xyz = torch.from_numpy(w["xyz"]).cuda()
    gobs = gm.filter_cloud(xyz, w["T"], w["workspace"], cap=131072)
    out = gm.alloc_rollout_out(256, prm.n_steps, want_cost4=True)
    gm.rollout_agents(gobs, to_dev_agents(w["agents"]), prm, out=out)
    gm.sync()
    idx = np.arange(0, 256, 22)
    obs, r_O = _filtered(w)
    sub = {k: np.ascontiguousarray(v[..., idx]) for k, v in w["agents"].items()}
    ref = oracle.rollout(obs, r_O, sub, prm, want_trace=True)
    want = oracle.four_term_costs(ref["traj"], ref["m_trace"], prm.goal, prm.dt, 0.05, 50.0)
    ct = out["cost_terms"].cpu().numpy()[:, idx].astype(np.float64)
    terr = np.abs(out["traj"].cpu().numpy()[idx] - ref["traj"]).max()
    assert terr <= POS_TOL
    assert np.abs(ct[0] / prm.n_steps - want["goal"]).max() <= terr / 0.05 + 1e-5
    assert np.abs(ct[1] / prm.n_steps - want["obs"]).max() <= terr / 0.05 + 1e-5
    assert np.abs(ct[2] - want["L"]).max() <= POS_TOL
    assert np.allclose(ct[3], want["J"], rtol=1e-2, atol=1e-12)


def test_four_term_costs_ensemble(gm):
    w = _sphere(n_agents=10)
    w["agents"] = synth.ensemble_agents(w["agents"], 4)
    obs, r_O = _filtered(w)
    prm = w["params"]
    ref = oracle.rollout(obs, r_O, w["agents"], prm, want_trace=True, n_apf=4)
    out = gm.alloc_rollout_out(10, prm.n_steps, want_cost4=True)
    gm.rollout_ensemble(_gpu_obstacles(gm, obs, r_O), to_dev_agents(w["agents"]), 4, prm, out=out)
    gm.sync()
    _terms_vs_oracle(gm, out, ref, prm)


def test_replanning_hysteresis_on_device(gm):
    """C_best stays on the device across ticks: tick 1 picks the argmin and
    stores its cost; tick 2 (same scene) finds no agent below alpha C_best
    and keeps the plan (i* = -1, C_best unchanged); tick 3, with the
    obstacles gone, finds cheaper agents and switches."""
    import torch
    w = _sphere()
    obs, r_O = _filtered(w)
    prm = w["params"]
    ag = to_dev_agents(w["agents"])
    o = _gpu_obstacles(gm, obs, r_O)
    far = _gpu_obstacles(gm, obs + 10.0, r_O)
    c_best = torch.full((1,), math.nan, dtype=torch.float32, device="cuda")
    alpha = 0.98
    picks = []
    for scene in (o, o, far):
        out = gm.alloc_rollout_out(8, prm.n_steps, want_cost4=True)
        gm.rollout_agents(scene, ag, prm, out=out)
        before = float(c_best.item())
        sel = gm.score_and_select4(out, prm, c_best=c_best, alpha=alpha)
        gm.sync()
        C = sel["costs"].cpu().numpy().astype(np.float64)
        b = int(sel["best"].item())
        want = oracle.select(C, before, alpha)
        assert b == want
        if b >= 0:
            assert float(c_best.item()) == np.float32(C[b])
            assert torch.equal(sel["best_traj"], out["traj"][b])
        else:
            assert float(c_best.item()) == before
        picks.append(b)
    assert picks[0] >= 0 and picks[1] == -1 and picks[2] >= 0


def test_cost4_invalid_arguments(gm):
    w = _sphere(n_agents=2, n_steps=10)
    obs, r_O = _filtered(w)
    o = _gpu_obstacles(gm, obs, r_O)
    ag = to_dev_agents(w["agents"])
    out = gm.alloc_rollout_out(2, 10, want_cost4=True)
    with pytest.raises(gm.GmappError) as e:
        gm.rollout_agents(o, ag, dataclasses.replace(w["params"], cost_radius=0.0), out=out)
    assert e.value.status == 1
    plain = gm.rollout_agents(o, ag, w["params"])
    with pytest.raises(gm.GmappError) as e:
        gm.score_and_select4(plain, w["params"])
    assert e.value.status == 1
    gm.rollout_agents(o, ag, w["params"], out=out)
    with pytest.raises(gm.GmappError) as e:
        gm.score_and_select4(out, dataclasses.replace(w["params"], a_max=0.0))
    assert e.value.status == 1
