"""GPU score_and_select vs the oracle (Sec. IV-A cost and selection):
costs, argmin with ties to the lowest index, alpha-hysteresis, NaN costs and
the copy of the winner's trajectory; and the end-to-end selection rule on a
full rollout (GPU i* equals the oracle's unless their oracle costs differ by
less than 1e-6)."""

import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from synth.workloads import PhysicsParams

from _helpers import to_dev_agents

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def gm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2606_12579_b300 as gm
    gm.context()
    return gm


def _ro(path_len, p_final, clear_pen, traj=None):
    import torch
    t = lambda a: torch.tensor(np.asarray(a, np.float32)).cuda()  # noqa: E731
    return {"path_len": t(path_len), "p_final": t(p_final).contiguous(), "clear_pen": t(clear_pen),
            "traj": t(traj) if traj is not None else None}


def test_golden_costs_hysteresis(gm):
    g = json.load(open(os.path.join(GOLD, "cost_tiny.json")))
    prm = PhysicsParams(goal=tuple(g["goal"]), n_steps=1, w_path=g["w_path"], w_goal=g["w_goal"],
                        w_clear=g["w_clear"])
    traj = np.arange(3 * 2 * 3, dtype=np.float32).reshape(3, 2, 3)
    ro = _ro(g["path_len"], g["p_final"], g["clear_pen"], traj)
    out = gm.score_and_select(ro, prm)
    gm.sync()
    assert np.allclose(out["costs"].cpu().numpy(), g["costs"], rtol=1e-6)
    assert int(out["best"].item()) == g["best"]
    assert np.array_equal(out["best_traj"].cpu().numpy(), traj[g["best"]])
    for h in g["hysteresis"]:
        o = gm.score_and_select(ro, prm, prev_best_cost=h["prev_best_cost"], alpha=h["alpha"])
        gm.sync()
        assert int(o["best"].item()) == h["best"]


@pytest.mark.parametrize("n", [1, 31, 32, 33, 1000, 1024, 1025, 5000])
def test_random_costs_ties_and_nan(gm, n):
    g = np.random.Generator(np.random.PCG64(n))
    L = g.uniform(0.5, 2.0, n).astype(np.float32)
    pf = g.uniform(-1, 1, (3, n)).astype(np.float32)
    pen = g.uniform(0, 1, n).astype(np.float32)
    prm = PhysicsParams(goal=(0.1, 0.2, 0.3), n_steps=1, w_clear=0.5)
    if n > 3:
        # exact tie between two agents at the minimum, and a NaN agent
        j = int(g.integers(0, n))
        k = (j + n // 2) % n
        L[:] = 10.0
        L[j] = L[k] = 0.1
        pf[:, j] = np.asarray(prm.goal, np.float32)
        pen[j] = 0.0
        pf[:, k], pen[k] = pf[:, j], pen[j]
        L[(j + 1) % n if (j + 1) % n != k else (j + 2) % n] = np.nan
    ro = _ro(L, pf, pen)
    out = gm.score_and_select(ro, prm, best_traj=False)
    gm.sync()
    c64 = oracle.costs({"path_len": L.astype(np.float64), "p_final": pf.astype(np.float64),
                        "clear_pen": pen.astype(np.float64)}, prm)
    cg = out["costs"].cpu().numpy()
    fin = np.isfinite(c64)
    assert np.allclose(cg[fin], c64[fin], rtol=2e-6)
    best = int(out["best"].item())
    c_nan_last = np.where(np.isnan(c64), np.inf, c64)
    ob = oracle.select(c_nan_last)
    assert best == ob or abs(c64[best] - c64[ob]) < 1e-6 * max(1.0, abs(c64[ob]))
    if n > 3:
        assert best == min(j, k)


def test_selection_on_full_rollout(gm):
    import torch
    w = synth.sphere_workload(n_agents=64, n_steps=200)
    ref_f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    obs = np.stack([ref_f["x"], ref_f["y"], ref_f["z"]])
    ref = oracle.rollout(obs, ref_f["r_O"], w["agents"], w["params"], want_traj=False)
    c_ref = oracle.costs(ref, w["params"])
    gobs = gm.filter_cloud(torch.from_numpy(w["xyz"]).cuda(), w["T"], w["workspace"], cap=4096)
    ro = gm.rollout_agents(gobs, to_dev_agents(w["agents"]), w["params"])
    sel = gm.score_and_select(ro, w["params"])
    gm.sync()
    gi = int(sel["best"].item())
    oi = oracle.select(c_ref)
    assert gi == oi or abs(c_ref[gi] - c_ref[oi]) < 1e-6
    assert np.allclose(sel["costs"].cpu().numpy(), c_ref, rtol=1e-4, atol=1e-4)
    assert torch.equal(sel["best_traj"], ro["traj"][gi])
