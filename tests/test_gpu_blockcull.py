"""rollout_agents_blockcull: spatial culling over the key-sorted obstacle set
(Alg. 1's gate zeroes every pair beyond r_d + R).  A warp visits only the
blocks of 128 obstacles whose bounding box meets an agent's gate, and
evaluates them exactly as rollout_agents does, in the same order.  So W, the
trajectories and the path lengths must equal rollout_agents' at the same
launch shape bit for bit, whatever the obstacle order.  The clearance must be
exact wherever the nearest obstacle lies within the reach (at least r_d
elsewhere), and the trajectories must lie within 1e-3 m of the FP64 oracle."""

import numpy as np
import pytest

import oracle
import synth

from _helpers import to_dev_agents

pytestmark = pytest.mark.gpu
POS_TOL = 1e-3
TABLE = (5, 6, 256, 1)
TABLE_CLUSTER = (5, 6, 384, 0)


@pytest.fixture(scope="module")
def gm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2606_12579_b300 as gm
    gm.context()
    return gm


def _bits(t):
    return t.cpu().numpy().view(np.uint32)


def _pair(gm, obs, dev, prm, tuning, clear):
    import torch
    outs = []
    for fn in (gm.rollout_agents, gm.rollout_agents_blockcull):
        o = gm.alloc_rollout_out(int(dev["k_r"].numel()), int(prm.n_steps), want_traj=True,
                                 want_trace=True, want_clear=clear)
        o["f_trace"] = None
        if not clear:
            o["m_trace"] = None
        o["heur_pairs"] = torch.zeros(1, dtype=torch.int64, device="cuda")
        fn(obs, dev, prm, out=o, tuning=tuning)
        outs.append(o)
    gm.sync()
    return outs


@pytest.mark.parametrize("tuning", [TABLE, TABLE_CLUSTER])
@pytest.mark.parametrize("clear", [False, True])
def test_tabletop_equals_all_pairs_bit_for_bit(gm, tuning, clear):
    import torch
    w = synth.tabletop_workload(n_agents=60, n_steps=300)
    obs = gm.filter_cloud(torch.from_numpy(w["xyz"]).cuda(), w["T"], w["workspace"], cap=80000)
    a, b = _pair(gm, obs, to_dev_agents(w["agents"]), w["params"], tuning, clear)
    for key in ("w_trace", "traj", "path_len", "p_final", "v_final"):
        assert np.array_equal(_bits(a[key]), _bits(b[key])), key
    assert np.count_nonzero(a["w_trace"].cpu().numpy()) > 1000
    total = 60 * obs.count() * 300
    hb = int(b["heur_pairs"].item())
    assert 0 < hb < 0.5 * total       # culled: most blocks are never visited


def test_any_obstacle_order_gives_the_same_results(gm):
    """Obstacles in a random order (blocks no longer compact): still equal
    to rollout_agents on the same order."""
    import torch
    w = synth.sphere_workload(n_agents=24, n_steps=200)
    f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    o = np.stack([f["x"], f["y"], f["z"]])
    perm = np.random.default_rng(3).permutation(o.shape[1])
    obs = gm.Obstacles.from_points(torch.from_numpy(np.ascontiguousarray(o[:, perm])), f["r_O"])
    a, b = _pair(gm, obs, to_dev_agents(w["agents"]), w["params"], (2, 4, 256, 1), False)
    for key in ("w_trace", "traj"):
        assert np.array_equal(_bits(a[key]), _bits(b[key])), key


def test_ungated_agent_and_sphere_oracle(gm):
    """One agent without a gate (r_d = inf) makes its group evaluate every
    pair; the rest are culled.  Trajectories within 1e-3 m of the oracle, the
    clearance exact where the nearest obstacle is within reach."""
    import torch
    w = synth.sphere_workload(n_agents=16, n_steps=200)
    ag = dict(w["agents"])
    ag["r_d"] = ag["r_d"].copy()
    ag["r_d"][5] = np.inf
    obs = gm.filter_cloud(torch.from_numpy(w["xyz"]).cuda(), w["T"], w["workspace"], cap=8192)
    a, b = _pair(gm, obs, to_dev_agents(ag), w["params"], (2, 4, 256, 1), True)
    for key in ("w_trace", "traj"):
        assert np.array_equal(_bits(a[key]), _bits(b[key])), key
    f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    ref = oracle.rollout(np.stack([f["x"], f["y"], f["z"]]), f["r_O"], ag, w["params"])
    assert np.abs(b["traj"].cpu().numpy() - ref["traj"]).max() <= POS_TOL
    mc, rm = b["min_clear"].cpu().numpy(), ref["min_clear"]
    rd = ag["r_d"].astype(np.float64)
    near = rm < rd
    assert np.abs(mc[near] - rm[near]).max(initial=0) <= POS_TOL
    assert np.all(mc[~near] >= rd[~near] - POS_TOL)


def test_four_term_cost_sums_equal_all_pairs(gm):
    """The four-term cost sums (goal, obstacle, path, jerk, d1) depend on the
    positions, the forces and -- through the obstacle term max(r_c - m, 0)
    -- on the clearance only where it is below r_c <= r_d, where the culled
    clearance is exact.  So they, and the agent score_and_select4 picks,
    equal rollout_agents' bit for bit."""
    import dataclasses
    import torch
    w = synth.tabletop_workload(n_agents=60, n_steps=300)
    prm = dataclasses.replace(w["params"], cost_radius=0.05)
    assert prm.cost_radius <= float(np.min(w["agents"]["r_d"]))
    obs = gm.filter_cloud(torch.from_numpy(w["xyz"]).cuda(), w["T"], w["workspace"], cap=80000)
    dev = to_dev_agents(w["agents"])
    outs, sels = [], []
    for fn in (gm.rollout_agents, gm.rollout_agents_blockcull):
        o = gm.alloc_rollout_out(60, 300, want_traj=True, want_clear=True, want_cost4=True)
        fn(obs, dev, prm, out=o, tuning=TABLE)
        outs.append(o)
        sels.append(gm.score_and_select4(o, prm))
    gm.sync()
    assert np.array_equal(_bits(outs[0]["cost_terms"]), _bits(outs[1]["cost_terms"]))
    assert int(sels[0]["best"].item()) == int(sels[1]["best"].item())


@pytest.mark.parametrize("n_proj,n_apf", [(0, 60), (60, 0), (20, 20)])
@pytest.mark.parametrize("clear", [False, True])
def test_ensemble_equals_rollout_ensemble_bit_for_bit(gm, n_proj, n_apf, clear):
    """APF and projected-current groups (and MFI beside them) culled by the
    block boxes: forces and trajectories equal rollout_ensemble's."""
    import torch
    w = synth.tabletop_workload(n_agents=60, n_steps=200)
    ag = synth.ensemble_agents(w["agents"], n_apf)
    obs = gm.filter_cloud(torch.from_numpy(w["xyz"]).cuda(), w["T"], w["workspace"], cap=80000)
    dev = to_dev_agents(ag)
    outs = []
    for cull in (False, True):
        o = gm.alloc_rollout_out(60, 200, want_traj=True, want_trace=True, want_clear=clear)
        if not clear:
            o["m_trace"] = None
        o["heur_pairs"] = torch.zeros(1, dtype=torch.int64, device="cuda")
        gm.rollout_ensemble(obs, dev, n_apf, w["params"], out=o, tuning=TABLE, n_proj=n_proj,
                            cull=cull)
        outs.append(o)
    gm.sync()
    a, b = outs
    for key in ("w_trace", "f_trace", "traj", "path_len"):
        assert np.array_equal(_bits(a[key]), _bits(b[key])), key
    assert int(b["heur_pairs"].item()) < 0.5 * 60 * obs.count() * 200
