"""GPU rollout with spatial culling (the voxel grid as a neighbour grid) vs
the oracle's all-pairs definition (Eq. mfi, Alg. 1, Sec. IV-A).

Alg. 1's gate zeroes every pair beyond r_d + R, so the culled W equals the
all-pairs W up to the order of the FP32 additions: the trajectories must lie
within 1e-3 m of the FP64 oracle, the W of one step within 1e-5 relative of
the all-pairs kernel's at the same states, and the clearance must be exact
wherever the nearest obstacle lies within the reach (at least r_d
elsewhere).  The neighbour index must equal the lower bounds of the keys.
"""

import dataclasses

import numpy as np
import pytest

import oracle
import synth

from _helpers import to_dev_agents, subset_agents

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


def _check_clearance(gpu_mc, ref_mc, r_d):
    near = ref_mc < r_d
    assert np.abs(gpu_mc[near] - ref_mc[near]).max(initial=0) <= POS_TOL
    assert np.all(gpu_mc[~near] >= r_d[~near] - POS_TOL)


def _run(gm, w, cap):
    import torch
    xyz = torch.from_numpy(w["xyz"]).cuda()
    obs = gm.filter_cloud(xyz, w["T"], w["workspace"], cap=cap)
    index = gm.grid_index(obs, w["workspace"])
    out = gm.rollout_agents_culled(obs, w["workspace"], index, to_dev_agents(w["agents"]),
                                   w["params"])
    gm.sync()
    return obs, index, out


def test_grid_index_is_the_lower_bound_of_the_keys(gm):
    w = synth.tabletop_workload(n_agents=1, n_steps=1)
    ref = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    import torch
    obs = gm.filter_cloud(torch.from_numpy(w["xyz"]).cuda(), w["T"], w["workspace"], cap=131072)
    index = gm.grid_index(obs, w["workspace"])
    gm.sync()
    dims = w["workspace"].dims
    nw = (dims[0] * dims[1] * dims[2] + 31) // 32
    want = np.searchsorted(ref["keys"].astype(np.int64), 32 * np.arange(nw + 1, dtype=np.int64),
                           side="left")
    assert np.array_equal(index.cpu().numpy().view(np.uint32)[:nw + 1].astype(np.int64), want)


def test_sphere_culled_matches_oracle(gm):
    w = synth.sphere_workload(n_agents=24, n_steps=200)
    _, _, out = _run(gm, w, 8192)
    f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    obs = np.stack([f["x"], f["y"], f["z"]])
    ref = oracle.rollout(obs, f["r_O"], w["agents"], w["params"])
    err = np.abs(out["traj"].cpu().numpy() - ref["traj"]).max()
    assert err <= POS_TOL, err
    assert np.abs(out["path_len"].cpu().numpy() - ref["path_len"]).max() <= POS_TOL
    _check_clearance(out["min_clear"].cpu().numpy(), ref["min_clear"],
                     w["agents"]["r_d"].astype(np.float64))


def test_tabletop_culled_full_size_sampled_agents(gm):
    w = synth.tabletop_workload()
    _, _, out = _run(gm, w, 131072)
    idx = np.arange(0, 256, 16) + np.arange(16) % 5
    f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    obs = np.stack([f["x"], f["y"], f["z"]])
    ref = oracle.rollout(obs, f["r_O"], subset_agents(w["agents"], idx), w["params"])
    err = np.abs(out["traj"].cpu().numpy()[idx] - ref["traj"]).max()
    assert err <= POS_TOL, err
    _check_clearance(out["min_clear"].cpu().numpy()[idx], ref["min_clear"],
                     w["agents"]["r_d"][idx].astype(np.float64))


def test_culled_W_equals_all_pairs_W_at_the_same_states(gm):
    """One step (N_k = 1) from states along oracle trajectories, large and
    small radii: the culled sum equals the all-pairs kernel's."""
    w = synth.tabletop_workload(n_agents=64, n_steps=300)
    f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    obs_np = np.stack([f["x"], f["y"], f["z"]])
    ref = oracle.rollout(obs_np, f["r_O"], w["agents"], w["params"])
    ag = dict(w["agents"])
    ag["p0"] = np.ascontiguousarray(ref["traj"][:, 250].T.astype(np.float32))
    ag["r_d"] = np.where(np.arange(64) % 2, 0.05, 0.12).astype(np.float32)
    one = dataclasses.replace(w["params"], n_steps=1)
    import torch
    obs = gm.filter_cloud(torch.from_numpy(w["xyz"]).cuda(), w["T"], w["workspace"], cap=131072)
    index = gm.grid_index(obs, w["workspace"])
    dev = to_dev_agents(ag)
    a = gm.rollout_agents_culled(obs, w["workspace"], index, dev, one, want_trace=True)
    b = gm.rollout_agents(obs, dev, one, want_trace=True)
    gm.sync()
    Wa, Wb = a["w_trace"][:, 0].cpu().numpy(), b["w_trace"][:, 0].cpu().numpy()
    assert np.count_nonzero(Wb) >= 20
    assert np.allclose(Wa, Wb, rtol=1e-5, atol=0)


def test_agents_at_the_grid_edges(gm):
    """Agents starting at and beyond the workspace corners: the neighbour
    box is clamped to the grid."""
    w = synth.sphere_workload(n_agents=6, n_steps=120)
    ag = dict(w["agents"])
    starts = np.array([[0.0, -0.5, 0.0], [0.999, 0.499, 0.799], [-0.05, 0.0, 0.4],
                       [0.5, 0.6, 0.4], [0.42, 0.0, 0.4], [0.5, 0.0, 0.29]], np.float32).T
    ag["p0"] = np.ascontiguousarray(starts)
    w["agents"] = ag
    _, _, out = _run(gm, w, 8192)
    f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    obs = np.stack([f["x"], f["y"], f["z"]])
    ref = oracle.rollout(obs, f["r_O"], ag, w["params"])
    assert np.abs(out["traj"].cpu().numpy() - ref["traj"]).max() <= POS_TOL
    _check_clearance(out["min_clear"].cpu().numpy(), ref["min_clear"],
                     ag["r_d"].astype(np.float64))


def test_culled_errors(gm):
    w = synth.sphere_workload(n_agents=3, n_steps=10)
    obs, index, _ = _run(gm, w, 8192)
    ag = dict(w["agents"])
    ag["r_d"] = np.array([0.05, np.inf, 0.05], np.float32)   # no gate: nothing to cull by
    gm.rollout_agents_culled(obs, w["workspace"], index, to_dev_agents(ag), w["params"])
    with pytest.raises(gm.GmappError) as e:
        gm.sync()
    assert e.value.status == 1
    out = gm.alloc_rollout_out(3, 10, want_trace=True)   # f_trace is not produced
    with pytest.raises(gm.GmappError) as e:
        gm.rollout_agents_culled(obs, w["workspace"], index, to_dev_agents(w["agents"]),
                                 w["params"], out=out)
    assert e.value.status == 1
