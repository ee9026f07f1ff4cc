"""GPU rollout_adjoint and the autograd Function vs the FP64 oracle adjoint
and FP64 central finite differences.

Tolerance: relative L2 error over all gradient entries <= 1e-3 against the
oracle's adjoint (FP32 recomputation of 10^2-10^3 steps against FP64), and
per-entry error <= 1e-3 of the agent's gradient scale against FD samples
that cross no kink.
"""

import dataclasses

import numpy as np
import pytest

import oracle
import synth

from _helpers import to_dev_agents, subset_agents

pytestmark = pytest.mark.gpu
GRAD_TOL = 1e-3
GROUPS = {"v0": slice(0, 3), "k_r": slice(3, 4), "k_a": slice(4, 5), "c": slice(5, 8)}


@pytest.fixture(scope="module")
def gm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2606_12579_b300 as gm
    gm.context()
    return gm


def _gpu_forward_adjoint(gm, obs, r_O, agents, prm, cap=None):
    import torch
    o = gm.Obstacles.from_points(torch.from_numpy(np.ascontiguousarray(obs, np.float32)), r_O,
                                 cap=cap)
    ag = to_dev_agents(agents)
    na, K = int(ag["k_r"].numel()), int(prm.ckpt_every)
    out = gm.alloc_rollout_out(na, prm.n_steps)
    out["ckpt"] = torch.empty((prm.n_steps + K - 1) // K, 6, na, device="cuda")
    gm.rollout_agents(o, ag, prm, out=out)
    adj = gm.rollout_adjoint(o, ag, prm, out["ckpt"], want_cost=True)
    gm.sync()
    return {k: (v.cpu().numpy().astype(np.float64) if v is not None else None)
            for k, v in adj.items()}, out


def _stack(adj, idx=None):
    parts = [adj["g_v0"], adj["g_kr"][None], adj["g_ka"][None], adj["g_c"]]
    g = np.concatenate(parts, axis=0)
    return g if idx is None else g[:, idx]


def _rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _groups_ok(got, want):
    """Each parameter group (v0, k_r, k_a, c) within its own relative L2."""
    for name, sl in GROUPS.items():
        assert _rel_l2(got[sl], want[sl]) <= GRAD_TOL, name


@pytest.mark.parametrize("n_steps", [230, 50, 37])
def test_dense_vs_oracle_adjoint(gm, n_steps):
    w = synth.adjoint_workload(n_obs=6000, n_agents=24, n_steps=n_steps)
    g, _ = _gpu_forward_adjoint(gm, w["obstacles"], w["r_O"], w["agents"], w["params"])
    ref = oracle.adjoint(w["obstacles"], w["r_O"], w["agents"], w["params"])
    assert _rel_l2(_stack(g), _stack(ref)) <= GRAD_TOL
    _groups_ok(_stack(g), _stack(ref))
    assert np.allclose(g["cost"], ref["cost"], rtol=1e-4, atol=1e-5)


def test_gated_sphere_with_clearance(gm):
    w = synth.sphere_workload(n_agents=16, n_steps=200)
    f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    obs = np.stack([f["x"], f["y"], f["z"]])
    prm = dataclasses.replace(w["params"], w_clear=1.0)
    g, _ = _gpu_forward_adjoint(gm, obs, f["r_O"], w["agents"], prm)
    ref = oracle.adjoint(obs, f["r_O"], w["agents"], prm)
    assert _rel_l2(_stack(g), _stack(ref)) <= GRAD_TOL
    _groups_ok(_stack(g), _stack(ref))
    assert np.allclose(g["cost"], ref["cost"], rtol=1e-4, atol=1e-5)


def test_full_size_per_group_and_fd(gm):
    """50,000 obstacles, 512 agents, 1000 steps, checkpoints every 50 (the
    differentiable-rollout workload).  Oracle adjoint on 12 agents, each
    parameter group (v0, k_r, k_a, c) with its own relative L2 error, so a
    group of small gradients cannot hide under the large ones; FP64 central
    FD on 4 agents, every kink-free entry within 1e-3 of its group's scale."""
    w = synth.adjoint_workload()
    g, _ = _gpu_forward_adjoint(gm, w["obstacles"], w["r_O"], w["agents"], w["params"])
    idx = [0, 3, 57, 100, 200, 255, 256, 311, 400, 444, 509, 510]
    ref = oracle.adjoint(w["obstacles"], w["r_O"], subset_agents(w["agents"], idx), w["params"])
    got, want = _stack(g, idx), _stack(ref)
    assert _rel_l2(got, want) <= GRAD_TOL
    for name, sl in GROUPS.items():
        e = _rel_l2(got[sl], want[sl])
        print(f"group {name}: relative L2 error {e:.2e}")
        assert e <= GRAD_TOL, name
    assert np.allclose(g["cost"][idx], ref["cost"], rtol=1e-4, atol=1e-5)
    fd_ids = [3, 100, 311, 510]
    fd = oracle.fd_gradient(w["obstacles"], w["r_O"], w["agents"], w["params"], fd_ids)
    n_ok = 0
    for i in fd_ids:
        gf, ok = fd[i]
        n_ok += int(ok.sum())
        gi = _stack(g, [i])[:, 0]
        for name, sl in GROUPS.items():
            scale = np.abs(gf[sl]).max()
            sel = ok[sl]
            assert np.all(np.abs(gi[sl] - gf[sl])[sel] <= GRAD_TOL * scale), (i, name)
    print(f"FD: {n_ok} of {8 * len(fd_ids)} entries kink-free")
    assert n_ok >= 16


def test_many_agents_loop_over_groups(gm):
    """More agents than the co-resident CTA groups hold at once (2,000 agents
    on a small obstacle set: every group of CTAs works through several agent
    groups in one launch); sampled agents vs the oracle adjoint."""
    w = synth.adjoint_workload(n_obs=600, n_agents=2000, n_steps=64)
    prm = dataclasses.replace(w["params"], ckpt_every=16)
    g, _ = _gpu_forward_adjoint(gm, w["obstacles"], w["r_O"], w["agents"], prm)
    idx = [0, 1, 777, 1500, 1998, 1999]
    ref = oracle.adjoint(w["obstacles"], w["r_O"], subset_agents(w["agents"], idx), prm)
    assert _rel_l2(_stack(g, idx), _stack(ref)) <= GRAD_TOL
    assert np.allclose(g["cost"][idx], ref["cost"], rtol=1e-4, atol=1e-5)


@pytest.mark.parametrize("n_obs", [1, 3, 17])
def test_tiny_obstacle_sets(gm, n_obs):
    w = synth.adjoint_workload(n_obs=n_obs, n_agents=5, n_steps=45)
    prm = dataclasses.replace(w["params"], ckpt_every=10)
    g, _ = _gpu_forward_adjoint(gm, w["obstacles"], w["r_O"], w["agents"], prm)
    ref = oracle.adjoint(w["obstacles"], w["r_O"], w["agents"], prm)
    assert _rel_l2(_stack(g), _stack(ref)) <= GRAD_TOL
    assert np.allclose(g["cost"], ref["cost"], rtol=1e-4, atol=1e-5)


def test_adjoint_repeats_bitwise(gm):
    """Two adjoint passes over the same checkpoints give the same bits (the
    launch epoch separates their exchange words)."""
    import torch
    w = synth.adjoint_workload(n_obs=3000, n_agents=40, n_steps=90)
    o = gm.Obstacles.from_points(torch.from_numpy(w["obstacles"]), w["r_O"])
    ag = to_dev_agents(w["agents"])
    prm = w["params"]
    out = gm.alloc_rollout_out(40, prm.n_steps)
    K = int(prm.ckpt_every)
    out["ckpt"] = torch.empty((prm.n_steps + K - 1) // K, 6, 40, device="cuda")
    gm.rollout_agents(o, ag, prm, out=out)
    a = gm.rollout_adjoint(o, ag, prm, out["ckpt"], want_cost=True)
    b = gm.rollout_adjoint(o, ag, prm, out["ckpt"], want_cost=True)
    gm.sync()
    for k in ("g_v0", "g_kr", "g_ka", "g_c", "cost"):
        assert torch.equal(a[k], b[k]), k


def test_autograd_function_matches_adjoint(gm):
    import torch
    w = synth.adjoint_workload(n_obs=4000, n_agents=12, n_steps=120)
    prm = w["params"]
    o = gm.Obstacles.from_points(torch.from_numpy(w["obstacles"]), w["r_O"])
    ag = to_dev_agents(w["agents"])
    v0 = ag["v0"].clone().requires_grad_(True)
    k_r = ag["k_r"].clone().requires_grad_(True)
    k_a = ag["k_a"].clone().requires_grad_(True)
    c = ag["c"].clone().requires_grad_(True)
    rest = {k: ag[k] for k in ("p0", "r_d", "r_a")}
    costs = gm.GMappRollout.apply(v0, k_r, k_a, c, o, rest, prm)
    wts = torch.linspace(0.5, 2.0, 12, device="cuda")
    (costs * wts).sum().backward()
    ref = oracle.adjoint(w["obstacles"], w["r_O"], w["agents"], prm)
    assert np.allclose(costs.detach().cpu().numpy(), ref["cost"], rtol=1e-4, atol=1e-5)
    s = wts.cpu().numpy()
    got = np.concatenate([v0.grad.cpu().numpy(), k_r.grad.cpu().numpy()[None],
                          k_a.grad.cpu().numpy()[None], c.grad.cpu().numpy()], axis=0)
    assert _rel_l2(got, _stack(ref) * s[None, :]) <= GRAD_TOL


def test_gradient_step_lowers_cost(gm):
    """Agents refined by one gradient step on v0 get cheaper plans."""
    import torch
    w = synth.adjoint_workload(n_obs=4000, n_agents=32, n_steps=200)
    prm = w["params"]
    o = gm.Obstacles.from_points(torch.from_numpy(w["obstacles"]), w["r_O"])
    ag = to_dev_agents(w["agents"])
    rest = {k: ag[k] for k in ("p0", "r_d", "r_a")}
    v0 = ag["v0"].clone().requires_grad_(True)
    costs = gm.GMappRollout.apply(v0, ag["k_r"], ag["k_a"], ag["c"], o, rest, prm)
    costs.sum().backward()
    g = v0.grad
    step = 1e-3 / g.norm(dim=0).clamp_min(1e-12)
    with torch.no_grad():
        v1 = v0 - g * step
        c1 = gm.GMappRollout.apply(v1, ag["k_r"], ag["k_a"], ag["c"], o, rest, prm)
    better = (c1 < costs.detach()).float().mean().item()
    assert better >= 0.9
