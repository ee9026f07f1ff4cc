"""The pair loop's block test: Alg. 1 evaluates the heuristic terms of a
pair only inside the detection gate, and the rollout kernel takes that
branch per warp, for a block of 128 obstacles at once.  Without the
clearance, a block is tested on the expanded distance |o|^2 - 2 p.o (three
FMAs per pair) with a rounding margin.  With the clearance, every pair's
exact |d|^2 is tested.  Neither test may skip a pair that the exact |d|^2
puts inside the gate.  So at one launch shape both variants must give
bit-identical W and trajectories, and the count of evaluated heuristic pairs
must cover every pair inside the gates.  The cases: obstacles within a few
ulp of the gate radius, a scene tens of metres from the origin, and a whole
tabletop rollout."""

import dataclasses

import numpy as np
import pytest

import synth

from _helpers import to_dev_agents

pytestmark = pytest.mark.gpu
SMALL = (3, 6, 256, 1)    # 20k obstacles: shards of 6.7k
TABLE = (5, 6, 256, 1)    # tabletop: shards of 16k


@pytest.fixture(scope="module")
def gm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2606_12579_b300 as gm
    gm.context()
    return gm


def _both(gm, obs, agents, prm, tuning):
    """W traces and trajectories without and with the clearance, plus the
    heuristic-pair counts of each launch."""
    import torch
    na, nk = int(agents["k_r"].numel()), int(prm.n_steps)
    outs = []
    for clear in (False, True):
        o = gm.alloc_rollout_out(na, nk, want_traj=True, want_trace=True, want_clear=clear)
        o["f_trace"] = None
        if not clear:
            o["m_trace"] = None
        o["heur_pairs"] = torch.zeros(1, dtype=torch.int64, device="cuda")
        gm.rollout_agents(obs, agents, prm, out=o, tuning=tuning)
        outs.append(o)
    gm.sync()
    return outs


def _boundary_agents(rng, obs_np, R, r_d, n):
    """n agents, each placed at the gate radius (r_d + R) of one obstacle,
    scaled by (1 + k 2^-23) for k in -4..4: pairs right at the boundary."""
    j = rng.integers(0, obs_np.shape[1], n)
    u = rng.normal(size=(3, n))
    u /= np.linalg.norm(u, axis=0)
    k = np.arange(n) % 9 - 4
    rad = (r_d + R) * (1.0 + k * 2.0 ** -23)
    p0 = (obs_np[:, j].astype(np.float64) + u * rad).astype(np.float32)
    v = rng.normal(size=(3, n)).astype(np.float32) * 0.05
    c = rng.normal(size=(3, n)).astype(np.float32)
    return {"p0": p0, "v0": v, "c": c,
            "k_r": np.full(n, 1.0, np.float32), "k_a": np.full(n, 2.0, np.float32),
            "r_d": np.full(n, r_d, np.float32), "r_a": np.full(n, R - 0.005, np.float32)}


@pytest.mark.parametrize("offset", [(0.0, 0.0, 0.0), (30.0, -40.0, 12.0)])
def test_boundary_pairs_are_never_skipped(gm, offset):
    import torch
    rng = np.random.default_rng(1701)
    off = np.asarray(offset, np.float64)[:, None]
    obs_np = (rng.uniform(0.0, 1.0, size=(3, 20000)) + off).astype(np.float32)
    r_O, r_d = 0.005, 0.05
    R = 0.01 + r_O
    ag = _boundary_agents(rng, obs_np, R, r_d, 288)
    obs = gm.Obstacles.from_points(torch.from_numpy(obs_np), r_O)
    prm = dataclasses.replace(synth.sphere_workload(n_agents=1, n_steps=1)["params"], n_steps=1,
                              goal=tuple(float(v) for v in (off[:, 0] + 0.5)))
    a, b = _both(gm, obs, to_dev_agents(ag), prm, SMALL)
    Wa, Wb = a["w_trace"].cpu().numpy(), b["w_trace"].cpu().numpy()
    assert np.count_nonzero(Wb) >= 100   # the boundary pairs are exercised
    assert np.array_equal(Wa.view(np.uint32), Wb.view(np.uint32))
    assert np.array_equal(a["traj"].cpu().numpy().view(np.uint32),
                          b["traj"].cpu().numpy().view(np.uint32))
    ha, hb = int(a["heur_pairs"].item()), int(b["heur_pairs"].item())
    assert ha % 64 == 0 and hb % 64 == 0 and hb <= ha


def test_tabletop_rollout_identical_with_and_without_clearance(gm):
    import torch
    w = synth.tabletop_workload(n_agents=48, n_steps=300)
    obs = gm.filter_cloud(torch.from_numpy(w["xyz"]).cuda(), w["T"], w["workspace"], cap=80000)
    a, b = _both(gm, obs, to_dev_agents(w["agents"]), w["params"], TABLE)
    assert np.array_equal(a["w_trace"].cpu().numpy().view(np.uint32),
                          b["w_trace"].cpu().numpy().view(np.uint32))
    assert np.array_equal(a["traj"].cpu().numpy().view(np.uint32),
                          b["traj"].cpu().numpy().view(np.uint32))
    assert np.count_nonzero(b["w_trace"].cpu().numpy()) > 1000


def test_heuristic_pair_count_covers_the_gated_pairs(gm):
    """N_k = 1: the count is a multiple of 64, at least the number of pairs
    inside the gates at the start (FP64, away from the boundary), and at
    most every pair; agents far from every obstacle evaluate none."""
    import torch
    w = synth.tabletop_workload(n_agents=64, n_steps=1)
    xyz = torch.from_numpy(w["xyz"]).cuda()
    obs = gm.filter_cloud(xyz, w["T"], w["workspace"], cap=80000)
    n_obs = obs.count()
    o_np = np.stack([t[:n_obs].cpu().numpy() for t in (obs.x, obs.y, obs.z)]).astype(np.float64)
    ag = dict(w["agents"])
    # start half the agents right above the table surface
    rng = np.random.default_rng(5)
    pick = rng.integers(0, n_obs, 32)
    ag["p0"] = ag["p0"].copy()
    ag["p0"][:, :32] = (o_np[:, pick] + np.array([[0.0], [0.0], [0.03]])).astype(np.float32)
    a, _ = _both(gm, obs, to_dev_agents(ag), w["params"], TABLE)
    R = ag["r_a"].astype(np.float64) + obs.r_O
    inside = 0
    for i in range(64):
        d = np.sqrt(((o_np - ag["p0"][:, i:i + 1].astype(np.float64)) ** 2).sum(axis=0))
        inside += int(np.count_nonzero(d <= (ag["r_d"][i] + R[i]) * (1 - 1e-5)))
    h = int(a["heur_pairs"].item())
    assert inside > 1000
    assert h % 64 == 0 and inside <= h <= 66 * (n_obs + 128 * 5)   # 11 groups x 6 slots
    far = dict(ag)
    far["p0"] = np.ascontiguousarray(ag["p0"] + np.float32(5.0))
    f, _ = _both(gm, obs, to_dev_agents(far), w["params"], TABLE)
    assert int(f["heur_pairs"].item()) == 0


@pytest.mark.parametrize("n_proj,n_apf", [(0, 48), (48, 0), (24, 24)])
def test_ensemble_identical_with_and_without_clearance(gm, n_proj, n_apf):
    """APF and projected-current groups (and MFI beside them): the block
    test of the clearance variant (exact |d|^2) and of the plain one
    (expanded distance) give bit-identical force records and trajectories."""
    import torch
    w = synth.tabletop_workload(n_agents=96, n_steps=200)
    ag = synth.ensemble_agents(w["agents"], n_apf)
    obs = gm.filter_cloud(torch.from_numpy(w["xyz"]).cuda(), w["T"], w["workspace"], cap=80000)
    dev = to_dev_agents(ag)
    outs = []
    for clear in (False, True):
        o = gm.alloc_rollout_out(96, 200, want_traj=True, want_trace=True, want_clear=clear)
        if not clear:
            o["m_trace"] = None
        gm.rollout_ensemble(obs, dev, n_apf, w["params"], out=o, tuning=TABLE, n_proj=n_proj)
        outs.append(o)
    gm.sync()
    a, b = outs
    for key in ("traj", "w_trace", "f_trace"):
        assert np.array_equal(a[key].cpu().numpy().view(np.uint32),
                              b[key].cpu().numpy().view(np.uint32)), key
    assert np.count_nonzero(b["w_trace"].cpu().numpy()) > 1000


def test_clearance_equals_the_batched_kernel_without_gated_pairs(gm):
    """The clearance minimum of the rollout kernel (per-block exact test,
    blocks dealt round-robin over the CTAs) against the batched kernel (one
    CTA, resident obstacles in order).  With r_d below eps no pair passes a
    gate (W = 0), so the trajectories are the attractor's alone and equal in
    both kernels: the clearance sums and minima must then be equal bit for
    bit, as the minimum of the same exact |d|^2 values."""
    import torch
    w = synth.tabletop_workload(n_agents=40, n_steps=300)
    ag = dict(w["agents"])
    ag["r_d"] = np.full(40, 0.5e-3, np.float32)          # below eps: no gate
    rng = np.random.default_rng(11)
    ag["p0"] = (ag["p0"] + rng.normal(scale=0.05, size=ag["p0"].shape)).astype(np.float32)
    dev = to_dev_agents(ag)
    xyz = torch.from_numpy(w["xyz"]).cuda()
    obs = gm.filter_cloud(xyz, w["T"], w["workspace"], cap=80000)
    a = gm.rollout_agents(obs, dev, w["params"], tuning=TABLE, want_clear=True)
    b = gm.Batch([{"xyz": xyz, "T": w["T"], "ws": w["workspace"], "agents": dev,
                   "prm": w["params"], "obs_cap": 80000}], want_clear=True)
    b.run()
    gm.sync()
    o = b.results[0]["out"]
    for key in ("traj", "clear_pen", "min_clear"):
        assert np.array_equal(a[key].cpu().numpy().view(np.uint32),
                              o[key].cpu().numpy().view(np.uint32)), key
    assert np.all(np.isfinite(a["min_clear"].cpu().numpy()))
