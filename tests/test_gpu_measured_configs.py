"""Parity at the configurations the benchmark measures (Sec. IV-A step,
Eq. (mfi), Alg. 1's clamp and gate).

  * the tabletop query exactly as bench.py runs it: a frame of its ring,
    obs_cap = first-frame N_O x 1.05 rounded up to 64, the launch shape its
    autotuner picks (candidates = 16, probe = 100 steps) and the shape the
    recorded runs picked, (5, 9, 384, grid exchange); 24 agents compared
    point by point with the oracle's trajectories;
  * per-force parity at fixed oracle states on the tabletop set (5 mm voxels,
    ~74k obstacles, the block gate test at full size, NaN-padded last block)
    with agents placed within +-4 ulp of an obstacle's gate radius, and on the
    dense ungated set (50,000 obstacles, r_d = inf: the plain pair loop), under
    the bound of test_gpu_rollout.test_force_parity_at_oracle_states:
    |f_gpu - f_ref| <= 1e-5 |f_ref| + (1/r_d) rho k_r |g| per gate-ambiguous pair.
"""

import dataclasses

import numpy as np
import pytest

import oracle
import synth

from _helpers import to_dev_agents, subset_agents, gate_allowance

pytestmark = pytest.mark.gpu
POS_TOL = 1e-3     # m, after N_k steps
FORCE_TOL = 1e-5   # relative, per force vector
BENCH_SHAPE = (5, 9, 384, 1)


@pytest.fixture(scope="module")
def gm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2606_12579_b300 as gm
    gm.context()
    return gm


def _bench_frame(f=0):
    """Frame f of bench.py's ring (rank 0) with the tabletop query's agents."""
    base = synth.tabletop_workload()
    frame = synth.tabletop_workload(frame_seed=7_000_000 + f, n_agents=1, n_steps=1)
    return base, frame["xyz"]


def _compare(gpu, ref, idx):
    traj = gpu["traj"].cpu().numpy().astype(np.float64)[idx]
    err = np.abs(traj - ref["traj"]).max()
    assert err <= POS_TOL, f"trajectory error {err:.3e} m"
    assert np.abs(gpu["p_final"].cpu().numpy()[:, idx] - ref["p_final"]).max() <= POS_TOL
    assert np.abs(gpu["path_len"].cpu().numpy()[idx] - ref["path_len"]).max() <= POS_TOL
    return err


def test_tabletop_at_the_bench_launch(gm):
    import torch
    base, xyz_np = _bench_frame(0)
    prm = base["params"]
    xyz = torch.from_numpy(xyz_np).cuda()
    probe = gm.filter_cloud(xyz, base["T"], base["workspace"], cap=131072)
    obs_cap = (int(probe.count() * 1.05) + 63) // 64 * 64
    obs = gm.Obstacles.empty(obs_cap)
    gm.filter_cloud(xyz, base["T"], base["workspace"], out=obs)
    agents = to_dev_agents(base["agents"])
    ro = gm.alloc_rollout_out(256, int(prm.n_steps), want_traj=True, want_clear=False)
    gm.rollout_agents(obs, agents, prm, out=ro)
    gm.sync()
    tuned, _ = gm.autotune_rollout(obs, agents, prm, out=ro, candidates=16, probe_steps=100)
    f = oracle.filter_cloud(xyz_np, base["T"], base["workspace"])
    assert obs.count() == f["n"] <= obs_cap
    o = np.stack([f["x"], f["y"], f["z"]])
    idx = np.sort(np.concatenate([np.arange(0, 256, 16) + np.arange(16) % 9,
                                  np.array([1, 2, 3, 127, 128, 129, 254, 255])]))
    ref = oracle.rollout(o, f["r_O"], subset_agents(base["agents"], idx), prm)
    shapes = [BENCH_SHAPE] + ([tuned] if tuple(tuned) != BENCH_SHAPE else [])
    for shape in shapes:
        out = gm.alloc_rollout_out(256, int(prm.n_steps), want_traj=True, want_clear=False)
        gm.rollout_agents(obs, agents, prm, out=out, tuning=shape)
        gm.sync()
        err = _compare(out, ref, idx)
        print(f"shape {shape}: max trajectory error {err:.2e} m over {idx.size} agents")
        costs = gm.score_and_select(out, prm)
        gm.sync()
        c_ref = oracle.costs(ref, prm)
        got = costs["costs"].cpu().numpy()[idx]
        assert np.allclose(got, c_ref, rtol=1e-4, atol=1e-4)


def _force_parity(gm, obs, r_O, ag, prm, tuning=None, cap=None):
    """Evaluate f_r once (N_k = 1) at the agents' (p0, v0) and compare with
    the oracle's FP64 evaluation at the same FP32 states.  Returns the number
    of agents with a nonzero force and of gate-ambiguous pairs."""
    import torch
    one = dataclasses.replace(prm, n_steps=1)
    o = gm.Obstacles.from_points(torch.from_numpy(np.ascontiguousarray(obs, np.float32)), r_O,
                                 cap=cap)
    out = gm.rollout_agents(o, to_dev_agents(ag), one, want_trace=True, tuning=tuning)
    gm.sync()
    f_gpu = out["f_trace"][:, 0, :].cpu().numpy().T.astype(np.float64)
    P, V = ag["p0"].astype(np.float64), ag["v0"].astype(np.float64)
    r = oracle.cf_eval(obs.astype(np.float64), r_O, P, V, ag, prm.rho, prm.eps)
    amb = gate_allowance(obs.astype(np.float64), P, ag["r_a"].astype(np.float64) + r_O,
                         ag["r_d"].astype(np.float64))
    gnorm = np.linalg.norm(r["f_r"], axis=0) / np.maximum(r["W"], 1e-300)
    allow = amb * gnorm / ag["r_d"].astype(np.float64)
    fn = np.linalg.norm(r["f_r"], axis=0)
    err = np.linalg.norm(f_gpu - r["f_r"], axis=0)
    bad = err > FORCE_TOL * fn + allow + 1e-12
    assert not bad.any(), (np.flatnonzero(bad)[:8], (err / np.maximum(fn, 1e-30)).max())
    m_gpu = out["m_trace"][:, 0].cpu().numpy()
    assert np.abs(m_gpu - r["m"]).max() <= 1e-6
    return int((fn > 0).sum()), int(amb.sum())


def _oracle_states(obs, r_O, agents, prm, ks):
    """(p_k, v_{k-1}) of the oracle's trajectories at the listed steps, as
    FP32 agent inputs (the other agent fields repeated)."""
    ref = oracle.rollout(obs, r_O, agents, prm)
    na = agents["k_r"].size
    P, V, cols = [], [], []
    for k in ks:
        P.append(ref["traj"][:, k].T)
        V.append((ref["traj"][:, k] - ref["traj"][:, k - 1]).T / prm.dt)
        cols.append(np.arange(na))
    ag = subset_agents(agents, np.concatenate(cols))
    ag["p0"] = np.ascontiguousarray(np.concatenate(P, axis=1).astype(np.float32))
    ag["v0"] = np.ascontiguousarray(np.concatenate(V, axis=1).astype(np.float32))
    return ag


def _near_gate_states(obs, agents, r_O, n=48, seed=5):
    """Agents placed at (R + r_d)(1 + k 2^-23), k in -4..4, from a random
    obstacle along a random direction: their pair with that obstacle sits
    within a few ulp of the gate (Alg. 1's s <= r_d)."""
    g = np.random.Generator(np.random.PCG64(seed))
    na = agents["k_r"].size
    pick = g.integers(0, na, n)
    ag = subset_agents(agents, pick)
    j = g.integers(0, obs.shape[1], n)
    u = g.normal(size=(3, n))
    u /= np.linalg.norm(u, axis=0)
    k = np.arange(n) % 9 - 4
    R = ag["r_a"].astype(np.float64) + r_O
    rad = (R + ag["r_d"].astype(np.float64)) * (1.0 + k * 2.0 ** -23)
    ag["p0"] = np.ascontiguousarray((obs[:, j].astype(np.float64) + u * rad).astype(np.float32))
    v = g.normal(size=(3, n))
    ag["v0"] = np.ascontiguousarray((v / np.linalg.norm(v, axis=0)).astype(np.float32))
    return ag


@pytest.mark.parametrize("tuning", [None, BENCH_SHAPE], ids=["default", "bench_shape"])
def test_force_parity_tabletop_states(gm, tuning):
    base, xyz_np = _bench_frame(0)
    prm = base["params"]
    f = oracle.filter_cloud(xyz_np, base["T"], base["workspace"])
    obs = np.stack([f["x"], f["y"], f["z"]])
    assert obs.shape[1] > 60000
    idx = np.arange(0, 256, 16)
    ag = _oracle_states(obs, f["r_O"], subset_agents(base["agents"], idx), prm,
                        ks=(1, 100, 200, 300, 400, 499))
    near = _near_gate_states(obs, base["agents"], f["r_O"])
    both = {key: np.ascontiguousarray(np.concatenate([ag[key], near[key]], axis=-1))
            for key in ag}
    cap = (obs.shape[1] + 127) // 128 * 128 + 64  # a NaN-padded last block
    active, amb = _force_parity(gm, obs, f["r_O"], both, prm, tuning=tuning, cap=cap)
    print(f"tabletop: {both['k_r'].size} states, {active} with a force, {amb} gate-ambiguous pairs")
    assert active >= 48 and amb >= 1


def test_force_parity_dense_ungated_states(gm):
    w = synth.adjoint_workload()
    obs, r_O, prm = w["obstacles"], w["r_O"], w["params"]
    idx = np.array([0, 37, 128, 255, 300, 411, 480, 511])
    short = dataclasses.replace(prm, n_steps=300)
    ag = _oracle_states(obs, r_O, subset_agents(w["agents"], idx), short, ks=(1, 100, 200, 299))
    active, amb = _force_parity(gm, obs, r_O, ag, prm)
    print(f"dense: {ag['k_r'].size} states, {active} with a force")
    assert active == ag["k_r"].size and amb == 0
