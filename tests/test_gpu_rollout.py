"""GPU rollout_agents vs the oracle (Sec. IV-A, Eq. mfi, Alg. 1).

  * per-force parity at fixed oracle states: |f_gpu - f_ref| <= 1e-5 |f_ref|
    plus 1/r_d per gate-ambiguous pair (FP32 and FP64 may decide a pair whose
    distance is within rounding of r_d differently);
  * rollout parity: every trajectory point within 1e-3 m after N_k steps, on
    the sphere workload (full), the tabletop workload (full 256 agents on the
    GPU in the bench's launch shape, a sample of agents on the oracle), for
    many launch shapes, and on the edge cases (no obstacles, one obstacle,
    one agent, no gate, obstacle counts that are not multiples of the
    cluster or of 4, capacity errors);
  * bit-identical repeats.
"""

import dataclasses
import math

import numpy as np
import pytest

import oracle
import synth

from _helpers import to_dev_agents, subset_agents, gate_allowance

pytestmark = pytest.mark.gpu
POS_TOL = 1e-3     # m, after N_k steps
FORCE_TOL = 1e-5   # relative, per force vector


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
    obs = np.stack([ref["x"], ref["y"], ref["z"]])
    return obs, ref["r_O"]


def _gpu_obstacles(gm, obs, r_O, cap=None):
    import torch
    return gm.Obstacles.from_points(torch.from_numpy(np.ascontiguousarray(obs, np.float32)), r_O,
                                    cap=cap)


def _compare_rollout(gpu, ref, idx=None, tol=POS_TOL):
    traj = gpu["traj"].cpu().numpy().astype(np.float64)
    if idx is not None:
        traj = traj[idx]
    err = np.abs(traj - ref["traj"]).max()
    assert err <= tol, f"trajectory error {err:.3e} m"
    pf = gpu["p_final"].cpu().numpy()
    pf = pf[:, idx] if idx is not None else pf
    assert np.abs(pf - ref["p_final"]).max() <= tol
    L = gpu["path_len"].cpu().numpy()
    L = L[idx] if idx is not None else L
    assert np.abs(L - ref["path_len"]).max() <= tol
    mc = gpu["min_clear"].cpu().numpy()
    mc = mc[idx] if idx is not None else mc
    fin = np.isfinite(ref["min_clear"])
    assert np.array_equal(np.isfinite(mc), fin)
    assert np.abs(mc[fin] - ref["min_clear"][fin]).max(initial=0) <= tol
    return err


def test_force_parity_at_oracle_states(gm):
    """Evaluate f_r once (N_k = 1) at states taken from oracle trajectories
    close to the obstacles and compare the force vectors."""
    import torch
    w = synth.sphere_workload()
    obs, r_O = _filtered(w)
    prm = w["params"]
    ref = oracle.rollout(obs, r_O, w["agents"], prm)
    na = w["agents"]["k_r"].size
    states_p, states_v, cols = [], [], []
    for k in (1, 60, 120, 160, 180, 199):
        p = ref["traj"][:, k].T
        v = (ref["traj"][:, k] - ref["traj"][:, k - 1]).T / prm.dt
        states_p.append(p)
        states_v.append(v)
        cols.append(np.arange(na))
    P = np.concatenate(states_p, axis=1).astype(np.float32)
    V = np.concatenate(states_v, axis=1).astype(np.float32)
    idx = np.concatenate(cols)
    ag = subset_agents(w["agents"], idx)
    ag["p0"], ag["v0"] = np.ascontiguousarray(P), np.ascontiguousarray(V)
    one = dataclasses.replace(prm, n_steps=1)
    out = gm.rollout_agents(_gpu_obstacles(gm, obs, r_O), to_dev_agents(ag), one, want_trace=True)
    gm.sync()
    f_gpu = out["f_trace"][:, 0, :].cpu().numpy().T.astype(np.float64)
    W_gpu = out["w_trace"][:, 0].cpu().numpy()
    r = oracle.cf_eval(obs, r_O, P.astype(np.float64), V.astype(np.float64), ag, prm.rho, prm.eps)
    amb = gate_allowance(obs.astype(np.float64), P.astype(np.float64),
                         ag["r_a"].astype(np.float64) + r_O, ag["r_d"].astype(np.float64))
    gnorm = np.linalg.norm(r["f_r"], axis=0) / np.maximum(r["W"], 1e-300)
    allow = amb * gnorm / ag["r_d"].astype(np.float64)
    fn = np.linalg.norm(r["f_r"], axis=0)
    err = np.linalg.norm(f_gpu - r["f_r"], axis=0)
    active = fn > 0
    assert active.sum() >= 8, "the states must be inside the detection radius"
    assert np.all(err <= FORCE_TOL * fn + allow + 1e-12), (err / np.maximum(fn, 1e-30)).max()
    assert np.allclose(W_gpu, r["W"], rtol=FORCE_TOL, atol=0) or np.any(amb)
    m_gpu = out["m_trace"][:, 0].cpu().numpy()
    assert np.abs(m_gpu - r["m"]).max() <= 1e-6


def test_sphere_workload_full(gm):
    w = synth.sphere_workload()
    obs, r_O = _filtered(w)
    ref = oracle.rollout(obs, r_O, w["agents"], w["params"])
    import torch
    xyz = torch.from_numpy(w["xyz"]).cuda()
    gobs = gm.filter_cloud(xyz, w["T"], w["workspace"], cap=8192)
    out = gm.rollout_agents(gobs, to_dev_agents(w["agents"]), w["params"])
    gm.sync()
    _compare_rollout(out, ref)


def test_tabletop_full_size_sampled_agents(gm):
    """All 256 agents x 500 steps on the GPU (default launch shape, as the
    bench runs it); 16 agents checked against the oracle."""
    import torch
    w = synth.tabletop_workload()
    xyz = torch.from_numpy(w["xyz"]).cuda()
    gobs = gm.filter_cloud(xyz, w["T"], w["workspace"], cap=131072)
    out = gm.rollout_agents(gobs, to_dev_agents(w["agents"]), w["params"])
    gm.sync()
    idx = np.arange(0, 256, 16) + np.arange(16) % 7
    obs, r_O = _filtered(w)
    ref = oracle.rollout(obs, r_O, subset_agents(w["agents"], idx), w["params"])
    _compare_rollout(out, ref, idx=idx)


# (cluster, agents per group, compute threads[, exchange]); exchange 1 = the
# cooperative-grid exchange through global memory
SHAPES = [(1, 8, 256), (1, 3, 128), (2, 4, 256), (3, 5, 384), (4, 8, 512), (5, 2, 256),
          (8, 1, 128), (8, 16, 256), (16, 7, 256), (16, 8, 512), (7, 10, 384), (2, 14, 384),
          (3, 10, 512), (5, 10, 384, 1), (1, 8, 256, 1), (3, 5, 128, 1), (16, 3, 512, 1),
          (2, 16, 256, 1)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "c%d_a%d_t%d" % s[:3] + ("_grid" if s[3:] == (1,) else ""))
def test_launch_shapes(gm, shape):
    w = synth.sphere_workload(n_agents=21, n_steps=120)
    obs, r_O = _filtered(w)
    ref = oracle.rollout(obs, r_O, w["agents"], w["params"])
    out = gm.rollout_agents(_gpu_obstacles(gm, obs, r_O, cap=4096), to_dev_agents(w["agents"]),
                            w["params"], tuning=shape)
    gm.sync()
    _compare_rollout(out, ref)


@pytest.mark.parametrize("gated", [True, False])
@pytest.mark.parametrize("n_obs", [0, 1, 2, 3, 5, 17, 1001])
def test_small_obstacle_counts(gm, n_obs, gated):
    """Shards of every size and parity (one to many CTAs per group), with and
    without a detection gate (r_d = inf: the pair loop without the gate
    masks over the real obstacles, the masked loop for an odd last one)."""
    g = np.random.Generator(np.random.PCG64(n_obs))
    obs = np.stack([g.uniform(0.35, 0.45, n_obs), g.uniform(-0.03, 0.03, n_obs),
                    g.uniform(0.37, 0.43, n_obs)]).astype(np.float32)
    w = synth.sphere_workload(n_agents=5, n_steps=150)
    if not gated:
        w["agents"] = dict(w["agents"], r_d=np.full(5, np.inf, np.float32))
    ref = oracle.rollout(obs, 0.005, w["agents"], w["params"])
    for shape in ((1, 5, 128), (4, 2, 256), (16, 3, 128), (4, 2, 256, 1), (16, 3, 128, 1)):
        out = gm.rollout_agents(_gpu_obstacles(gm, obs, 0.005, cap=1024), to_dev_agents(w["agents"]),
                                w["params"], tuning=shape)
        gm.sync()
        _compare_rollout(out, ref)


def test_single_agent_no_gate_dense(gm):
    w = synth.adjoint_workload(n_obs=6000, n_agents=3, n_steps=200)
    ref = oracle.rollout(w["obstacles"], w["r_O"], w["agents"], w["params"], want_trace=True)
    out = gm.rollout_agents(_gpu_obstacles(gm, w["obstacles"], w["r_O"]), to_dev_agents(w["agents"]),
                            w["params"], want_trace=True)
    gm.sync()
    _compare_rollout(out, ref)
    pen = out["clear_pen"].cpu().numpy()
    assert np.allclose(pen, ref["clear_pen"], rtol=1e-3, atol=1e-5)
    one = subset_agents(w["agents"], [1])
    ref1 = oracle.rollout(w["obstacles"], w["r_O"], one, w["params"])
    out1 = gm.rollout_agents(_gpu_obstacles(gm, w["obstacles"], w["r_O"]), to_dev_agents(one),
                             w["params"])
    gm.sync()
    _compare_rollout(out1, ref1)


def test_capacity_error_and_nothing_written(gm):
    import torch
    w = synth.sphere_workload(n_agents=4, n_steps=10)
    obs, r_O = _filtered(w)
    o = _gpu_obstacles(gm, obs, r_O, cap=4096)
    o.n.fill_(5000)  # more than cap
    out = gm.alloc_rollout_out(4, 10)
    out["p_final"].fill_(7.0)
    gm.rollout_agents(o, to_dev_agents(w["agents"]), w["params"], out=out)
    with pytest.raises(gm.GmappError) as e:
        gm.sync()
    assert e.value.status == 2
    assert torch.all(out["p_final"] == 7.0)
    # shard that cannot fit: a launch shape too small for the capacity is refused on the host
    with pytest.raises(gm.GmappError):
        gm.rollout_agents(_gpu_obstacles(gm, obs, r_O, cap=1 << 20), to_dev_agents(w["agents"]),
                          w["params"], tuning=(1, 4, 256))


def test_bit_identical_repeats(gm):
    w = synth.sphere_workload(n_agents=40, n_steps=200)
    obs, r_O = _filtered(w)
    o = _gpu_obstacles(gm, obs, r_O)
    ag = to_dev_agents(w["agents"])
    a = gm.rollout_agents(o, ag, w["params"])
    b = gm.rollout_agents(o, ag, w["params"])
    gm.sync()
    assert np.array_equal(a["traj"].cpu().numpy(), b["traj"].cpu().numpy())
    assert np.array_equal(a["path_len"].cpu().numpy(), b["path_len"].cpu().numpy())


def test_invalid_arguments(gm):
    w = synth.sphere_workload(n_agents=2, n_steps=5)
    obs, r_O = _filtered(w)
    o = _gpu_obstacles(gm, obs, r_O)
    ag = to_dev_agents(w["agents"])
    for bad in (dict(n_steps=0), dict(dt=0.0), dict(eps=0.0), dict(dt=math.nan)):
        with pytest.raises(gm.GmappError) as e:
            gm.rollout_agents(o, ag, dataclasses.replace(w["params"], **bad))
        assert e.value.status == 1
    with pytest.raises(gm.GmappError):
        gm.rollout_agents(o, ag, w["params"], tuning=(17, 4, 256))
    with pytest.raises(gm.GmappError):
        gm.rollout_agents(o, ag, w["params"], tuning=(2, 4, 200))


def test_grid_exchange_matches_cluster_bitwise(gm):
    """Both exchanges sum the same CTA partials in rank order, so a shape
    gives bit-identical trajectories whichever carries the partials."""
    w = synth.sphere_workload(n_agents=37, n_steps=160)
    obs, r_O = _filtered(w)
    o = _gpu_obstacles(gm, obs, r_O, cap=4096)
    ag = to_dev_agents(w["agents"])
    for shape, clear in (((4, 6, 256), True), ((2, 10, 384), False), ((1, 12, 128), True),
                         ((5, 8, 512), False)):
        a = gm.rollout_agents(o, ag, w["params"], tuning=shape + (0,), want_clear=clear)
        b = gm.rollout_agents(o, ag, w["params"], tuning=shape + (1,), want_clear=clear)
        gm.sync()
        for k in ("traj", "p_final", "v_final", "path_len", "clear_pen", "min_clear"):
            if a[k] is not None:
                assert np.array_equal(a[k].cpu().numpy(), b[k].cpu().numpy()), (shape, k)


def test_grid_exchange_repeats_across_streams(gm):
    """The launch epoch keeps stale slot words of earlier launches from
    matching: back-to-back grid-exchange launches, alternating between two
    streams and with changing shapes, all give the same result."""
    import torch
    w = synth.sphere_workload(n_agents=40, n_steps=60)
    obs, r_O = _filtered(w)
    o = _gpu_obstacles(gm, obs, r_O, cap=4096)
    ag = to_dev_agents(w["agents"])
    ref = gm.rollout_agents(o, ag, w["params"], tuning=(4, 8, 256, 1))
    gm.sync()
    ref_p = ref["p_final"].cpu().numpy()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = []
    for i in range(12):
        shape = (4, 8, 256, 1) if i % 3 else (5, 5, 128, 1)
        s = streams[i % 2]
        with torch.cuda.stream(s):
            outs.append((shape, gm.rollout_agents(o, ag, w["params"], tuning=shape, stream=s)))
    torch.cuda.synchronize()
    gm.sync()
    for shape, out in outs:
        if shape == (4, 8, 256, 1):
            assert np.array_equal(out["p_final"].cpu().numpy(), ref_p)
        else:
            assert np.abs(out["p_final"].cpu().numpy() - ref_p).max() < 1e-4


def test_autotuner_picks_a_measured_shape(gm):
    """The autotuner times candidate shapes on the caller's inputs, caches
    the fastest, and later rollouts of the same sizes use it."""
    w = synth.sphere_workload(n_agents=40, n_steps=150)
    obs, r_O = _filtered(w)
    o = _gpu_obstacles(gm, obs, r_O, cap=4096)
    ag = to_dev_agents(w["agents"])
    out = gm.alloc_rollout_out(40, 150, want_clear=False)
    shape, ms = gm.autotune_rollout(o, ag, w["params"], out=out, candidates=6, probe_steps=30)
    assert ms > 0 and len(shape) == 4
    assert gm.pick_tuning(4096, 40) == shape
    res = gm.rollout_agents(o, ag, w["params"])
    gm.sync()
    ref = oracle.rollout(obs, r_O, w["agents"], w["params"])
    _compare_rollout(res, ref)
