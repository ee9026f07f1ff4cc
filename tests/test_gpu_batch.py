"""Batched uneven queries (one persistent rollout launch, CUDA-graph replay,
autotuned work items) vs the oracle and vs each query run alone."""

import dataclasses

import numpy as np
import pytest

import oracle
import synth

from _helpers import to_dev_agents, subset_agents, u32

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


def _small_queries(n=9, seed=77):
    """Uneven sphere scenes, small enough for the oracle."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for q in range(n):
        w = synth.sphere_workload(seed=int(g.integers(1, 1 << 30)),
                                  n_raw=int(g.integers(3000, 40000)),
                                  voxel=float(np.float32(g.uniform(0.006, 0.012))),
                                  n_agents=int(g.integers(1, 40)), n_steps=int(g.integers(20, 160)))
        out.append(w)
    return out


def _specs(ws_list, cap=None):
    import torch
    specs = []
    for w in ws_list:
        specs.append({"xyz": torch.from_numpy(w["xyz"]).cuda(), "T": w["T"], "ws": w["workspace"],
                      "agents": to_dev_agents(w["agents"]), "prm": w["params"],
                      "obs_cap": cap if cap is not None else 16384})
    return specs


def test_batch_matches_oracle_per_query(gm):
    ws_list = _small_queries()
    b = gm.Batch(_specs(ws_list))
    b.run()
    gm.sync()
    for w, r in zip(ws_list, b.results):
        ref_f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
        n = r["obs"].count()
        assert n == ref_f["n"]
        assert np.array_equal(u32(r["obs"].keys[:n]), ref_f["keys"])
        obs = np.stack([ref_f["x"], ref_f["y"], ref_f["z"]])
        ref = oracle.rollout(obs, ref_f["r_O"], w["agents"], w["params"])
        err = np.abs(r["out"]["traj"].cpu().numpy() - ref["traj"]).max()
        assert err <= POS_TOL
        c_ref = oracle.costs(ref, w["params"])
        gi, oi = int(r["best"].item()), oracle.select(c_ref)
        assert gi == oi or abs(c_ref[gi] - c_ref[oi]) < 1e-6
        assert np.allclose(r["costs"].cpu().numpy(), c_ref, rtol=1e-4, atol=1e-4)


def test_query_alone_equals_query_in_batch(gm):
    """Work items depend only on their own query: bit-identical results."""
    ws_list = _small_queries(seed=5)
    big = gm.Batch(_specs(ws_list))
    big.run()
    gm.sync()
    for q in (0, 4, 8):
        alone = gm.Batch(_specs([ws_list[q]]))
        alone.run()
        gm.sync()
        a, bq = alone.results[0], big.results[q]
        for k in ("traj", "p_final", "path_len"):
            assert np.array_equal(a["out"][k].cpu().numpy(), bq["out"][k].cpu().numpy()), k
        assert np.array_equal(a["costs"].cpu().numpy(), bq["costs"].cpu().numpy())
        assert int(a["best"].item()) == int(bq["best"].item())


def test_graph_replay_equals_direct_run(gm):
    import torch
    ws_list = _small_queries(seed=9)
    b = gm.Batch(_specs(ws_list))
    b.run()
    gm.sync()
    ref = [r["out"]["traj"].clone() for r in b.results]
    s = torch.cuda.Stream()
    for _ in range(2):
        for r in b.results:
            r["out"]["traj"].zero_()
        torch.cuda.synchronize()
        b.launch_graph(s)
        s.synchronize()
        gm.sync()
        for r, t in zip(b.results, ref):
            assert torch.equal(r["out"]["traj"], t)


def test_autotuner_and_every_tuning_agree_with_oracle(gm):
    ws_list = _small_queries(n=5, seed=21)
    b = gm.Batch(_specs(ws_list))
    shape, ms = b.autotune()
    assert ms > 0 and shape[0] in (2, 4, 6, 8, 12, 16)
    for tune in ((2, 256), (16, 256), (6, 384), (8, 512)):
        b.set_tuning(*tune)
        b.run()
        gm.sync()
        for w, r in zip(ws_list, b.results):
            ref_f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
            obs = np.stack([ref_f["x"], ref_f["y"], ref_f["z"]])
            ref = oracle.rollout(obs, ref_f["r_O"], w["agents"], w["params"], want_traj=False)
            assert np.abs(r["out"]["p_final"].cpu().numpy() - ref["p_final"]).max() <= POS_TOL


def test_full_64_scene_batch(gm):
    """The 64 uneven sphere scenes (raw 5k-300k points, 4-10 mm voxels,
    32-1024 agents, 100-1000 steps): every filter bit-exact, rollouts of
    sampled agents within tolerance."""
    ws_list = synth.batch_workloads()
    b = gm.Batch(_specs(ws_list, cap=32768), want_traj=False)
    b.run()
    gm.sync()
    rng = np.random.Generator(np.random.PCG64(3))
    for q, (w, r) in enumerate(zip(ws_list, b.results)):
        ref_f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
        n = r["obs"].count()
        assert n == ref_f["n"], q
        assert np.array_equal(u32(r["obs"].keys[:n]), ref_f["keys"])
        if q % 8 == 0:
            na = w["agents"]["k_r"].size
            idx = np.sort(rng.choice(na, size=min(3, na), replace=False))
            obs = np.stack([ref_f["x"], ref_f["y"], ref_f["z"]])
            ref = oracle.rollout(obs, ref_f["r_O"], subset_agents(w["agents"], idx), w["params"],
                                 want_traj=False)
            got = r["out"]["p_final"].cpu().numpy()[:, idx]
            assert np.abs(got - ref["p_final"]).max() <= POS_TOL


def test_capacity_errors(gm):
    ws_list = _small_queries(n=3, seed=31)
    b = gm.Batch(_specs(ws_list, cap=64))
    b.run()
    with pytest.raises(gm.GmappError) as e:
        gm.sync()
    assert e.value.status == 2


def test_obstacle_sets_larger_than_shared_memory(gm):
    """A 2 mm voxel sphere scene holds more obstacles than one CTA's shared
    memory; the remainder is streamed from L2 with the same arithmetic."""
    w = synth.sphere_workload(seed=4242, n_raw=120000, voxel=0.003, n_agents=9, n_steps=60)
    ref_f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    assert ref_f["n"] > 19000
    b = gm.Batch(_specs([w], cap=1 << 16))
    b.run()
    gm.sync()
    r = b.results[0]
    assert r["obs"].count() == ref_f["n"]
    obs = np.stack([ref_f["x"], ref_f["y"], ref_f["z"]])
    ref = oracle.rollout(obs, ref_f["r_O"], w["agents"], w["params"])
    assert np.abs(r["out"]["traj"].cpu().numpy() - ref["traj"]).max() <= POS_TOL


@pytest.mark.parametrize("clear", [False, True])
def test_block_culled_batch_equals_unculled(gm, clear):
    """gmapp_batch_set_culling: the work items visit only the resident
    obstacle blocks whose bounding box meets a gate; trajectories, path
    lengths, costs and the selections equal the unculled batch's bit for bit
    (with the clearance, the costs use the culled clearance, so only the
    trajectories and path lengths are compared)."""
    ws_list = _small_queries(seed=11)
    outs = []
    for cull in (False, True):
        b = gm.Batch(_specs(ws_list), want_clear=clear)
        b.set_culling(cull)
        b.run()
        gm.sync()
        outs.append(b)
    for q in range(len(ws_list)):
        a, c = outs[0].results[q], outs[1].results[q]
        for k in ("traj", "p_final", "v_final", "path_len"):
            assert np.array_equal(a["out"][k].cpu().numpy().view(np.uint32),
                                  c["out"][k].cpu().numpy().view(np.uint32)), (q, k)
        if not clear:
            assert np.array_equal(a["costs"].cpu().numpy().view(np.uint32),
                                  c["costs"].cpu().numpy().view(np.uint32)), q
            assert int(a["best"].item()) == int(c["best"].item())


def test_rejected_tuning_leaves_batch_unchanged(gm):
    """A tuning the batch rejects (more work items than the planner holds)
    leaves the kernel, its shared-memory shard and the item list as they
    were: the next run gives the same results bit for bit, within tolerance
    of the oracle.  The obstacle capacity exceeds one CTA's shared memory, so
    a shard size taken from the rejected tuning would not fit the kernel."""
    g = np.random.Generator(np.random.PCG64(404))
    ws_list = [synth.sphere_workload(seed=int(g.integers(1, 1 << 30)), n_raw=3000, voxel=0.01,
                                     n_agents=1000, n_steps=12) for _ in range(17)]
    b = gm.Batch(_specs(ws_list, cap=1 << 16), want_traj=False)
    b.set_tuning(16, 256)
    b.run()
    gm.sync()
    first = [r["out"]["p_final"].cpu().numpy().copy() for r in b.results]
    with pytest.raises(gm.GmappError) as e:
        b.set_tuning(2, 256)  # 17 x 500 items > the planner's 8192
    assert e.value.status == 2
    b.run()
    gm.sync()
    for q, (w, r) in enumerate(zip(ws_list, b.results)):
        got = r["out"]["p_final"].cpu().numpy()
        assert np.array_equal(got.view(np.uint32), first[q].view(np.uint32)), q
        if q % 8 == 0:
            ref_f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
            idx = np.array([0, 499, 999])
            obs = np.stack([ref_f["x"], ref_f["y"], ref_f["z"]])
            ref = oracle.rollout(obs, ref_f["r_O"], subset_agents(w["agents"], idx), w["params"],
                                 want_traj=False)
            assert np.abs(got[:, idx] - ref["p_final"]).max() <= POS_TOL


@pytest.mark.parametrize("clear", [False, True])
def test_block_culled_batch_equals_unculled_beyond_shared_memory(gm, clear):
    """Obstacle sets larger than one CTA's shared memory (the remainder comes
    from L2): culled and unculled batches keep the same obstacles resident,
    so their results are equal bit for bit here too."""
    ws_list = [synth.sphere_workload(seed=4242, n_raw=120000, voxel=0.003, n_agents=9, n_steps=60),
               synth.sphere_workload(seed=77, n_raw=150000, voxel=0.0025, n_agents=21, n_steps=40)]
    outs = []
    for cull in (False, True):
        b = gm.Batch(_specs(ws_list, cap=1 << 16), want_clear=clear)
        b.set_culling(cull)
        b.run()
        gm.sync()
        outs.append(b)
    assert min(r["obs"].count() for r in outs[0].results) > 19000
    for q in range(len(ws_list)):
        a, c = outs[0].results[q], outs[1].results[q]
        for k in ("traj", "p_final", "v_final", "path_len"):
            assert np.array_equal(a["out"][k].cpu().numpy().view(np.uint32),
                                  c["out"][k].cpu().numpy().view(np.uint32)), (q, k)


def test_four_term_cost_in_the_batch(gm):
    """Batched queries scored by the paper's four-term cost (Eq.
    cost_function) with the selection against each query's C_best on the
    device: run 1 picks the argmin and stores its cost, run 2 (same scenes)
    applies i* = argmin {C_i < alpha C_best}.  Costs agree with
    rollout_agents + score_and_select4 on each query and with the oracle's
    four_term_costs; selections follow the alpha rule on the batch's costs."""
    import math
    import torch
    ws_list = _small_queries(n=5, seed=61)
    specs = _specs(ws_list)
    alpha = 0.999
    for w, sp in zip(ws_list, specs):
        w["params"] = dataclasses.replace(w["params"], cost_radius=0.05, a_max=50.0,
                                          w4=(1.0, 2.0, 1.0, 0.5))
        sp["prm"] = w["params"]
        sp["cost4"] = True
        sp["alpha"] = alpha
        sp["c_best"] = torch.full((1,), math.nan, dtype=torch.float32, device="cuda")
    b = gm.Batch(specs)
    prev = [math.nan] * len(ws_list)
    for run in range(2):
        b.run()
        gm.sync()
        for q, (w, sp, r) in enumerate(zip(ws_list, specs, b.results)):
            prm = w["params"]
            C = r["costs"].cpu().numpy().astype(np.float64)
            best = int(r["best"].item())
            assert best == oracle.select(C, prev[q], alpha)
            if best >= 0:
                assert float(sp["c_best"].item()) == np.float32(C[best])
                prev[q] = float(np.float32(C[best]))
            if run == 0:
                out = gm.alloc_rollout_out(w["agents"]["k_r"].size, prm.n_steps, want_cost4=True)
                gm.rollout_agents(r["obs"], to_dev_agents(w["agents"]), prm, out=out)
                sel = gm.score_and_select4(out, prm)
                gm.sync()
                assert np.allclose(C, sel["costs"].cpu().numpy(), rtol=1e-4, atol=1e-5)
                f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
                o = np.stack([f["x"], f["y"], f["z"]])
                ref = oracle.rollout(o, f["r_O"], w["agents"], prm, want_trace=True)
                want = oracle.four_term_costs(ref["traj"], ref["m_trace"], prm.goal, prm.dt,
                                              prm.cost_radius, prm.a_max, prm.w4)["C"]
                assert np.allclose(C, want, rtol=1e-3, atol=1e-3)
