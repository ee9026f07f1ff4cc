"""Served control loop with continuous batching: requests admitted by
memory, advanced together in chunks; each result equals the same request
served alone (bit for bit) and the oracle's (selection rule, costs and the
chosen trajectory within tolerance)."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2606_12579_b300 as gm
    gm.context()
    return gm


def _requests(n=6, seed=3):
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for r in range(n):
        w = synth.tabletop_workload(seed=int(g.integers(1, 1 << 30)), n_points=30000, voxel=0.01,
                                    n_agents=int(g.choice([5, 17, 40])), n_steps=int(g.integers(40, 121)),
                                    spheres_at=0.1 * r, sphere_seed=11, scene_seed=99)
        out.append(w)
    return out


def _serve(gm, ws, arena=1 << 28, slots=8, stagger=False, chunk=16, culled=False):
    srv = gm.Server(max_slots=slots, max_agents=64, max_steps=200, obs_cap=16384,
                    arena_bytes=arena, chunk_steps=chunk, agents_per_item=8, culled=culled)
    tickets, results, max_active, max_pending = [], {}, 0, 0
    for i, w in enumerate(ws):
        tickets.append(srv.submit(w["xyz"], w["T"], w["workspace"], w["agents"], w["params"]))
        if stagger:
            max_active = max(max_active, srv.tick())
    for _ in range(10000):
        if len(results) == len(tickets):
            break
        max_active = max(max_active, srv.tick())
        max_pending = max(max_pending, srv.stats()["pending"])
        for t in tickets:
            if t not in results:
                r = srv.poll(t)
                if r is not None:
                    results[t] = r
    assert len(results) == len(tickets)
    out = [results[t] for t in tickets]
    for t in tickets:
        srv.release(t)
    return out, max_active, max_pending


def test_mix_equals_alone_and_oracle(gm):
    ws = _requests()
    mixed, max_active, _ = _serve(gm, ws, stagger=True)
    assert max_active >= 2, "requests must overlap on the device"
    for w, r in zip(ws, mixed):
        alone, _, _ = _serve(gm, [w])
        a = alone[0]
        assert a["best"] == r["best"]
        assert np.array_equal(a["costs"], r["costs"])
        assert np.array_equal(a["best_traj"], r["best_traj"])
        ref_f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
        assert r["n_obs"] == ref_f["n"]
        obs = np.stack([ref_f["x"], ref_f["y"], ref_f["z"]])
        ref = oracle.rollout(obs, ref_f["r_O"], w["agents"], w["params"])
        c_ref = oracle.costs(ref, w["params"])
        oi = oracle.select(c_ref)
        assert r["best"] == oi or abs(c_ref[r["best"]] - c_ref[oi]) < 1e-6
        assert np.allclose(r["costs"], c_ref, rtol=1e-4, atol=1e-4)
        assert np.abs(r["best_traj"] - ref["traj"][r["best"]]).max() <= 1e-3
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]


def test_admission_by_memory(gm):
    ws = _requests(n=5, seed=8)
    # each request needs ~1.1 MB; an arena of 2.4 MB holds two at once
    mixed, _, max_pending = _serve(gm, ws, arena=2400 << 10, slots=8)
    assert max_pending >= 1
    for w, r in zip(ws, mixed):
        alone, _, _ = _serve(gm, [w])
        assert np.array_equal(alone[0]["best_traj"], r["best_traj"])


def test_chunk_size_does_not_change_results(gm):
    ws = _requests(n=3, seed=12)
    a, _, _ = _serve(gm, ws, chunk=7)
    b, _, _ = _serve(gm, ws, chunk=200)
    for x, y in zip(a, b):
        assert np.array_equal(x["best_traj"], y["best_traj"])
        assert np.array_equal(x["costs"], y["costs"])


def test_rejections(gm):
    w = _requests(n=1)[0]
    srv = gm.Server(max_slots=2, max_agents=8, max_steps=200, obs_cap=16384,
                    arena_bytes=1 << 28, chunk_steps=16, agents_per_item=8)
    with pytest.raises(gm.GmappError) as e:
        big = dict(w["agents"])
        big = {k: np.ascontiguousarray(np.repeat(v, 20, axis=-1)) for k, v in w["agents"].items()}
        srv.submit(w["xyz"], w["T"], w["workspace"], big, w["params"])
    assert e.value.status == 1
    tiny = gm.Server(max_slots=2, max_agents=64, max_steps=200, obs_cap=16384,
                     arena_bytes=1 << 20, chunk_steps=16, agents_per_item=8)
    with pytest.raises(gm.GmappError) as e:
        tiny.submit(w["xyz"], w["T"], w["workspace"], w["agents"], w["params"])
    assert e.value.status == 2


# ---- the culled server (each agent visits the obstacles within its reach) --

def test_culled_mix_equals_alone_equals_single_query_and_oracle(gm):
    """Culled serving: every result is bit-identical alone and in the mix,
    and bit-identical to rollout_agents_culled of the same request (same
    per-step arithmetic, state kept exactly between chunks); within the
    rollout tolerance of the oracle's all-pairs definition."""
    import torch
    ws = _requests(n=5, seed=21)
    mixed, max_active, _ = _serve(gm, ws, stagger=True, culled=True)
    assert max_active >= 2
    for w, r in zip(ws, mixed):
        alone, _, _ = _serve(gm, [w], culled=True)
        assert np.array_equal(alone[0]["costs"], r["costs"])
        assert np.array_equal(alone[0]["best_traj"], r["best_traj"])
        obs = gm.filter_cloud(torch.from_numpy(w["xyz"]).cuda(), w["T"], w["workspace"],
                              cap=16384)
        index = gm.grid_index(obs, w["workspace"])
        ag = {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda()
              for k, v in w["agents"].items()}
        single = gm.rollout_agents_culled(obs, w["workspace"], index, ag, w["params"],
                                          want_clear=False)
        sel = gm.score_and_select(single, w["params"])
        gm.sync()
        assert np.array_equal(sel["costs"].cpu().numpy(), r["costs"])
        assert np.array_equal(single["traj"][r["best"]].cpu().numpy(), r["best_traj"])
        ref_f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
        o = np.stack([ref_f["x"], ref_f["y"], ref_f["z"]])
        ref = oracle.rollout(o, ref_f["r_O"], w["agents"], w["params"])
        c_ref = oracle.costs(ref, w["params"])
        oi = oracle.select(c_ref)
        assert r["best"] == oi or abs(c_ref[r["best"]] - c_ref[oi]) < 1e-6
        assert np.abs(r["best_traj"] - ref["traj"][r["best"]]).max() <= 1e-3


def test_culled_chunk_size_does_not_change_results(gm):
    ws = _requests(n=3, seed=13)
    a, _, _ = _serve(gm, ws, chunk=5, culled=True)
    b, _, _ = _serve(gm, ws, chunk=200, culled=True)
    for x, y in zip(a, b):
        assert np.array_equal(x["best_traj"], y["best_traj"])
        assert np.array_equal(x["costs"], y["costs"])


def test_block_culled_server_equals_all_pairs_server(gm):
    """culled = "blocks": each work item's agents visit only the resident
    obstacle blocks whose bounding box meets a gate, in the voting loop's
    order, so every result equals the all-pairs server's bit for bit."""
    ws = _requests()
    a, _, _ = _serve(gm, ws, stagger=True)
    b, _, _ = _serve(gm, ws, stagger=True, culled="blocks")
    for ra, rb in zip(a, b):
        assert ra["best"] == rb["best"] and ra["n_obs"] == rb["n_obs"]
        assert np.array_equal(ra["costs"].view(np.uint32), rb["costs"].view(np.uint32))
        assert np.array_equal(ra["best_traj"].view(np.uint32), rb["best_traj"].view(np.uint32))


def test_block_culled_server_equals_all_pairs_beyond_shared_memory(gm):
    """Frames whose obstacle sets exceed one CTA's shared memory (5 mm voxels,
    the remainder streamed from L2): both chunk-kernel modes keep the same
    obstacles resident, so the block-culled server still equals the
    all-pairs server bit for bit."""
    g = np.random.Generator(np.random.PCG64(55))
    ws = [synth.tabletop_workload(seed=int(g.integers(1, 1 << 30)), n_points=60000, voxel=0.005,
                                  n_agents=int(g.choice([5, 17, 40])), n_steps=int(g.integers(40, 101)),
                                  spheres_at=0.1 * r, sphere_seed=11, scene_seed=99)
          for r in range(3)]
    res, caps = [], []
    for culled in (False, "blocks"):
        srv = gm.Server(max_slots=4, max_agents=64, max_steps=200, obs_cap=65536,
                        arena_bytes=1 << 29, chunk_steps=16, agents_per_item=8, culled=culled)
        caps.append(srv.stats()["shard_cap"])
        tickets = [srv.submit(w["xyz"], w["T"], w["workspace"], w["agents"], w["params"]) for w in ws]
        done = {}
        for _ in range(10000):
            if len(done) == len(tickets):
                break
            srv.tick()
            for t in tickets:
                if t not in done:
                    r = srv.poll(t)
                    if r is not None:
                        done[t] = r
        res.append([done[t] for t in tickets])
    assert caps[0] == caps[1] < 20000
    for ra, rb in zip(res[0], res[1]):
        assert ra["n_obs"] > caps[0]
        assert ra["best"] == rb["best"] and ra["n_obs"] == rb["n_obs"]
        assert np.array_equal(ra["costs"].view(np.uint32), rb["costs"].view(np.uint32))
        assert np.array_equal(ra["best_traj"].view(np.uint32), rb["best_traj"].view(np.uint32))


def test_served_stream_shape_mix_equals_alone_and_oracle(gm):
    """The served control loop at the stream's own shape: 200k-point tabletop
    frames with 4 moving spheres (1 cm voxels), N_a in {64, 256, 1024},
    N_k = 300, a server sized for 1024 agents, 9 requests in flight together.
    Each result equals the same request served alone bit for bit; every
    agent's cost, the selection and the chosen trajectory agree with the
    oracle."""
    _, na_choice, request = synth.serve_stream(n_requests=10000)
    picks = [r for r in range(64) if na_choice[r] == 1024][:3] + \
            [r for r in range(64) if na_choice[r] == 256][:3] + \
            [r for r in range(64) if na_choice[r] == 64][:3]
    ws = [request(r) for r in sorted(picks)]
    assert sorted({w["agents"]["k_r"].size for w in ws}) == [64, 256, 1024]

    def serve(batch):
        srv = gm.Server(max_slots=16, max_agents=1024, max_steps=300, obs_cap=32768,
                        arena_bytes=2 << 30, chunk_steps=50, agents_per_item=8, threads=256)
        tickets = [srv.submit(w["xyz"], w["T"], w["workspace"], w["agents"], w["params"])
                   for w in batch]
        done, max_active = {}, 0
        for _ in range(100000):
            if len(done) == len(tickets):
                break
            max_active = max(max_active, srv.tick())
            for t in tickets:
                if t not in done:
                    r = srv.poll(t)
                    if r is not None:
                        done[t] = r
        return [done[t] for t in tickets], max_active

    mixed, max_active = serve(ws)
    assert max_active >= 8, "the requests must be in flight together"
    for w, r in zip(ws, mixed):
        (a,), _ = serve([w])
        assert a["best"] == r["best"] and a["n_obs"] == r["n_obs"]
        assert np.array_equal(a["costs"].view(np.uint32), r["costs"].view(np.uint32))
        assert np.array_equal(a["best_traj"].view(np.uint32), r["best_traj"].view(np.uint32))
        ref_f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
        assert r["n_obs"] == ref_f["n"]
        obs = np.stack([ref_f["x"], ref_f["y"], ref_f["z"]])
        ref = oracle.rollout(obs, ref_f["r_O"], w["agents"], w["params"])
        c_ref = oracle.costs(ref, w["params"])
        oi = oracle.select(c_ref)
        assert r["best"] == oi or abs(c_ref[r["best"]] - c_ref[oi]) < 1e-6
        assert np.allclose(r["costs"], c_ref, rtol=1e-4, atol=1e-4)
        assert np.abs(r["best_traj"] - ref["traj"][r["best"]]).max() <= 1e-3


def _four_term_requests():
    """A plan stream of successive frames (moving spheres) plus plain-cost
    requests and a four-term request without a stream, interleaved."""
    import dataclasses
    ws = _requests(n=8, seed=41)
    for w in ws:
        w["params"] = dataclasses.replace(w["params"], cost_radius=0.05, a_max=50.0,
                                          w4=(1.0, 2.0, 1.0, 0.5))
    # (request, cost4, plan_stream)
    kinds = [(0, True, 0), (1, False, -1), (2, True, 0), (3, True, -1), (4, True, 0),
             (5, False, -1), (6, True, 0), (7, True, 0)]
    return ws, kinds


def _serve4(gm, ws, kinds, alpha, one_at_a_time=False, bypass=4, culled=False):
    srv = gm.Server(max_slots=8, max_agents=64, max_steps=200, obs_cap=16384,
                    arena_bytes=1 << 28, chunk_steps=16, agents_per_item=8,
                    four_term=True, max_plan_streams=2, admit_bypass=bypass, culled=culled)
    out, max_active = [], 0
    tickets = []
    for r, c4, ps in kinds:
        w = ws[r]
        t = srv.submit(w["xyz"], w["T"], w["workspace"], w["agents"], w["params"], cost4=c4,
                       alpha=alpha, plan_stream=ps)
        tickets.append(t)
        if one_at_a_time:
            res = None
            while res is None:
                srv.tick()
                res = srv.poll(t)
        else:
            max_active = max(max_active, srv.tick())
    done = {}
    for _ in range(10000):
        if len(done) == len(tickets):
            break
        max_active = max(max_active, srv.tick())
        for t in tickets:
            if t not in done:
                res = srv.poll(t)
                if res is not None:
                    done[t] = res
    return [done[t] for t in tickets], max_active


@pytest.mark.parametrize("culled", [False, True, "blocks"], ids=["all_pairs", "grid", "blocks"])
def test_four_term_server_plan_stream(gm, culled):
    """The paper's four-term cost (Eq. cost_function) and the selection
    against the current plan (i* = argmin {C_i < alpha C_best}) in the served
    loop.  A plan stream of five requests shares one device-resident C_best,
    mixed with plain-cost requests and a four-term request without a
    stream.  Every result equals the same sequence served one request at a
    time, bit for bit; each four-term request's costs and selection agree
    with rollout_agents + score_and_select4 on the same query with its own
    C_best chain; the selection follows alpha C_best on the server's costs;
    and the costs and selections agree with the oracle's four_term_costs and
    select on the oracle's own chain.  The culled servers (voxel grid, obstacle
    blocks) use the culled clearance, which equals the exact one wherever it
    counts here: the cost radius (5 cm) does not exceed the detection radius,
    so obstacles beyond an agent's reach add nothing to the obstacle term."""
    import math
    import torch
    alpha = 0.95
    ws, kinds = _four_term_requests()
    mixed, max_active = _serve4(gm, ws, kinds, alpha, culled=culled)
    assert max_active >= 2
    alone, _ = _serve4(gm, ws, kinds, alpha, one_at_a_time=True, bypass=0, culled=culled)
    for a, b in zip(alone, mixed):
        assert a["best"] == b["best"]
        assert np.array_equal(a["costs"].view(np.uint32), b["costs"].view(np.uint32))
        if b["best"] >= 0:
            assert np.array_equal(a["best_traj"].view(np.uint32), b["best_traj"].view(np.uint32))
    c_dev = torch.full((1,), math.nan, dtype=torch.float32, device="cuda")
    srv_best, ora_best = math.nan, math.nan
    kept, agree = 0, 0
    for (r, c4, ps), res in zip(kinds, mixed):
        w = ws[r]
        prm = w["params"]
        if not c4:
            continue
        # the same query through the single-query calls
        obs = gm.filter_cloud(torch.from_numpy(w["xyz"]).cuda(), w["T"], w["workspace"],
                              cap=16384)
        out = gm.alloc_rollout_out(w["agents"]["k_r"].size, prm.n_steps, want_cost4=True)
        gm.rollout_agents(obs, {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda()
                                for k, v in w["agents"].items()}, prm, out=out)
        sel = gm.score_and_select4(out, prm, c_best=c_dev if ps == 0 else None, alpha=alpha)
        gm.sync()
        direct = sel["costs"].cpu().numpy().astype(np.float64)
        assert np.allclose(res["costs"], direct, rtol=1e-4, atol=1e-5)
        # the server's selection follows the alpha rule on its own costs
        prev = srv_best if ps == 0 else math.nan
        want = oracle.select(res["costs"].astype(np.float64), prev, alpha)
        assert res["best"] == want
        if ps == 0 and res["best"] >= 0:
            srv_best = float(res["costs"][res["best"]])
        kept += res["best"] < 0
        # the oracle on its own chain
        f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
        o = np.stack([f["x"], f["y"], f["z"]])
        ref = oracle.rollout(o, f["r_O"], w["agents"], prm, want_trace=True)
        C = oracle.four_term_costs(ref["traj"], ref["m_trace"], prm.goal, prm.dt,
                                   prm.cost_radius, prm.a_max, prm.w4)["C"]
        assert np.allclose(res["costs"], C, rtol=1e-3, atol=1e-3)
        oprev = ora_best if ps == 0 else math.nan
        oi = oracle.select(C, oprev, alpha)
        if ps == 0 and oi >= 0:
            ora_best = float(C[oi])
        gi = res["best"]
        same = gi == oi or (gi >= 0 and oi >= 0 and abs(C[gi] - C[oi]) < 1e-4)
        agree += same
    print(f"four-term server: {kept} requests kept the current plan; {agree} of 6 selections "
          f"agree with the oracle's chain")
    assert agree >= 5


def _admission_case():
    """A small request, then a large one (a 300k-point frame), then eight
    small ones, all queued before the first tick."""
    small = _requests(n=9, seed=71)
    g = np.random.Generator(np.random.PCG64(72))
    big = synth.tabletop_workload(seed=int(g.integers(1, 1 << 30)), n_points=300000, voxel=0.01,
                                  n_agents=17, n_steps=60, spheres_at=0.3, sphere_seed=11,
                                  scene_seed=99)
    return [small[0], big] + small[1:]


def _bytes_of(gm, w):
    """Arena bytes the server gives one request (read from its free bytes)."""
    srv = gm.Server(max_slots=2, max_agents=64, max_steps=200, obs_cap=32768,
                    arena_bytes=64 << 20, chunk_steps=1, agents_per_item=8)
    free0 = srv.stats()["arena_free_bytes"]
    srv.submit(w["xyz"], w["T"], w["workspace"], w["agents"], w["params"])
    srv.tick()
    used = free0 - srv.stats()["arena_free_bytes"]
    while srv.poll(1) is None:
        srv.tick()
    return used


def test_first_fit_admission_with_aging_bound(gm):
    """admit_bypass = k: queued requests that fit are admitted past an older
    one that does not, but once that one has been overtaken k times nothing
    later is admitted before it.  k = 0 is strict arrival order.  Results do
    not depend on the order (bit for bit)."""
    ws = _admission_case()
    b_small, b_big = _bytes_of(gm, ws[0]), _bytes_of(gm, ws[1])
    assert b_big >= b_small + 2 * _bytes_of(gm, ws[2])
    arena = (b_big + 4095) // 4096 * 4096  # the large request fits only alone

    def run(bypass):
        srv = gm.Server(max_slots=8, max_agents=64, max_steps=200, obs_cap=32768,
                        arena_bytes=arena, chunk_steps=16, agents_per_item=8,
                        admit_bypass=bypass)
        tickets = [srv.submit(w["xyz"], w["T"], w["workspace"], w["agents"], w["params"])
                   for w in ws]
        done = {}
        for _ in range(100000):
            if len(done) == len(tickets):
                break
            srv.tick()
            for t in tickets:
                if t not in done:
                    r = srv.poll(t)
                    if r is not None:
                        done[t] = r
        res = [done[t] for t in tickets]
        overtook = sum(r["t_admit"] < res[1]["t_admit"] for r in res[2:])
        return res, overtook

    strict, n0 = run(0)
    aged, n2 = run(2)
    free, n64 = run(64)
    gm.sync()  # no capacity or timeout flag from any of the runs
    assert n0 == 0 and n2 == 2 and n64 > 2, (n0, n2, n64)
    for a, b, c in zip(strict, aged, free):
        assert a["best"] == b["best"] == c["best"]
        assert np.array_equal(a["costs"], b["costs"]) and np.array_equal(a["costs"], c["costs"])
        assert np.array_equal(a["best_traj"], b["best_traj"])
