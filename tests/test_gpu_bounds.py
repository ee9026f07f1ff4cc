"""The bounds-checked build (-DGMAPP_BOUNDS_CHECK, loaded with
GMAPP_BOUNDS_CHECK=1): its index checks set GMAPP_DEVERR_BOUNDS in the
device error word instead of faulting.  The path runs here on small cases
(N_O <= 64 obstacles, N_a <= 4 agents) compared with the oracle and on the
full tabletop frame through every rollout form, the stream filter over
several waves, a four-term batch and four-term served requests; the error
word must stay clean.  The check runs in a child process, which loads the checked library
in place of the normal one."""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import dataclasses, os, sys
import numpy as np, torch
sys.path.insert(0, os.path.join(sys.argv[1], "tests"))
import oracle, synth
import paper_2606_12579_b300 as gm
from _helpers import to_dev_agents
assert gm._abi.LIB_PATH.endswith("libgmapp_bc.so"), gm._abi.LIB_PATH
gm.context()

# small: a sparse sphere cloud (<= 64 voxels) and 4 agents, against the oracle
w = synth.sphere_workload(n_agents=4, n_steps=120)
xyz = w["xyz"][::400].copy()
f = oracle.filter_cloud(xyz, w["T"], w["workspace"])
assert 0 < f["n"] <= 64, f["n"]
obs = gm.filter_cloud(torch.from_numpy(xyz).cuda(), w["T"], w["workspace"], cap=64)
ref = oracle.rollout(np.stack([f["x"], f["y"], f["z"]]), f["r_O"], w["agents"], w["params"])
dev = to_dev_agents(w["agents"])
for tun in [(1, 4, 128, 0), (2, 2, 256, 1), (3, 4, 128, 0)]:
    for fn in (gm.rollout_agents, gm.rollout_agents_blockcull):
        out = fn(obs, dev, w["params"], tuning=tun)
        gm.sync()
        err = np.abs(out["traj"].cpu().numpy() - ref["traj"]).max()
        assert err <= 1e-3, (tun, err)

# full tabletop frame through every rollout form
t = synth.tabletop_workload(n_agents=48, n_steps=100)
cloud = torch.from_numpy(t["xyz"]).cuda()
obs = gm.filter_cloud(cloud, t["T"], t["workspace"], cap=80000)
ag = synth.ensemble_agents(t["agents"], 16)
dev = to_dev_agents(ag)
gm.rollout_agents(obs, dev, t["params"], tuning=(5, 6, 256, 1), want_trace=True)
gm.rollout_agents(obs, dev, t["params"], tuning=(5, 6, 384, 0))
gm.rollout_agents_blockcull(obs, dev, t["params"], tuning=(5, 6, 256, 1))
gm.rollout_ensemble(obs, dev, 16, t["params"], tuning=(5, 6, 256, 1), n_proj=16)
b = gm.Batch([{"xyz": cloud, "T": t["T"], "ws": t["workspace"], "agents": dev,
               "prm": t["params"], "obs_cap": 80000}])
b.run()
gm.sync()

# the stream filter over several waves, a four-term batch and a four-term
# served request
frames = [torch.from_numpy(synth.tabletop_workload(frame_seed=300 + i, n_agents=1,
                                                   n_steps=1)["xyz"]).cuda() for i in range(20)]
fb = gm.FilterBatch(frames, t["T"], t["workspace"], caps=[131072] * 20)
fb.run()
fb.run()
gm.sync()
p4 = dataclasses.replace(t["params"], cost_radius=0.05, a_max=50.0)
cb = torch.full((1,), float("nan"), device="cuda")
b4 = gm.Batch([{"xyz": cloud, "T": t["T"], "ws": t["workspace"], "agents": dev, "prm": p4,
                "obs_cap": 80000, "cost4": True, "alpha": 0.95, "c_best": cb}])
b4.run()
b4.run()
gm.sync()
s = synth.tabletop_workload(n_agents=20, n_steps=60, n_points=30000, voxel=0.01)
srv = gm.Server(max_slots=4, max_agents=64, max_steps=100, obs_cap=16384, arena_bytes=1 << 28,
                chunk_steps=16, agents_per_item=8, four_term=True, max_plan_streams=1,
                admit_bypass=2)
tk = [srv.submit(s["xyz"], s["T"], s["workspace"], s["agents"],
                 dataclasses.replace(s["params"], cost_radius=0.05, a_max=50.0), cost4=True,
                 alpha=0.95, plan_stream=0) for _ in range(3)]
while any(srv.poll(x) is None for x in tk):
    srv.tick()
gm.sync()
print("bounds-checked build clean")
'''


def test_bounds_checked_build_runs_clean():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    lib = os.path.join(ROOT, "paper_2606_12579_b300", "libgmapp_bc.so")
    if not os.path.exists(lib):
        from paper_2606_12579_b300 import build
        build.build(bounds_check=True)
    env = dict(os.environ, GMAPP_BOUNDS_CHECK="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "bounds-checked build clean" in r.stdout
