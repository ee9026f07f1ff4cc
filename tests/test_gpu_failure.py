"""Failure path of the bounded device-side waits, exercised without a hang
or a fault: with the context's wait limit at one poll, the grid exchange of
a multi-CTA rollout gives up (its partners' partials are not there yet), the
kernel flags GMAPP_DEVERR_TIMEOUT and still finishes -- a CTA whose wait ran
out skips its later waits -- and the host reads GMAPP_ERR_TIMEOUT.  The
context stays usable: with the limit restored the same launch matches the
oracle, for MFI rollouts and an ensemble; repeated timeouts leave the grid
exchange's launch epochs consistent.  (Only the global-memory polls of the
grid exchange are capped: nothing is in flight into shared memory when a
CTA gives up.)"""

import numpy as np
import pytest

import oracle
import synth

from _helpers import to_dev_agents

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2606_12579_b300 as gm
    gm.context()
    return gm


@pytest.fixture(scope="module")
def scene():
    w = synth.sphere_workload(n_agents=16, n_steps=120)
    f = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    obs = np.stack([f["x"], f["y"], f["z"]])
    ref = oracle.rollout(obs, f["r_O"], w["agents"], w["params"])
    return w, obs, f["r_O"], ref


def _obstacles(gm, obs, r_O):
    import torch
    return gm.Obstacles.from_points(torch.from_numpy(np.ascontiguousarray(obs, np.float32)), r_O)


@pytest.mark.parametrize("shape", [(4, 4, 256, 1), (8, 2, 128, 1)], ids=["grid4", "grid8"])
def test_exchange_timeout_is_reported_and_the_context_recovers(gm, scene, shape):
    w, obs, r_O, ref = scene
    ctx = gm.context()
    o = _obstacles(gm, obs, r_O)
    ag = to_dev_agents(w["agents"])
    try:
        ctx.set_wait_limit(1)
        for _ in range(2):   # twice: the epoch bookkeeping survives a failed launch
            gm.rollout_agents(o, ag, w["params"], tuning=shape)
            with pytest.raises(gm.GmappError) as e:
                gm.sync()
            assert e.value.status == 4     # GMAPP_ERR_TIMEOUT
    finally:
        ctx.set_wait_limit(0)
    out = gm.rollout_agents(o, ag, w["params"], tuning=shape)
    gm.sync()
    assert np.abs(out["traj"].cpu().numpy() - ref["traj"]).max() <= 1e-3


def test_ensemble_timeout_then_recovery(gm, scene):
    w, obs, r_O, _ = scene
    ag_np = synth.ensemble_agents(w["agents"], 6)
    ref = oracle.rollout(obs, r_O, ag_np, w["params"], n_apf=6, n_proj=4)
    ctx = gm.context()
    o = _obstacles(gm, obs, r_O)
    ag = to_dev_agents(ag_np)
    try:
        ctx.set_wait_limit(1)
        gm.rollout_ensemble(o, ag, 6, w["params"], tuning=(3, 3, 256, 1), n_proj=4)
        with pytest.raises(gm.GmappError) as e:
            gm.sync()
        assert e.value.status == 4
    finally:
        ctx.set_wait_limit(0)
    out = gm.rollout_ensemble(o, ag, 6, w["params"], tuning=(3, 3, 256, 1), n_proj=4)
    gm.sync()
    assert np.abs(out["traj"].cpu().numpy() - ref["traj"]).max() <= 1e-3
