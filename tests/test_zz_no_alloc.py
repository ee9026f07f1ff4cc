"""The allocation-free filter entry point (filter_cloud_noalloc) gives the
same S_W as filter_cloud.

filter_cloud_noalloc serves callers that may not allocate device memory once
running, e.g. a fixed-memory real-time control loop: its scratch is a fixed
array in the library instead of a caller workspace.  Two calls in a row are
compared with filter_cloud's result (bit-exact: the filter is integer work
plus an exact binary32 sequence), so leftovers of the first call in the
shared array cannot leak into the second.  This file is collected last."""

import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _fields(o, n):
    return {f: getattr(o, f)[:n].cpu().numpy().copy() for f in ("keys", "counts", "rep_idx", "x", "y", "z")}


def test_noalloc_filter_matches_filter_cloud_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2606_12579_b300 as gm
    from paper_2606_12579_b300 import _abi

    lib = _abi.load()
    cases = [synth.tabletop_workload(n_agents=1, n_steps=1),
             synth.sphere_workload(),
             synth.tabletop_workload(n_agents=1, n_steps=1, frame_seed=99)]
    ref_obs = gm.Obstacles.empty(131072)
    for w in cases:
        xyz = torch.from_numpy(w["xyz"]).cuda()
        gm.filter_cloud(xyz, w["T"], w["workspace"], out=ref_obs)
        gm.sync()
        n_ref = ref_obs.count()
        ref = _fields(ref_obs, n_ref)
        for call in range(2):
            out = gm.Obstacles.empty(131072)
            out.x.fill_(-1.0)
            out.counts.fill_(-1)
            Tc = (C.c_float * 12)(*[float(v) for v in w["T"]])
            wss = gm._ws_struct(w["workspace"])
            ob = out._struct()
            st = lib.filter_cloud_noalloc(C.c_void_p(xyz.data_ptr()), xyz.shape[0], C.byref(Tc),
                                          C.byref(wss), C.byref(ob),
                                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert st == 0, lib.gmapp_last_error()
            torch.cuda.synchronize()
            assert out.count() == n_ref, (call, out.count(), n_ref)
            got = _fields(out, n_ref)
            for f in ref:
                assert np.array_equal(got[f], ref[f]), (call, f)
            assert ob.r_O == pytest.approx(w["workspace"].voxel / 2)


def test_noalloc_rejects_oversize_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2606_12579_b300 as gm
    from synth.workloads import Workspace
    xyz = torch.zeros(1024, 3, device="cuda")
    out = gm.Obstacles.empty(1024)
    big = Workspace(lo=(0, 0, 0), voxel=0.001, dims=(1000, 1000, 1000))  # 125 MB bitmap
    with pytest.raises(gm.GmappError) as e:
        gm.filter_cloud_noalloc(xyz, [1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], big, out)
    assert e.value.status == 2
    assert "16777216" in str(e.value)
