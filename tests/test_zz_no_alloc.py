"""The allocation-free filter entry point (filter_cloud_noalloc) gives the
same S_W as filter_cloud.

filter_cloud_noalloc serves callers that may not allocate device memory once
running, e.g. a fixed-memory real-time control loop: its scratch is a fixed
array in the library instead of a caller workspace.  Two calls in a row are
compared with filter_cloud's result (bit-exact: the filter is integer work
plus an exact binary32 sequence), so leftovers of the first call in the
shared array cannot leak into the second; the first case is also compared
with the oracle directly.  Besides the plain grid (min_pts = 1) the tests run
the compaction branch (min_pts = 2, whose temporary arrays are carved from the
same fixed array) and an output buffer too small for the result, whose
capacity flag filter_cloud_noalloc_status reports and the next call clears.
This file is collected last."""

import ctypes as C
import dataclasses

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

FIELDS = ("keys", "counts", "rep_idx", "x", "y", "z")


def _fields(o, n):
    return {f: getattr(o, f)[:n].cpu().numpy().copy() for f in FIELDS}


def _noalloc_raw(lib, gm, xyz, w_T, ws, out):
    """One call through the C-ABI exactly as a C caller makes it."""
    import torch
    Tc = (C.c_float * 12)(*[float(v) for v in w_T])
    wss = gm._ws_struct(ws)
    ob = out._struct()
    st = lib.filter_cloud_noalloc(C.c_void_p(xyz.data_ptr()), xyz.shape[0], C.byref(Tc),
                                  C.byref(wss), C.byref(ob),
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.gmapp_last_error()
    return ob


def _cases():
    tab = synth.tabletop_workload(n_agents=1, n_steps=1)
    sph = synth.sphere_workload()
    tab2 = synth.tabletop_workload(n_agents=1, n_steps=1, frame_seed=99)
    # min_pts = 2: the compaction branch (k_keep_sums / k_keep_emit)
    ws2 = dataclasses.replace(tab["workspace"], min_pts=2)
    return [(tab["xyz"], tab["T"], tab["workspace"]), (sph["xyz"], sph["T"], sph["workspace"]),
            (tab2["xyz"], tab2["T"], tab2["workspace"]), (tab2["xyz"], tab2["T"], ws2)]


def test_noalloc_filter_matches_filter_cloud_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2606_12579_b300 as gm
    from paper_2606_12579_b300 import _abi

    lib = _abi.load()
    ref_obs = gm.Obstacles.empty(131072)
    for ci, (xyz_np, T, ws) in enumerate(_cases()):
        xyz = torch.from_numpy(xyz_np).cuda()
        gm.filter_cloud(xyz, T, ws, out=ref_obs)
        gm.sync()
        n_ref = ref_obs.count()
        ref = _fields(ref_obs, n_ref)
        if ci == 0:  # the oracle itself, on the first case
            o = oracle.filter_cloud(xyz_np, T, ws)
            assert o["n"] == n_ref
            for f in FIELDS:
                assert np.array_equal(np.asarray(o[f]).view(ref[f].dtype), ref[f]), f
        for call in range(2):
            out = gm.Obstacles.empty(131072)
            out.x.fill_(-1.0)
            out.counts.fill_(-1)
            ob = _noalloc_raw(lib, gm, xyz, T, ws, out)
            torch.cuda.synchronize()
            assert lib.filter_cloud_noalloc_status(
                C.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
            assert out.count() == n_ref, (ci, call, out.count(), n_ref)
            got = _fields(out, n_ref)
            for f in ref:
                assert np.array_equal(got[f], ref[f]), (ci, call, f)
            assert ob.r_O == pytest.approx(ws.voxel / 2)


@pytest.mark.parametrize("min_pts", [1, 2])
def test_noalloc_overflow_reports_capacity_then_clears(min_pts):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2606_12579_b300 as gm
    from paper_2606_12579_b300 import _abi

    lib = _abi.load()
    w = synth.sphere_workload()
    ws = dataclasses.replace(w["workspace"], min_pts=min_pts)
    xyz = torch.from_numpy(w["xyz"]).cuda()
    ref_obs = gm.Obstacles.empty(8192)
    gm.filter_cloud(xyz, w["T"], ws, out=ref_obs)
    gm.sync()
    n_ref = ref_obs.count()
    ref = _fields(ref_obs, n_ref)
    cap = 256
    assert n_ref > cap
    for call in range(2):
        small = gm.Obstacles.empty(cap)
        _noalloc_raw(lib, gm, xyz, w["T"], ws, small)
        with pytest.raises(gm.GmappError) as e:
            gm.filter_cloud_noalloc_status()
        assert e.value.status == 2  # GMAPP_ERR_CAPACITY
        assert small.count() == n_ref  # the number needed
        got = _fields(small, cap)
        for f in ref:  # the first cap voxels by key, as filter_cloud writes them
            assert np.array_equal(got[f], ref[f][:cap]), (call, f)
        # a call that fits clears the flag
        big = gm.Obstacles.empty(8192)
        _noalloc_raw(lib, gm, xyz, w["T"], ws, big)
        gm.filter_cloud_noalloc_status()
        assert big.count() == n_ref


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
