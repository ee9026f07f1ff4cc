"""Pins for the oracle's perception filter (Sec. IV-B, Sec. V-A).

The filter's result has a plain definition (group points by the voxel that
contains them), so it is pinned by: a hand-derived fixture with points on
voxel faces, on the upper edge and non-finite; an O(n^2) brute-force grouping
on tiny clouds; and containment/bijection invariants on a full frame.
"""

import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from synth.workloads import Workspace

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _pts(raw):
    return np.array([[float(v) for v in p] for p in raw], dtype=np.float32)


def test_golden_tiny_frame():
    g = _load("filter_tiny.json")
    ws = Workspace(lo=tuple(g["lo"]), voxel=g["voxel"], dims=tuple(g["dims"]))
    out = oracle.filter_cloud(_pts(g["points"]), np.array(g["T"], np.float32), ws)
    e = g["expected_min_pts_1"]
    assert out["n"] == len(e["keys"])
    for k in ("keys", "counts", "rep_idx"):
        assert out[k].tolist() == e[k], k
    for k in ("x", "y", "z"):
        assert out[k].tolist() == e[k], k
    ws2 = Workspace(lo=tuple(g["lo"]), voxel=g["voxel"], dims=tuple(g["dims"]), min_pts=2)
    out2 = oracle.filter_cloud(_pts(g["points"]), np.array(g["T"], np.float32), ws2)
    e2 = g["expected_min_pts_2"]
    for k in ("keys", "counts", "rep_idx"):
        assert out2[k].tolist() == e2[k], k


def _brute_force(xyz, T, ws):
    """O(n^2) grouping: two kept points share a voxel iff their integer voxel
    indices agree; each group's count and smallest index."""
    f = np.float32
    T = T.reshape(3, 4)
    idx = []
    for i, p in enumerate(xyz):
        if not np.all(np.isfinite(p)):
            idx.append(None)
            continue
        cell = []
        for a in range(3):
            w = ((f(T[a, 0]) * p[0] + f(T[a, 1]) * p[1]) + f(T[a, 2]) * p[2]) + f(T[a, 3])
            q = (f(w) - f(ws.lo[a])) / f(ws.voxel)
            if not (q >= 0 and q < ws.dims[a]):
                cell = None
                break
            cell.append(int(math.floor(q)))
        idx.append(tuple(cell) if cell is not None else None)
    groups = []
    seen = [False] * len(xyz)
    for i in range(len(xyz)):
        if idx[i] is None or seen[i]:
            continue
        members = [j for j in range(len(xyz)) if idx[j] == idx[i]]
        for j in members:
            seen[j] = True
        ix, iy, iz = idx[i]
        key = (iz * ws.dims[1] + iy) * ws.dims[0] + ix
        groups.append((key, len(members), min(members)))
    groups.sort()
    return groups


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_tiny_clouds(seed):
    g = np.random.Generator(np.random.PCG64(seed))
    n = int(g.integers(1, 65))
    # points clustered in a few voxels so that groups have several members
    centres = g.uniform(0.0, 0.4, size=(4, 3))
    xyz = (centres[g.integers(0, 4, n)] + g.normal(0, 0.01, (n, 3))).astype(np.float32)
    xyz[g.random(n) < 0.1] = np.nan
    ang = g.uniform(0, 2 * np.pi)
    R = np.array([[np.cos(ang), -np.sin(ang), 0], [np.sin(ang), np.cos(ang), 0], [0, 0, 1]])
    T = np.concatenate([R, g.uniform(-0.1, 0.3, (3, 1))], axis=1).reshape(-1).astype(np.float32)
    ws = Workspace(lo=(-0.2, -0.2, -0.1), voxel=float(np.float32(0.02)), dims=(40, 40, 30))
    out = oracle.filter_cloud(xyz, T, ws)
    bf = _brute_force(xyz, T, ws)
    assert out["n"] == len(bf)
    assert [(int(k), int(c), int(r)) for k, c, r in zip(out["keys"], out["counts"], out["rep_idx"])] == bf


def test_full_frame_invariants():
    w = synth.tabletop_workload(n_agents=1, n_steps=1)
    xyz, T, ws = w["xyz"], w["T"], w["workspace"]
    out = oracle.filter_cloud(xyz, T, ws)
    n = out["n"]
    assert 20000 < n < 120000
    keys = out["keys"].astype(np.int64)
    assert np.all(np.diff(keys) > 0), "keys strictly ascending (unique)"
    # every representative point lies inside its voxel (float64 check with slack)
    Tm = T.reshape(3, 4).astype(np.float64)
    rep = xyz[out["rep_idx"]].astype(np.float64)
    wpt = rep @ Tm[:, :3].T + Tm[:, 3]
    ctr = np.stack([out["x"], out["y"], out["z"]], axis=1).astype(np.float64)
    assert np.all(np.abs(wpt - ctr) <= ws.voxel / 2 + 1e-6)
    # bijection: the counts add up to the number of points inside the workspace
    allw = xyz.astype(np.float64) @ Tm[:, :3].T + Tm[:, 3]
    lo = np.array(ws.lo)
    hi = lo + np.array(ws.dims) * ws.voxel
    finite = np.all(np.isfinite(xyz), axis=1)
    inside = finite & np.all((allw >= lo) & (allw < hi), axis=1)
    # float64 and the binary32 sequence may disagree only for points within
    # rounding of a workspace face
    near = finite & np.any((np.abs(allw - lo) < 1e-6) | (np.abs(allw - hi) < 1e-6), axis=1)
    assert abs(int(out["counts"].sum()) - int(inside.sum())) <= int(near.sum())
    # the centre of key k is the centre of its (ix, iy, iz) cell
    nx, ny = ws.dims[0], ws.dims[1]
    ix, iy, iz = keys % nx, (keys // nx) % ny, keys // (nx * ny)
    assert np.allclose(ctr[:, 0], ws.lo[0] + (ix + 0.5) * ws.voxel, atol=1e-6)
    assert np.allclose(ctr[:, 1], ws.lo[1] + (iy + 0.5) * ws.voxel, atol=1e-6)
    assert np.allclose(ctr[:, 2], ws.lo[2] + (iz + 0.5) * ws.voxel, atol=1e-6)


def test_capacity_reports_needed_size():
    w = synth.sphere_workload()
    full = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    part = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"], cap=100)
    assert part["n"] == full["n"]
    assert part["keys"].tolist() == full["keys"][:100].tolist()


def test_empty_and_all_rejected():
    ws = Workspace(lo=(0, 0, 0), voxel=0.1, dims=(10, 10, 10))
    T = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32)
    assert oracle.filter_cloud(np.zeros((0, 3), np.float32), T, ws)["n"] == 0
    far = np.full((50, 3), 5.0, np.float32)
    assert oracle.filter_cloud(far, T, ws)["n"] == 0


# ---- several sensors fused into one obstacle set (Sec. IV-B) --------------

def _ws_small():
    return synth.Workspace(lo=(0.0, -0.5, -0.02), voxel=0.01, dims=(100, 100, 80))


def test_fusion_of_one_sensor_is_the_single_filter():
    m = synth.multi_sensor_frames(n_sensors=1, n_points=20000)
    xyz, T = m["clouds"][0]
    a = oracle.filter_clouds(m["clouds"], _ws_small())
    b = oracle.filter_cloud(xyz, T, _ws_small())
    for k in ("keys", "counts", "rep_idx", "x", "y", "z"):
        assert np.array_equal(a[k], b[k]), k


def test_fusion_with_identity_transforms_is_the_concatenated_cloud():
    g = np.random.Generator(np.random.PCG64(4))
    c1 = g.uniform([0, -0.5, 0], [1, 0.5, 0.8], (3001, 3)).astype(np.float32)
    c2 = g.uniform([0.2, -0.2, 0], [0.6, 0.3, 0.5], (1999, 3)).astype(np.float32)
    I = synth.workloads.IDENTITY_T
    a = oracle.filter_clouds([(c1, I), (c2, I)], _ws_small())
    b = oracle.filter_cloud(np.concatenate([c1, c2]), I, _ws_small())
    for k in ("keys", "counts", "rep_idx", "x", "y", "z"):
        assert np.array_equal(a[k], b[k]), k


def test_fusion_is_the_union_with_summed_counts_and_global_indices():
    m = synth.multi_sensor_frames(n_sensors=3, n_points=30000)
    ws = _ws_small()
    fused = oracle.filter_clouds(m["clouds"], ws)
    singles = [oracle.filter_cloud(x, T, ws) for x, T in m["clouds"]]
    offsets = np.cumsum([0] + [x.shape[0] for x, _ in m["clouds"]])[:-1]
    count, rep = {}, {}
    for s, f in enumerate(singles):
        for k, c, r in zip(f["keys"], f["counts"], f["rep_idx"]):
            count[int(k)] = count.get(int(k), 0) + int(c)
            rep[int(k)] = min(rep.get(int(k), 1 << 40), int(r) + int(offsets[s]))
    keys = np.array(sorted(count), dtype=np.uint32)
    assert np.array_equal(fused["keys"], keys)
    assert np.array_equal(fused["counts"], np.array([count[int(k)] for k in keys], np.uint32))
    assert np.array_equal(fused["rep_idx"], np.array([rep[int(k)] for k in keys], np.uint32))
    assert len(set(singles[0]["keys"].tolist()) & set(singles[1]["keys"].tolist())) > 100
