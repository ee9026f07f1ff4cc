"""GPU filter_cloud vs the oracle: bit-exact keys, counts, smallest indices
and voxel centres (Sec. IV-B, Sec. V-A), at full frame sizes and on the edge
cases (empty, all rejected, ragged sizes, faces and upper edge, capacity
overflow, min_pts > 1), plus run-to-run determinism."""

import json
import os

import numpy as np
import pytest

import oracle
import synth
from synth.workloads import Workspace

from _helpers import u32, f32_bits

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def gm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2606_12579_b300 as gm
    gm.context()
    return gm


def _run(gm, xyz, T, ws, cap=None):
    import torch
    x = torch.from_numpy(np.ascontiguousarray(xyz, dtype=np.float32)).cuda()
    return gm.filter_cloud(x, T, ws, cap=cap if cap is not None else max(4, xyz.shape[0]))


def _assert_same(obs, ref):
    n = obs.count()
    assert n == ref["n"]
    k = min(n, obs.cap)
    assert np.array_equal(u32(obs.keys[:k]), ref["keys"][:k])
    assert np.array_equal(u32(obs.counts[:k]), ref["counts"][:k])
    assert np.array_equal(u32(obs.rep_idx[:k]), ref["rep_idx"][:k])
    for a in ("x", "y", "z"):
        assert np.array_equal(f32_bits(getattr(obs, a)[:k]), ref[a][:k].view(np.uint32)), a


@pytest.mark.parametrize("which", ["sphere", "tabletop", "tabletop_200k_1cm"])
def test_full_frames_bit_exact(gm, which):
    if which == "sphere":
        w = synth.sphere_workload()
    elif which == "tabletop":
        w = synth.tabletop_workload(n_agents=1, n_steps=1)
    else:
        w = synth.tabletop_workload(n_agents=1, n_steps=1, n_points=200000, voxel=0.01,
                                    spheres_at=0.37, sphere_seed=5)
    ref = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    obs = _run(gm, w["xyz"], w["T"], w["workspace"])
    gm.sync()
    _assert_same(obs, ref)
    assert obs.r_O == pytest.approx(w["workspace"].voxel / 2)


def test_golden_tiny_frame(gm):
    g = json.load(open(os.path.join(GOLD, "filter_tiny.json")))
    xyz = np.array([[float(v) for v in p] for p in g["points"]], np.float32)
    for mp, key in ((1, "expected_min_pts_1"), (2, "expected_min_pts_2")):
        ws = Workspace(lo=tuple(g["lo"]), voxel=g["voxel"], dims=tuple(g["dims"]), min_pts=mp)
        obs = _run(gm, xyz, np.array(g["T"], np.float32), ws)
        gm.sync()
        e = g[key]
        n = obs.count()
        assert n == len(e["keys"])
        assert u32(obs.keys[:n]).tolist() == e["keys"]
        assert u32(obs.counts[:n]).tolist() == e["counts"]
        assert u32(obs.rep_idx[:n]).tolist() == e["rep_idx"]


@pytest.mark.parametrize("seed", range(8))
def test_random_small_clouds_ragged(gm, seed):
    """Clusters of points (many per voxel), NaN rows, a random rigid
    transform, and sizes that are not multiples of 4 or of a block."""
    g = np.random.Generator(np.random.PCG64(100 + seed))
    n = int(g.integers(1, 5000)) * 4 + int(g.integers(0, 4))
    centres = g.uniform(0.0, 0.4, size=(16, 3))
    xyz = (centres[g.integers(0, 16, n)] + g.normal(0, 0.02, (n, 3))).astype(np.float32)
    xyz[g.random(n) < 0.05] = np.nan
    xyz[g.random(n) < 0.01, 1] = np.inf
    ang = g.uniform(0, 2 * np.pi)
    R = np.array([[np.cos(ang), 0, np.sin(ang)], [0, 1, 0], [-np.sin(ang), 0, np.cos(ang)]])
    T = np.concatenate([R, g.uniform(-0.1, 0.3, (3, 1))], axis=1).reshape(-1).astype(np.float32)
    ws = Workspace(lo=(-0.3, -0.2, -0.4), voxel=float(g.uniform(0.005, 0.03)),
                   dims=(int(g.integers(20, 90)), int(g.integers(20, 90)), int(g.integers(20, 90))),
                   min_pts=int(g.integers(1, 4)))
    ref = oracle.filter_cloud(xyz, T, ws)
    obs = _run(gm, xyz, T, ws)
    gm.sync()
    _assert_same(obs, ref)


def test_empty_and_all_rejected(gm):
    ws = Workspace(lo=(0, 0, 0), voxel=0.1, dims=(10, 10, 10))
    T = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32)
    for xyz in (np.zeros((0, 3), np.float32), np.full((37, 3), 5.0, np.float32),
                np.full((9, 3), np.nan, np.float32)):
        obs = _run(gm, xyz, T, ws)
        gm.sync()
        assert obs.count() == 0


def test_capacity_overflow_reports_total(gm):
    w = synth.sphere_workload()
    ref = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    obs = _run(gm, w["xyz"], w["T"], w["workspace"], cap=256)
    with pytest.raises(gm.GmappError) as e:
        gm.sync()
    assert e.value.status == 2  # GMAPP_ERR_CAPACITY
    assert obs.count() == ref["n"]
    assert np.array_equal(u32(obs.keys[:256]), ref["keys"][:256])
    assert np.array_equal(u32(obs.counts[:256]), ref["counts"][:256])
    gm.sync()  # the error word was cleared


def test_large_grid_and_max_dims(gm):
    """A grid near the 2^32-cell limit (bitmap of 256 MB) with a ragged cloud."""
    g = np.random.Generator(np.random.PCG64(7))
    xyz = g.uniform(-1, 1, (100003, 3)).astype(np.float32)
    ws = Workspace(lo=(-1.0, -1.0, -1.0), voxel=float(np.float32(2.0 / 1600)), dims=(1600, 1600, 1600))
    ref = oracle.filter_cloud(xyz, np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32), ws)
    obs = _run(gm, xyz, np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32), ws)
    gm.sync()
    _assert_same(obs, ref)


def test_invalid_arguments_rejected_on_host(gm):
    import torch
    x = torch.zeros(12, 3, device="cuda")
    T = [1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0]
    for ws in (Workspace(lo=(0, 0, 0), voxel=0.0, dims=(4, 4, 4)),
               Workspace(lo=(0, 0, 0), voxel=0.1, dims=(0, 4, 4)),
               Workspace(lo=(0, 0, 0), voxel=0.1, dims=(4096, 4096, 4096)),
               Workspace(lo=(0, 0, 0), voxel=0.1, dims=(4, 4, 4), min_pts=0)):
        with pytest.raises(gm.GmappError) as e:
            gm.filter_cloud(x, T, ws)
        assert e.value.status == 1
    with pytest.raises(gm.GmappError):
        gm.filter_cloud(x, [1, 0, 0, float("nan"), 0, 1, 0, 0, 0, 0, 1, 0],
                        Workspace(lo=(0, 0, 0), voxel=0.1, dims=(4, 4, 4)))
    with pytest.raises(gm.GmappError):
        gm.filter_cloud(x[1:], T, Workspace(lo=(0, 0, 0), voxel=0.1, dims=(4, 4, 4)))  # misaligned


def test_repeat_determinism(gm):
    w = synth.tabletop_workload(n_agents=1, n_steps=1)
    a = _run(gm, w["xyz"], w["T"], w["workspace"])
    b = _run(gm, w["xyz"], w["T"], w["workspace"])
    gm.sync()
    n = a.count()
    assert n == b.count()
    for f in ("keys", "counts", "rep_idx", "x", "y", "z"):
        assert np.array_equal(getattr(a, f)[:n].cpu().numpy(), getattr(b, f)[:n].cpu().numpy())


def test_batched_filter_matches_filter_cloud_and_oracle(gm):
    """filter_cloud_batch over uneven clouds (a full tabletop frame, a sphere
    cloud on its own grid, a ragged tiny cloud, an empty one, one that
    overflows its capacity, points scattered over the whole grid so that a
    warp's 256 points touch more bitmap words than its word table holds, and
    20,003 points in one voxel, one long run of equal keys) gives each job
    the result of filter_cloud on the same cloud, bit for bit, and the
    oracle's; a second run repeats it."""
    import torch
    tab = synth.tabletop_workload(n_agents=1, n_steps=1)
    sph = synth.sphere_workload()
    g = np.random.Generator(np.random.PCG64(17))
    tiny = g.uniform(-0.05, 1.05, (13, 3)).astype(np.float32)
    empty = np.zeros((0, 3), np.float32)
    ws_t = tab["workspace"]
    I = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32)
    lo, hi = np.asarray(ws_t.lo, np.float64), np.asarray(ws_t.lo, np.float64) + \
        np.asarray(ws_t.dims, np.float64) * ws_t.voxel
    scattered = g.uniform(lo, hi, (50000, 3)).astype(np.float32)
    centre = lo + (np.array([17, 33, 9]) + 0.5) * ws_t.voxel
    one_voxel = (centre + g.uniform(-0.4, 0.4, (20003, 3)) * ws_t.voxel).astype(np.float32)
    jobs = [(tab["xyz"], tab["T"], tab["workspace"], None),
            (sph["xyz"], sph["T"], sph["workspace"], None),
            (tiny, tab["T"], tab["workspace"], None),
            (empty, tab["T"], tab["workspace"], None),
            (tab["xyz"], tab["T"], tab["workspace"], 1000),
            (scattered, I, ws_t, None),
            (one_voxel, I, ws_t, None)]
    clouds = [torch.from_numpy(np.ascontiguousarray(x)).cuda() if x.shape[0] else
              torch.empty(0, 3, device="cuda") for x, _, _, _ in jobs]
    caps = [c if c is not None else max(4, (x.shape[0] + 3) // 4 * 4) for x, _, _, c in jobs]
    fb = gm.FilterBatch(clouds, [j[1] for j in jobs], [j[2] for j in jobs], caps=caps)
    for rep in range(2):
        fb.run()
        with pytest.raises(gm.GmappError) as e:
            gm.sync()               # job 4 overflows its capacity of 1000
        assert e.value.status == 2
        for q, (x, T, ws, cap) in enumerate(jobs):
            ref = oracle.filter_cloud(x, T, ws)
            _assert_same(fb.outs[q], ref)
            if x.shape[0] and cap is None:
                single = _run(gm, x, T, ws, cap=caps[q])
                gm.sync()
                for a in ("x", "y", "z", "keys", "counts", "rep_idx"):
                    n = single.count()
                    assert torch.equal(getattr(single, a)[:n], getattr(fb.outs[q], a)[:n])


def test_voxel_faces_stress_bit_exact(gm):
    """Quotients (w - lo) / voxel at and around every integer of the grid:
    points within +-8 ulp of each voxel face along x (and the faces of the
    upper edge), plus random offsets; the GPU's voxel quotient must decide
    floor and crop exactly as the IEEE quotient of the oracle."""
    ws = Workspace(lo=(0.0, -0.5, 0.0), voxel=0.0043, dims=(232, 232, 186))
    v = np.float32(ws.voxel)
    k = np.arange(0, 233, dtype=np.float32)
    face = (k * v).astype(np.float32)
    steps = np.arange(-8, 9)
    x = np.concatenate([np.nextafter(face, np.float32(np.inf) if s > 0 else np.float32(-np.inf))
                        if s else face for s in [0]] +
                       [face + s * np.spacing(face) for s in steps])
    g = np.random.Generator(np.random.PCG64(8))
    x = np.concatenate([x, g.uniform(-0.01, 1.01, 200000).astype(np.float32)]).astype(np.float32)
    n = x.size
    y = np.full(n, np.float32(0.5 * v) - np.float32(0.5), np.float32)     # a cell centre in y
    z = g.uniform(0.0, 0.79, n).astype(np.float32)
    pts = np.stack([x, y, z], axis=1).astype(np.float32)
    I = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32)
    # also through a rotation: the transform's products and sums feed the quotient
    c, s = np.float32(np.cos(0.3)), np.float32(np.sin(0.3))
    Rz = np.array([c, -s, 0, 0.2, s, c, 0, -0.1, 0, 0, 1, 0.05], np.float32)
    for T in (I, Rz):
        ref = oracle.filter_cloud(pts, T, ws)
        obs = _run(gm, pts, T, ws)
        gm.sync()
        _assert_same(obs, ref)


def test_batched_filter_many_waves_matches_filter_cloud(gm):
    """40 tabletop frames: more than one L2-sized wave (about 15 tabletop
    frames), so the batch deals its waves round-robin to its streams and
    reuses each stream's scratch slots.  Every job's S_W equals filter_cloud's bit for bit,
    on two runs in a row and through a CUDA-graph replay."""
    import torch
    base = [synth.tabletop_workload(frame_seed=9_100_000 + f, n_agents=1, n_steps=1)
            for f in range(4)]
    g = np.random.Generator(np.random.PCG64(23))
    frames = []
    for i in range(40):
        x = base[i % 4]["xyz"]
        frames.append((x + g.normal(0.0, 1e-3, x.shape)).astype(np.float32))
    T, ws = base[0]["T"], base[0]["workspace"]
    clouds = [torch.from_numpy(f).cuda() for f in frames]
    fb = gm.FilterBatch(clouds, T, ws, caps=[131072] * len(clouds))
    ref = []
    for c in clouds:
        o = _run(gm, c.cpu().numpy(), T, ws, cap=131072)
        gm.sync()
        n = o.count()
        ref.append({f: getattr(o, f)[:n].clone() for f in ("x", "y", "z", "keys", "counts",
                                                            "rep_idx")})
    def check():
        for q, r in enumerate(ref):
            n = fb.outs[q].count()
            assert n == r["keys"].numel(), q
            for f, t in r.items():
                assert torch.equal(getattr(fb.outs[q], f)[:n], t), (q, f)
    for _ in range(2):
        fb.run()
        gm.sync()
        check()
    for o in fb.outs:
        o.counts.fill_(7)
        o.x.fill_(-1.0)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        fb.run(stream=s)
    graph.replay()
    torch.cuda.synchronize()
    gm.sync()
    check()
    # the first frame against the oracle as well
    _assert_same(fb.outs[0], oracle.filter_cloud(frames[0], T, ws))


def test_batched_filter_mixed_jobs_reuse_slots(gm):
    """45 jobs of four kinds in turn (a tabletop frame on its 200x200x160 grid,
    a sphere cloud on its 100x100x80 grid, a ragged 13-point cloud, an empty
    one): three waves, so the third reuses the first wave's scratch slots
    with jobs of other sizes and grids.  Every job equals filter_cloud bit for
    bit on two runs in a row."""
    import torch
    tab = synth.tabletop_workload(n_agents=1, n_steps=1)
    sph = synth.sphere_workload()
    g = np.random.Generator(np.random.PCG64(29))
    kinds = [(tab["xyz"], tab["T"], tab["workspace"]), (sph["xyz"], sph["T"], sph["workspace"]),
             (g.uniform(-0.05, 1.05, (13, 3)).astype(np.float32), tab["T"], tab["workspace"]),
             (np.zeros((0, 3), np.float32), tab["T"], tab["workspace"])]
    jobs = []
    for q in range(45):
        x, T, ws = kinds[q % 4]
        if x.shape[0] > 100:
            x = (x + g.normal(0.0, 1e-3, x.shape)).astype(np.float32)
        jobs.append((x, T, ws))
    clouds = [torch.from_numpy(np.ascontiguousarray(x)).cuda() if x.shape[0] else
              torch.empty(0, 3, device="cuda") for x, _, _ in jobs]
    caps = [max(4, (x.shape[0] + 3) // 4 * 4) for x, _, _ in jobs]
    fb = gm.FilterBatch(clouds, [j[1] for j in jobs], [j[2] for j in jobs], caps=caps)
    refs = []
    for (x, T, ws), cap in zip(jobs, caps):
        if x.shape[0]:
            o = _run(gm, x, T, ws, cap=cap)
            gm.sync()
            n = o.count()
            refs.append({f: getattr(o, f)[:n].clone() for f in ("x", "y", "z", "keys", "counts",
                                                                "rep_idx")})
        else:
            refs.append(None)
    for _ in range(2):
        fb.run()
        gm.sync()
        for q, r in enumerate(refs):
            n = fb.outs[q].count()
            if r is None:
                assert n == 0, q
                continue
            assert n == r["keys"].numel(), q
            for f, t in r.items():
                assert torch.equal(getattr(fb.outs[q], f)[:n], t), (q, f)
