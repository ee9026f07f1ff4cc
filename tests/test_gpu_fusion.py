"""GPU filter_clouds vs the oracle: several depth sensors fused into one
obstacle set (Sec. IV-B), bit-exact keys, counts, smallest global indices
and voxel centres -- two 848x480 cameras at full frame size, three cameras
with ragged cloud sizes and an empty one, eleven sensors (two fused launch
groups), min_pts > 1, one sensor equal to filter_cloud, repeats, invalid
arguments."""

import dataclasses

import numpy as np
import pytest

import oracle
import synth

from _helpers import u32, f32_bits

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2606_12579_b300 as gm
    gm.context()
    return gm


def _dev(clouds):
    import torch
    return [(torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda(), T) for x, T in clouds]


def _assert_same(obs, ref):
    n = obs.count()
    assert n == ref["n"]
    k = min(n, obs.cap)
    assert np.array_equal(u32(obs.keys[:k]), ref["keys"][:k])
    assert np.array_equal(u32(obs.counts[:k]), ref["counts"][:k])
    assert np.array_equal(u32(obs.rep_idx[:k]), ref["rep_idx"][:k])
    for a in ("x", "y", "z"):
        assert np.array_equal(f32_bits(getattr(obs, a)[:k]), ref[a][:k].view(np.uint32)), a


def test_two_full_frames_bit_exact(gm):
    m = synth.multi_sensor_frames(n_sensors=2)
    assert all(x.shape[0] == 848 * 480 for x, _ in m["clouds"])
    ref = oracle.filter_clouds(m["clouds"], m["workspace"])
    obs = gm.filter_clouds(_dev(m["clouds"]), m["workspace"], cap=200000)
    gm.sync()
    _assert_same(obs, ref)
    assert ref["n"] > 50000


@pytest.mark.parametrize("voxel", [0.005, 0.01])
def test_three_ragged_clouds_and_an_empty_one(gm, voxel):
    m = synth.multi_sensor_frames(n_sensors=3, n_points=20001)
    clouds = [m["clouds"][0], (m["clouds"][1][0][:15003], m["clouds"][1][1]),
              (np.zeros((0, 3), np.float32), m["clouds"][2][1]),
              (m["clouds"][2][0][:7], m["clouds"][2][1])]
    dims = tuple(int(round(e / voxel)) for e in (1.0, 1.0, 0.8))
    ws = dataclasses.replace(m["workspace"], voxel=voxel, dims=dims)
    ref = oracle.filter_clouds(clouds, ws)
    obs = gm.filter_clouds(_dev(clouds), ws, cap=60000)
    gm.sync()
    _assert_same(obs, ref)


def test_eleven_sensors_two_launch_groups(gm):
    """More sensors than one fused key launch takes (8): eleven ragged
    clouds (one empty) go through two key and two count launches; the index
    bases run across both groups."""
    m = synth.multi_sensor_frames(n_sensors=3, n_points=9001)
    sizes = [9001, 17, 4096, 0, 333, 9000, 1, 2048, 5555, 8191, 64]
    clouds = [(m["clouds"][i % 3][0][:n], m["clouds"][i % 3][1]) for i, n in enumerate(sizes)]
    ref = oracle.filter_clouds(clouds, m["workspace"])
    obs = gm.filter_clouds(_dev(clouds), m["workspace"], cap=60000)
    gm.sync()
    _assert_same(obs, ref)


def test_min_pts_fused(gm):
    m = synth.multi_sensor_frames(n_sensors=2, n_points=50001)
    ws = dataclasses.replace(m["workspace"], min_pts=3)
    ref = oracle.filter_clouds(m["clouds"], ws)
    obs = gm.filter_clouds(_dev(m["clouds"]), ws, cap=60000)
    gm.sync()
    _assert_same(obs, ref)


def test_one_sensor_is_filter_cloud_and_repeats_are_identical(gm):
    m = synth.multi_sensor_frames(n_sensors=1, n_points=30003)
    dev = _dev(m["clouds"])
    a = gm.filter_clouds(dev, m["workspace"], cap=40000)
    b = gm.filter_cloud(dev[0][0], m["clouds"][0][1], m["workspace"], cap=40000)
    c = gm.filter_clouds(dev, m["workspace"], cap=40000)
    gm.sync()
    n = a.count()
    assert n == b.count() == c.count()
    for o in (b, c):
        for f in ("keys", "counts", "rep_idx", "x", "y", "z"):
            assert np.array_equal(getattr(a, f)[:n].cpu().numpy(), getattr(o, f)[:n].cpu().numpy())


def test_fused_invalid_arguments(gm):
    import torch
    m = synth.multi_sensor_frames(n_sensors=2, n_points=1000)
    dev = _dev(m["clouds"])
    with pytest.raises(gm.GmappError) as e:
        gm.filter_clouds([], m["workspace"], cap=100)
    assert e.value.status == 1
    bad = torch.empty(1001 * 3 + 1, dtype=torch.float32, device="cuda")[1:].view(1001, 3)
    with pytest.raises(gm.GmappError) as e:   # not 16-byte aligned
        gm.filter_clouds([dev[0], (bad, m["clouds"][1][1])], m["workspace"], cap=100)
    assert e.value.status == 1
    nan_T = list(m["clouds"][1][1])
    nan_T[3] = float("nan")
    with pytest.raises(gm.GmappError) as e:
        gm.filter_clouds([dev[0], (dev[1][0], nan_T)], m["workspace"], cap=100)
    assert e.value.status == 1
