"""The served stream's frame renderer (synth.stream_frames, torch, any
device) casts the same rays as synth.render_depth_frame (numpy): with the
noise and dropouts off, every pixel's point agrees; with them on, the frames
have the recipe's pixel count, dropout rate and depth noise."""

import numpy as np
import pytest

import synth
from synth.scenes import moving_spheres, render_depth_frame, tabletop_scene
from synth.stream_frames import StreamFrames


@pytest.mark.parametrize("t", [0.0, 0.37, 2.5])
def test_exact_frames_match_the_numpy_ray_caster(t):
    r = StreamFrames(seed=1005, device="cpu")
    got = r.render([t], first=0, noise=False)[0].numpy()
    scene = tabletop_scene(1005)
    scene.spheres = moving_spheres(1005)(t)
    want, T = render_depth_frame(scene, seed=1, depth_noise=0.0, nan_frac=0.0)
    assert np.array_equal(T, r.T)
    assert got.shape == want.shape
    fin = np.isfinite(want[:, 2])
    assert np.array_equal(np.isfinite(got[:, 2]), fin)
    assert np.allclose(got[fin], want[fin], rtol=1e-6, atol=1e-7)
    # the spheres are in view: some pixels see them, nearer than the static scene
    bare, _ = render_depth_frame(tabletop_scene(1005), seed=1, depth_noise=0.0, nan_frac=0.0)
    nearer = fin & np.isfinite(bare[:, 2]) & (got[:, 2] < bare[:, 2] - 1e-4)
    assert nearer.sum() > 1000


def test_noisy_frames_follow_the_recipe():
    r = StreamFrames(seed=1005, n_points=200000, device="cpu")
    arrivals, _, _ = synth.serve_stream(n_requests=10000)
    f = r.render(arrivals[:3], first=0).numpy()
    assert f.shape == (3, 200000, 3) and f.dtype == np.float32
    nan = np.isnan(f[..., 2]).mean()
    assert 0.04 < nan < 0.07
    # depth noise along the ray: the rendered depth minus the exact one
    exact = r.render(arrivals[:1], first=0, noise=False)[0].numpy()
    assert not np.array_equal(f[0], f[1])
    # frames are reproducible for a given chunk
    g = r.render(arrivals[:3], first=0).numpy()
    assert np.array_equal(np.nan_to_num(f), np.nan_to_num(g))
    assert np.isfinite(exact[:, 2]).mean() > 0.9
