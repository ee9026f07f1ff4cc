"""GPU rollout_ensemble vs the oracle: a heterogeneous ensemble of APF
(Eq. apf) and MFI (Eq. mfi) agents in one launch (Sec. IV-A heuristics and
"Other Heuristics": agents per heuristic with large and small detection
radii; agents grouped by heuristic, Sec. IV-D).

  * APF per-force parity at fixed oracle states.  Each APF term is computed
    in FP32 from rsqrt.approx (relative error <= 2^-22.9), a clamp, the
    difference 1/rho - 1/r_d and three products, so its absolute error is at
    most about 6e-7 rho^-3; the FP32 sums add a few ulp of the largest
    partial sums.  The bound is therefore
        |f_gpu - f_ref| <= 1e-5 |f_ref| + 4e-6 k_f sum_j rho_j^-3
                           + (gate-ambiguous pairs) k_f (r_d + R)^-3,
    the middle term matters only where the terms of the vector sum cancel;
  * ensemble rollout parity: every trajectory point within 1e-3 m of the
    FP64 oracle after N_k steps, for both exchanges, with and without the
    clearance reduction, odd shard lengths (padding), all-APF, one-APF and
    no-gate ensembles, and the full tabletop ensemble (256 agents, half APF)
    in the library's launch shape with a sample checked against the oracle;
  * n_apf = 0 is rollout_agents bit for bit; repeats are bit-identical;
    invalid arguments are refused on the host.
"""

import dataclasses

import numpy as np
import pytest

import oracle
import synth

from _helpers import to_dev_agents, subset_agents, gate_allowance

pytestmark = pytest.mark.gpu
POS_TOL = 1e-3     # m, after N_k steps
FORCE_TOL = 1e-5   # relative, per force vector


@pytest.fixture(scope="module")
def gm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2606_12579_b300 as gm
    gm.context()
    return gm


def _filtered(w):
    ref = oracle.filter_cloud(w["xyz"], w["T"], w["workspace"])
    return np.stack([ref["x"], ref["y"], ref["z"]]), ref["r_O"]


def _gpu_obstacles(gm, obs, r_O, cap=None):
    import torch
    return gm.Obstacles.from_points(torch.from_numpy(np.ascontiguousarray(obs, np.float32)), r_O,
                                    cap=cap)


def _compare(gpu, ref, idx=None, clear=True):
    sel = (lambda a: a[idx]) if idx is not None else (lambda a: a)
    traj = sel(gpu["traj"].cpu().numpy().astype(np.float64))
    err = np.abs(traj - ref["traj"]).max()
    assert err <= POS_TOL, f"trajectory error {err:.3e} m"
    pf = gpu["p_final"].cpu().numpy()
    pf = pf[:, idx] if idx is not None else pf
    assert np.abs(pf - ref["p_final"]).max() <= POS_TOL
    assert np.abs(sel(gpu["path_len"].cpu().numpy()) - ref["path_len"]).max() <= POS_TOL
    if clear:
        mc = sel(gpu["min_clear"].cpu().numpy())
        fin = np.isfinite(ref["min_clear"])
        assert np.array_equal(np.isfinite(mc), fin)
        assert np.abs(mc[fin] - ref["min_clear"][fin]).max(initial=0) <= POS_TOL
    return err


def _sphere_ensemble(n_agents=12, n_apf=6, n_steps=200):
    w = synth.sphere_workload(n_agents=n_agents, n_steps=n_steps)
    w["agents"] = synth.ensemble_agents(w["agents"], n_apf)
    return w


def _rho_cube_sum(obs64, P, R, r_d, eps):
    """Per agent: sum of rho_j^-3 over the pairs inside (or within rounding
    of) the APF gate -- the scale of the FP32 error of the vector sum."""
    out = np.zeros(P.shape[1])
    for i in range(P.shape[1]):
        d = np.sqrt(((obs64 - P[:, i:i + 1]) ** 2).sum(axis=0))
        rho = np.maximum(d, R[i] + eps)
        near = d - R[i] < r_d[i] * (1 + 4e-7) + 1e-7
        out[i] = (rho[near] ** -3.0).sum()
    return out


def test_apf_force_parity_at_oracle_states(gm):
    """f_r of APF agents evaluated once (N_k = 1) at states taken from the
    oracle's ensemble trajectories near the sphere."""
    w = _sphere_ensemble(n_agents=12, n_apf=12)
    obs, r_O = _filtered(w)
    prm = w["params"]
    ref = oracle.rollout(obs, r_O, w["agents"], prm, n_apf=12)
    na = 12
    ps, vs, cols = [], [], []
    for k in (1, 40, 80, 110, 140, 170, 199):
        ps.append(ref["traj"][:, k].T)
        vs.append((ref["traj"][:, k] - ref["traj"][:, k - 1]).T / prm.dt)
        cols.append(np.arange(na))
    P = np.concatenate(ps, axis=1).astype(np.float32)
    V = np.concatenate(vs, axis=1).astype(np.float32)
    ag = subset_agents(w["agents"], np.concatenate(cols))
    ag["p0"], ag["v0"] = np.ascontiguousarray(P), np.ascontiguousarray(V)
    n = P.shape[1]
    one = dataclasses.replace(prm, n_steps=1)
    out = gm.rollout_ensemble(_gpu_obstacles(gm, obs, r_O), to_dev_agents(ag), n, one,
                              want_trace=True)
    gm.sync()
    f_gpu = out["f_trace"][:, 0, :].cpu().numpy().T.astype(np.float64)
    P64 = P.astype(np.float64)
    r = oracle.apf_eval(obs, r_O, P64, ag, prm.rho, prm.eps)
    R = ag["r_a"].astype(np.float64) + r_O
    r_d = ag["r_d"].astype(np.float64)
    kf = prm.rho * ag["k_r"].astype(np.float64)
    obs64 = obs.astype(np.float64)
    amb = gate_allowance(obs64, P64, R, r_d)
    scale = _rho_cube_sum(obs64, P64, R, r_d, prm.eps)
    fn = np.linalg.norm(r["f_r"], axis=0)
    err = np.linalg.norm(f_gpu - r["f_r"], axis=0)
    tol = FORCE_TOL * fn + 4e-6 * kf * scale + amb * kf * (r_d + R) ** -3.0
    assert (fn > 0).sum() >= 20, "the states must be inside the detection radius"
    assert np.all(err <= tol), (err / np.maximum(fn, 1e-30)).max()
    # where the terms do not cancel much, the plain 1e-5 relative bound holds
    plain = r["f_abs"] <= 2.0 * fn
    active = fn > 0
    print(f"APF force parity: {int(active.sum())} states with a force, "
          f"{int((plain & active).sum())} of them checked at the plain 1e-5 relative bound")
    assert (plain & active).sum() >= 10
    assert np.all(err[plain] <= FORCE_TOL * fn[plain] + amb[plain] * kf[plain] *
                  (r_d[plain] + R[plain]) ** -3.0)
    w_gpu = out["w_trace"][:, 0].cpu().numpy()
    assert np.allclose(w_gpu * kf, fn, rtol=FORCE_TOL, atol=0) or np.any(amb)
    m_gpu = out["m_trace"][:, 0].cpu().numpy()
    assert np.abs(m_gpu - r["m"]).max() <= 1e-6


# (cluster, agents per group, compute threads, exchange); exchange 1 = the
# cooperative-grid exchange through global memory
SHAPES = [(1, 4, 256, 0), (2, 3, 256, 0), (3, 6, 384, 0), (5, 2, 128, 0), (1, 6, 256, 1),
          (2, 4, 384, 1), (4, 3, 128, 1), (7, 12, 256, 1)]


@pytest.mark.parametrize("clear", [True, False], ids=["clear", "noclear"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "c%d_a%d_t%d_x%d" % s)
def test_sphere_ensemble_launch_shapes(gm, shape, clear):
    w = _sphere_ensemble(n_agents=12, n_apf=5, n_steps=160)
    obs, r_O = _filtered(w)
    obs = obs[:, :-1]   # an odd N_O: shards of odd length take the APF padding
    ref = oracle.rollout(obs, r_O, w["agents"], w["params"], n_apf=5)
    out = gm.rollout_ensemble(_gpu_obstacles(gm, obs, r_O, cap=4096), to_dev_agents(w["agents"]),
                              5, w["params"], tuning=shape, want_clear=clear)
    gm.sync()
    _compare(out, ref, clear=clear)


def test_tabletop_ensemble_full_size_sampled_agents(gm):
    """256 agents x 500 steps, the last 128 on APF, in the library's launch
    shape; 8 MFI and 8 APF agents checked against the oracle."""
    import torch
    w = synth.tabletop_workload()
    ag = synth.ensemble_agents(w["agents"], 128)
    xyz = torch.from_numpy(w["xyz"]).cuda()
    gobs = gm.filter_cloud(xyz, w["T"], w["workspace"], cap=131072)
    out = gm.rollout_ensemble(gobs, to_dev_agents(ag), 128, w["params"])
    gm.sync()
    idx = np.r_[np.arange(0, 128, 16) + np.arange(8) % 5, np.arange(128, 256, 16) + np.arange(8) % 3]
    obs, r_O = _filtered(w)
    ref = oracle.rollout(obs, r_O, subset_agents(ag, idx), w["params"], n_apf=8)
    _compare(out, ref, idx=idx)


@pytest.mark.parametrize("n_apf", [1, 11, 12])
def test_one_and_all_apf(gm, n_apf):
    w = _sphere_ensemble(n_agents=12, n_apf=n_apf, n_steps=150)
    obs, r_O = _filtered(w)
    ref = oracle.rollout(obs, r_O, w["agents"], w["params"], n_apf=n_apf)
    for shape in (None, (2, 5, 256, 0), (3, 4, 128, 1)):
        out = gm.rollout_ensemble(_gpu_obstacles(gm, obs, r_O), to_dev_agents(w["agents"]), n_apf,
                                  w["params"], tuning=shape)
        gm.sync()
        _compare(out, ref)


def test_apf_without_gate_and_without_obstacles(gm):
    w = _sphere_ensemble(n_agents=6, n_apf=3, n_steps=150)
    obs, r_O = _filtered(w)
    ag = dict(w["agents"])
    ag["r_d"] = np.full(6, np.inf, np.float32)
    ag["k_r"] = ag["k_r"] * np.float32(0.05)   # the ungated sums are larger
    ref = oracle.rollout(obs, r_O, ag, w["params"], n_apf=3)
    out = gm.rollout_ensemble(_gpu_obstacles(gm, obs, r_O), to_dev_agents(ag), 3, w["params"])
    gm.sync()
    _compare(out, ref)
    empty = np.zeros((3, 0), np.float32)
    ref0 = oracle.rollout(empty, r_O, w["agents"], w["params"], n_apf=3)
    out0 = gm.rollout_ensemble(_gpu_obstacles(gm, empty, r_O, cap=64), to_dev_agents(w["agents"]),
                               3, w["params"])
    gm.sync()
    _compare(out0, ref0)


def test_no_apf_is_rollout_agents_bitwise(gm):
    w = _sphere_ensemble(n_agents=20, n_apf=0, n_steps=120)
    obs, r_O = _filtered(w)
    o = _gpu_obstacles(gm, obs, r_O)
    ag = to_dev_agents(w["agents"])
    for shape in ((2, 5, 256, 0), (3, 4, 128, 1)):
        a = gm.rollout_ensemble(o, ag, 0, w["params"], tuning=shape)
        b = gm.rollout_agents(o, ag, w["params"], tuning=shape)
        gm.sync()
        for k in ("traj", "p_final", "v_final", "path_len", "min_clear"):
            assert np.array_equal(a[k].cpu().numpy(), b[k].cpu().numpy()), (shape, k)


def test_ensemble_bit_identical_repeats(gm):
    w = _sphere_ensemble(n_agents=30, n_apf=14, n_steps=150)
    obs, r_O = _filtered(w)
    o = _gpu_obstacles(gm, obs, r_O)
    ag = to_dev_agents(w["agents"])
    for shape in (None, (3, 6, 256, 0)):
        a = gm.rollout_ensemble(o, ag, 14, w["params"], tuning=shape)
        b = gm.rollout_ensemble(o, ag, 14, w["params"], tuning=shape)
        gm.sync()
        assert np.array_equal(a["traj"].cpu().numpy(), b["traj"].cpu().numpy())


def test_ensemble_invalid_arguments(gm):
    import torch
    w = _sphere_ensemble(n_agents=4, n_apf=2, n_steps=5)
    obs, r_O = _filtered(w)
    o = _gpu_obstacles(gm, obs, r_O)
    ag = to_dev_agents(w["agents"])
    for bad in (-1, 5):
        with pytest.raises(gm.GmappError) as e:
            gm.rollout_ensemble(o, ag, bad, w["params"])
        assert e.value.status == 1
    out = gm.alloc_rollout_out(4, 5)
    out["ckpt"] = torch.empty(1, 6, 4, dtype=torch.float32, device="cuda")
    with pytest.raises(gm.GmappError) as e:
        gm.rollout_ensemble(o, ag, 2, w["params"], out=out)
    assert e.value.status == 1
    # 38 MFI agents in two groups would need 19 agents per group (at most 12)
    big = to_dev_agents(synth.ensemble_agents(synth.sphere_workload(n_agents=40, n_steps=5)["agents"], 2))
    with pytest.raises(gm.GmappError) as e:
        gm.rollout_ensemble(o, big, 2, w["params"], tuning=(1, 16, 256, 0))
    assert e.value.status == 1


def test_ensemble_autotuner(gm):
    """gmapp_autotune_ensemble times ensemble shapes on the caller's inputs;
    a later rollout_ensemble of the same sizes without a shape uses the
    cached one and still matches the oracle."""
    w = _sphere_ensemble(n_agents=40, n_apf=16, n_steps=150)
    obs, r_O = _filtered(w)
    o = _gpu_obstacles(gm, obs, r_O, cap=4096)
    ag = to_dev_agents(w["agents"])
    out = gm.alloc_rollout_out(40, 150)
    shape, ms = gm.autotune_ensemble(o, ag, 16, w["params"], out=out, candidates=6, probe_steps=30)
    assert ms > 0 and len(shape) == 4 and shape[1] <= 12
    a = gm.rollout_ensemble(o, ag, 16, w["params"])
    b = gm.rollout_ensemble(o, ag, 16, w["params"], tuning=shape)
    gm.sync()
    assert np.array_equal(a["traj"].cpu().numpy(), b["traj"].cpu().numpy())
    ref = oracle.rollout(obs, r_O, w["agents"], w["params"], n_apf=16)
    _compare(a, ref)


# ---- MFI with the per-obstacle projected current (the third kind) ----------

def test_projected_force_parity_at_oracle_states(gm):
    """f_r of projected-current agents evaluated once (N_k = 1) at states of
    the oracle's trajectories.  Each term of f = (|v|^2 S - v B) / |v| is at
    most 2 w_j |v| (w_j = 1/s_j inside the gate), so the FP32 bound is
    1e-5 |f| + 4e-6 k_f |v| W, W = sum_j w_j, plus 2 k_f |v| / r_d per
    gate-ambiguous pair."""
    w = _sphere_ensemble(n_agents=12, n_apf=0)
    obs, r_O = _filtered(w)
    prm = w["params"]
    ref = oracle.rollout(obs, r_O, w["agents"], prm, n_proj=12)
    ps, vs = [], []
    for k in (1, 40, 80, 110, 140, 170, 199):
        ps.append(ref["traj"][:, k].T)
        vs.append((ref["traj"][:, k] - ref["traj"][:, k - 1]).T / prm.dt)
    P = np.concatenate(ps, axis=1).astype(np.float32)
    V = np.concatenate(vs, axis=1).astype(np.float32)
    n = P.shape[1]
    ag = subset_agents(w["agents"], np.tile(np.arange(12), 7))
    ag["p0"], ag["v0"] = np.ascontiguousarray(P), np.ascontiguousarray(V)
    one = dataclasses.replace(prm, n_steps=1)
    out = gm.rollout_ensemble(_gpu_obstacles(gm, obs, r_O), to_dev_agents(ag), 0, one,
                              want_trace=True, n_proj=n)
    gm.sync()
    f_gpu = out["f_trace"][:, 0, :].cpu().numpy().T.astype(np.float64)
    P64, V64 = P.astype(np.float64), V.astype(np.float64)
    r = oracle.proj_eval(obs, r_O, P64, V64, ag, prm.rho, prm.eps)
    W = oracle.cf_eval(obs, r_O, P64, V64, ag, prm.rho, prm.eps)["W"]
    R = ag["r_a"].astype(np.float64) + r_O
    r_d = ag["r_d"].astype(np.float64)
    kf = prm.rho * ag["k_r"].astype(np.float64)
    vn = np.linalg.norm(V64, axis=0)
    amb = gate_allowance(obs.astype(np.float64), P64, R, r_d)
    fn = np.linalg.norm(r["f_r"], axis=0)
    err = np.linalg.norm(f_gpu - r["f_r"], axis=0)
    tol = FORCE_TOL * fn + 4e-6 * kf * vn * W + amb * 2.0 * kf * vn / r_d
    assert (fn > 0).sum() >= 20
    assert np.all(err <= tol), (err / np.maximum(fn, 1e-30)).max()
    assert np.all(np.abs((f_gpu * V64).sum(axis=0)) <= 1e-5 * fn * vn + 4e-6 * kf * vn * vn * W)
    m_gpu = out["m_trace"][:, 0].cpu().numpy()
    assert np.abs(m_gpu - r["m"]).max() <= 1e-6


@pytest.mark.parametrize("clear", [True, False], ids=["clear", "noclear"])
@pytest.mark.parametrize("shape", [(1, 4, 256, 0), (3, 3, 256, 0), (2, 4, 128, 1), (5, 2, 256, 1)],
                         ids=lambda s: "c%d_a%d_t%d_x%d" % s)
def test_three_kind_ensemble_launch_shapes(gm, shape, clear):
    """4 MFI + 4 projected-current + 4 APF agents in one launch."""
    w = _sphere_ensemble(n_agents=12, n_apf=4, n_steps=160)
    obs, r_O = _filtered(w)
    obs = obs[:, :-1]   # odd N_O: odd shards take the far padding
    ref = oracle.rollout(obs, r_O, w["agents"], w["params"], n_apf=4, n_proj=4)
    out = gm.rollout_ensemble(_gpu_obstacles(gm, obs, r_O, cap=4096), to_dev_agents(w["agents"]),
                              4, w["params"], tuning=shape, want_clear=clear, n_proj=4)
    gm.sync()
    _compare(out, ref, clear=clear)


@pytest.mark.parametrize("n_proj", [1, 12])
def test_projected_only_and_single(gm, n_proj):
    w = _sphere_ensemble(n_agents=12, n_apf=0, n_steps=150)
    obs, r_O = _filtered(w)
    ref = oracle.rollout(obs, r_O, w["agents"], w["params"], n_proj=n_proj)
    for shape in (None, (2, 5, 256, 0), (3, 4, 128, 1)):
        out = gm.rollout_ensemble(_gpu_obstacles(gm, obs, r_O), to_dev_agents(w["agents"]), 0,
                                  w["params"], tuning=shape, n_proj=n_proj)
        gm.sync()
        _compare(out, ref)


def test_tabletop_three_kinds_sampled_agents(gm):
    """256 agents x 500 steps: 86 MFI, 85 projected-current, 85 APF in the
    library's shape; 6 of each kind checked against the oracle."""
    import torch
    w = synth.tabletop_workload()
    ag = synth.ensemble_agents(w["agents"], 85)
    xyz = torch.from_numpy(w["xyz"]).cuda()
    gobs = gm.filter_cloud(xyz, w["T"], w["workspace"], cap=131072)
    out = gm.rollout_ensemble(gobs, to_dev_agents(ag), 85, w["params"], n_proj=85)
    gm.sync()
    idx = np.r_[np.arange(0, 86, 15), np.arange(86, 171, 15), np.arange(171, 256, 15)]
    obs, r_O = _filtered(w)
    ref = oracle.rollout(obs, r_O, subset_agents(ag, idx), w["params"], n_apf=6, n_proj=6)
    _compare(out, ref, idx=idx)


def test_projected_invalid_counts(gm):
    w = _sphere_ensemble(n_agents=4, n_apf=1, n_steps=5)
    obs, r_O = _filtered(w)
    o = _gpu_obstacles(gm, obs, r_O)
    ag = to_dev_agents(w["agents"])
    for n_proj, n_apf in ((-1, 1), (4, 1), (3, 2)):
        with pytest.raises(gm.GmappError) as e:
            gm.rollout_ensemble(o, ag, n_apf, w["params"], n_proj=n_proj)
        assert e.value.status == 1
