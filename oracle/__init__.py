"""FP64 CPU oracle for the G-MAPP hot path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg
may import this package.  The product path never does; the CUDA library and
this oracle share no source, headers or helpers.  Inputs come from the seeded
generators in ``synth``.

Functions (each cites the paper passage it follows):
  filter_cloud    Sec. IV-B / V-A   camera cloud -> sorted voxel centres S_W
  filter_clouds   Sec. IV-B         several sensors' clouds fused into one S_W
  cf_eval         Eq. (mfi), Alg. 1 W, clearance and f_r at given states
  apf_eval        Eq. (apf)         APF force and clearance at given states
  rollout         Sec. IV-A         N_k-step point-mass rollout + cost sums
                                    (MFI agents, and APF agents of an ensemble)
  costs, select   Sec. IV-A         weighted cost and argmin selection
  four_term_costs Eq. (cost_function) goal, obstacle, path, smoothness terms
  fd_gradient     --                central finite differences of the cost
Parity pins for every function live in tests/test_oracle_*.py.
"""

from __future__ import annotations

import ctypes as C
import math

import numpy as np

from .build import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build())
        P = C.c_void_p
        i64 = C.c_int64
        _lib.oracle_filter.restype = i64
        _lib.oracle_filter.argtypes = [P, i64, P, P, C.c_float, P, C.c_int32, i64,
                                       P, P, P, P, P, P]
        _lib.oracle_filter_fused.restype = i64
        _lib.oracle_filter_fused.argtypes = [P, P, P, C.c_int32, P, C.c_float, P, C.c_int32, i64,
                                             P, P, P, P, P, P]
        _lib.oracle_cf_eval.restype = None
        _lib.oracle_cf_eval.argtypes = [i64, P, P, P, C.c_double, i64, P, P, P, P, P, P,
                                        C.c_double, C.c_double, P, P, P]
        _lib.oracle_rollout.restype = None
        _lib.oracle_rollout.argtypes = [i64, P, P, P, C.c_double, i64, P, P, P, P, P, P, P,
                                        P, P, P, P, P, P, P, P, P, i64, i64]
        _lib.oracle_proj_eval.restype = None
        _lib.oracle_proj_eval.argtypes = [i64, P, P, P, C.c_double, i64, P, P, P, P, P,
                                          C.c_double, C.c_double, P, P]
        _lib.oracle_apf_eval.restype = None
        _lib.oracle_apf_eval.argtypes = [i64, P, P, P, C.c_double, i64, P, P, P, P,
                                         C.c_double, C.c_double, P, P, P]
        _lib.oracle_max_threads.restype = C.c_int
        _lib.oracle_set_threads.argtypes = [C.c_int]
        _lib.oracle_adjoint.restype = None
        _lib.oracle_adjoint.argtypes = [i64, P, P, P, C.c_double, i64, P, P, P, P, P, P, P, P, P,
                                        P, P, P, P, P, P]
    return _lib


class _Params(C.Structure):
    _fields_ = [("goal", C.c_double * 3), ("dt", C.c_double), ("n_steps", C.c_int64),
                ("damping", C.c_double), ("inv_mass", C.c_double), ("rho", C.c_double),
                ("eps", C.c_double), ("vel_half", C.c_double),
                ("clear_margin", C.c_double), ("clear_beta", C.c_double)]


def _params(prm) -> _Params:
    p = _Params()
    for a in range(3):
        p.goal[a] = float(prm.goal[a])
    p.dt, p.n_steps = float(prm.dt), int(prm.n_steps)
    p.damping, p.inv_mass, p.rho = float(prm.damping), float(prm.inv_mass), float(prm.rho)
    p.eps, p.vel_half = float(prm.eps), float(prm.vel_half)
    p.clear_margin, p.clear_beta = float(prm.clear_margin), float(prm.clear_beta)
    return p


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(lib().oracle_max_threads())


# ---------------------------------------------------------------------------
# Perception (Sec. IV-B, Sec. V-A)
# ---------------------------------------------------------------------------

def filter_cloud(xyz: np.ndarray, T, workspace, cap: int | None = None) -> dict:
    """Transform, crop and voxelise a camera-frame cloud; returns the sorted
    occupied voxels (keys, counts, smallest point index) and their centres,
    exactly as the binary32 sequence in ``gmapp_oracle.c`` defines them."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
    T = np.ascontiguousarray(T, dtype=np.float32).reshape(12)
    lo = np.ascontiguousarray(workspace.lo, dtype=np.float32)
    dims = np.ascontiguousarray(workspace.dims, dtype=np.int32)
    n = xyz.shape[0]
    cap = n if cap is None else int(cap)
    keys = np.zeros(max(cap, 1), np.uint32)
    counts = np.zeros(max(cap, 1), np.uint32)
    rep = np.zeros(max(cap, 1), np.uint32)
    cx = np.zeros(max(cap, 1), np.float32)
    cy = np.zeros(max(cap, 1), np.float32)
    cz = np.zeros(max(cap, 1), np.float32)
    n_out = lib().oracle_filter(_ptr(xyz), n, _ptr(T), _ptr(lo), float(np.float32(workspace.voxel)),
                                _ptr(dims), int(workspace.min_pts), cap, _ptr(keys), _ptr(counts),
                                _ptr(rep), _ptr(cx), _ptr(cy), _ptr(cz))
    k = min(n_out, cap)
    return {"n": int(n_out), "keys": keys[:k], "counts": counts[:k], "rep_idx": rep[:k],
            "x": cx[:k], "y": cy[:k], "z": cz[:k],
            "r_O": float(np.float32(workspace.voxel) * np.float32(0.5))}


def filter_clouds(clouds, workspace, cap: int | None = None) -> dict:
    """Several sensors' clouds [(xyz, T), ...] fused into one obstacle set
    (Sec. IV-B); point i of cloud s has the index n_0 + ... + n_{s-1} + i."""
    xyzs = [np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 3) for x, _ in clouds]
    ns = np.array([x.shape[0] for x in xyzs], dtype=np.int64)
    xyz = np.ascontiguousarray(np.concatenate(xyzs, axis=0) if xyzs else np.zeros((0, 3), np.float32))
    T = np.ascontiguousarray(np.stack([np.asarray(t, np.float32).reshape(12) for _, t in clouds]))
    lo = np.ascontiguousarray(workspace.lo, dtype=np.float32)
    dims = np.ascontiguousarray(workspace.dims, dtype=np.int32)
    n = int(ns.sum())
    cap = n if cap is None else int(cap)
    out = {k: np.zeros(max(cap, 1), np.uint32) for k in ("keys", "counts", "rep_idx")}
    cs = [np.zeros(max(cap, 1), np.float32) for _ in range(3)]
    n_out = lib().oracle_filter_fused(_ptr(xyz), _ptr(ns), _ptr(T), len(clouds), _ptr(lo),
                                      float(np.float32(workspace.voxel)), _ptr(dims),
                                      int(workspace.min_pts), cap, _ptr(out["keys"]),
                                      _ptr(out["counts"]), _ptr(out["rep_idx"]), _ptr(cs[0]),
                                      _ptr(cs[1]), _ptr(cs[2]))
    k = min(n_out, cap)
    return {"n": int(n_out), "keys": out["keys"][:k], "counts": out["counts"][:k],
            "rep_idx": out["rep_idx"][:k], "x": cs[0][:k], "y": cs[1][:k], "z": cs[2][:k],
            "r_O": float(np.float32(workspace.voxel) * np.float32(0.5))}


# ---------------------------------------------------------------------------
# Force (Eq. mfi, Alg. 1) and rollout (Sec. IV-A)
# ---------------------------------------------------------------------------

def cf_eval(obs_xyz, r_O: float, p, v, agents: dict, rho: float, eps: float) -> dict:
    """W, clearance m and f_r = rho k_r W g for every agent at state (p, v).
    ``obs_xyz`` is [3, N_O]; p, v are [3, N_a]."""
    ox, oy, oz = (_f64(obs_xyz[a]) for a in range(3))
    p, v = _f64(p), _f64(v)
    na = p.shape[1]
    c = _f64(agents["c"])
    k_r, r_d, r_a = _f64(agents["k_r"]), _f64(agents["r_d"]), _f64(agents["r_a"])
    W = np.zeros(na)
    m = np.zeros(na)
    fr = np.zeros((3, na))
    lib().oracle_cf_eval(ox.size, _ptr(ox), _ptr(oy), _ptr(oz), float(r_O), na, _ptr(p), _ptr(v),
                         _ptr(c), _ptr(k_r), _ptr(r_d), _ptr(r_a), float(rho), float(eps),
                         _ptr(W), _ptr(m), _ptr(fr))
    return {"W": W, "m": m, "f_r": fr}


def apf_eval(obs_xyz, r_O: float, p, agents: dict, rho: float, eps: float) -> dict:
    """Clearance m and the APF force f_r = rho k_r f (Eq. apf) for every agent
    at positions p [3, N_a]; f_abs = |rho k_r| times the sum of the term
    magnitudes (the scale of the rounding error of the vector sum)."""
    ox, oy, oz = (_f64(obs_xyz[a]) for a in range(3))
    p = _f64(p)
    na = p.shape[1]
    k_r, r_d, r_a = _f64(agents["k_r"]), _f64(agents["r_d"]), _f64(agents["r_a"])
    m = np.zeros(na)
    fr = np.zeros((3, na))
    fa = np.zeros(na)
    lib().oracle_apf_eval(ox.size, _ptr(ox), _ptr(oy), _ptr(oz), float(r_O), na, _ptr(p),
                          _ptr(k_r), _ptr(r_d), _ptr(r_a), float(rho), float(eps), _ptr(m),
                          _ptr(fr), _ptr(fa))
    return {"m": m, "f_r": fr, "f_abs": fa}


def proj_eval(obs_xyz, r_O: float, p, v, agents: dict, rho: float, eps: float) -> dict:
    """Clearance m and the projected-current MFI force f_r = rho k_r f (Eq.
    mfi with the per-obstacle current c_j) for every agent at states (p, v),
    [3, N_a] each."""
    ox, oy, oz = (_f64(obs_xyz[a]) for a in range(3))
    p, v = _f64(p), _f64(v)
    na = p.shape[1]
    k_r, r_d, r_a = _f64(agents["k_r"]), _f64(agents["r_d"]), _f64(agents["r_a"])
    m = np.zeros(na)
    fr = np.zeros((3, na))
    lib().oracle_proj_eval(ox.size, _ptr(ox), _ptr(oy), _ptr(oz), float(r_O), na, _ptr(p),
                           _ptr(v), _ptr(k_r), _ptr(r_d), _ptr(r_a), float(rho), float(eps),
                           _ptr(m), _ptr(fr))
    return {"m": m, "f_r": fr}


def rollout(obs_xyz, r_O: float, agents: dict, prm, want_traj: bool = True,
            want_trace: bool = False, n_apf: int = 0, n_proj: int = 0) -> dict:
    """FP64 rollout of all agents; returns the trajectory [N_a, N_k+1, 3],
    final state, path length, clearance penalty sum and minimum clearance.
    The last ``n_apf`` agents use the APF heuristic (Eq. apf), the ``n_proj``
    before them MFI with the per-obstacle projected current, the others the
    MFI / circular field with the agent's own current (Eq. mfi)."""
    ox, oy, oz = (_f64(obs_xyz[a]) for a in range(3))
    ag = {k: _f64(v) for k, v in agents.items()}
    na = ag["k_r"].size
    N = int(prm.n_steps)
    traj = np.zeros((na, N + 1, 3)) if want_traj else None
    wtr = np.zeros((na, N)) if want_trace else None
    mtr = np.zeros((na, N)) if want_trace else None
    out = {"p_final": np.zeros((3, na)), "v_final": np.zeros((3, na)),
           "path_len": np.zeros(na), "clear_pen": np.zeros(na), "min_clear": np.zeros(na)}
    pr = _params(prm)
    nul = C.c_void_p(0)
    lib().oracle_rollout(ox.size, _ptr(ox), _ptr(oy), _ptr(oz), float(r_O), na,
                         _ptr(ag["p0"]), _ptr(ag["v0"]), _ptr(ag["c"]), _ptr(ag["k_r"]),
                         _ptr(ag["k_a"]), _ptr(ag["r_d"]), _ptr(ag["r_a"]), C.byref(pr),
                         _ptr(traj) if want_traj else nul, _ptr(out["p_final"]),
                         _ptr(out["v_final"]), _ptr(out["path_len"]), _ptr(out["clear_pen"]),
                         _ptr(out["min_clear"]), _ptr(wtr) if want_trace else nul,
                         _ptr(mtr) if want_trace else nul, int(n_apf), int(n_proj))
    if want_traj:
        out["traj"] = traj
    if want_trace:
        out["w_trace"], out["m_trace"] = wtr, mtr
    return out


# ---------------------------------------------------------------------------
# Cost and selection (Sec. IV-A "Cost Functions", "Selection Mechanism")
# ---------------------------------------------------------------------------

def costs(ro: dict, prm) -> np.ndarray:
    """C_i = w_path L_i + w_goal |p_i(N_k) - p_goal| + w_clear sum_k softplus."""
    g = np.asarray(prm.goal, dtype=np.float64)[:, None]
    dgoal = np.sqrt(((ro["p_final"] - g) ** 2).sum(axis=0))
    return prm.w_path * ro["path_len"] + prm.w_goal * dgoal + prm.w_clear * ro["clear_pen"]


def four_term_costs(traj, m_trace, goal, dt: float, r_c: float, a_max: float,
                    w=(1.0, 1.0, 1.0, 1.0)) -> dict:
    """Eq. (cost_function): C_i = sum_j w_j C_ij with the four terms of
    Sec. IV-A "Cost Functions", per agent, in FP64.

    The candidate trajectory is the N_k states at which the field is
    evaluated, xi^(k) = p_(k-1) for k = 1..N_k (so d^(1) is the distance of
    the start to the goal), taken from ``traj`` [N_a, N_k+1, 3]; the
    obstacle distance at xi^(k) is the clearance m_(k-1) of ``m_trace``
    [N_a, N_k] (inf without obstacles); r_c is the radius of Eqs. (cost_goal)
    and (cost_obs), one value for all agents.
      C_goal   = 1/N_k sum_k min(|xi^k - g|, r_c) / r_c                 Eq. (cost_goal)
      C_obs    = 1/N_k sum_k (1 - min(m^k, r_c) / r_c)                   Eq. (cost_obs)
      L        = sum_{k=2}^{N_k} |xi^k - xi^(k-1)|,  d1 = |xi^1 - g|
      C_path   = 1 - d1 / L  if L >= d1,  else 1 - L / d1  (0 when L = d1 = 0)   Eq. (cost_path)
      J        = sum_{k=4}^{N_k} |xi^k - 3 xi^(k-1) + 3 xi^(k-2) - xi^(k-3)|^2
      C_smooth = min(1, J / (N_k dt^4 a_max^2))                          Eq. (cost_smooth)
    Returns the four terms, L, J, d1 and the weighted total C."""
    traj = _f64(traj)
    xi = traj[:, :-1, :]
    nk = xi.shape[1]
    g = np.asarray(goal, dtype=np.float64)
    dg = np.sqrt(((xi - g) ** 2).sum(axis=2))
    c_goal = (np.minimum(dg, r_c) / r_c).sum(axis=1) / nk
    c_obs = (1.0 - np.minimum(_f64(m_trace), r_c) / r_c).sum(axis=1) / nk
    L = np.sqrt((np.diff(xi, axis=1) ** 2).sum(axis=2)).sum(axis=1)
    d1 = dg[:, 0]
    with np.errstate(divide="ignore", invalid="ignore"):
        c_path = np.where(L >= d1, 1.0 - d1 / L, 1.0 - L / d1)
    c_path = np.where((L == 0.0) & (d1 == 0.0), 0.0, c_path)
    if nk >= 4:
        j3 = xi[:, 3:] - 3.0 * xi[:, 2:-1] + 3.0 * xi[:, 1:-2] - xi[:, :-3]
        J = (j3 ** 2).sum(axis=(1, 2))
    else:
        J = np.zeros(xi.shape[0])
    c_smooth = np.minimum(1.0, J / (nk * dt ** 4 * a_max ** 2))
    C = w[0] * c_goal + w[1] * c_obs + w[2] * c_path + w[3] * c_smooth
    return {"goal": c_goal, "obs": c_obs, "path": c_path, "smooth": c_smooth, "L": L, "J": J,
            "d1": d1, "C": C}


def select(c: np.ndarray, prev_best_cost: float = math.nan, alpha: float = 1.0) -> int:
    """i* = argmin_i C_i (ties -> lowest index).  With a previous best cost
    C_best, only agents with C_i < alpha C_best qualify; -1 when none does
    (the previous best path is kept)."""
    c = np.asarray(c, dtype=np.float64)
    if math.isnan(prev_best_cost):
        return int(np.argmin(c))
    ok = np.nonzero(c < alpha * prev_best_cost)[0]
    if ok.size == 0:
        return -1
    return int(ok[np.argmin(c[ok])])


class _Weights(C.Structure):
    _fields_ = [("w_path", C.c_double), ("w_goal", C.c_double), ("w_clear", C.c_double)]


def adjoint(obs_xyz, r_O: float, agents: dict, prm) -> dict:
    """Cost of every agent and its gradient with respect to v0 [3, N_a],
    k_r, k_a [N_a] and c [3, N_a] by the discrete adjoint (reverse sweep of
    the stored FP64 rollout), plus each agent's branch signature."""
    ox, oy, oz = (_f64(obs_xyz[a]) for a in range(3))
    ag = {k: _f64(v) for k, v in agents.items()}
    na = ag["k_r"].size
    out = {"cost": np.zeros(na), "g_v0": np.zeros((3, na)), "g_kr": np.zeros(na),
           "g_ka": np.zeros(na), "g_c": np.zeros((3, na)), "sig": np.zeros(na, np.uint64)}
    pr = _params(prm)
    wt = _Weights(float(prm.w_path), float(prm.w_goal), float(prm.w_clear))
    lib().oracle_adjoint(ox.size, _ptr(ox), _ptr(oy), _ptr(oz), float(r_O), na, _ptr(ag["p0"]),
                         _ptr(ag["v0"]), _ptr(ag["c"]), _ptr(ag["k_r"]), _ptr(ag["k_a"]),
                         _ptr(ag["r_d"]), _ptr(ag["r_a"]), C.byref(pr), C.byref(wt),
                         _ptr(out["cost"]), _ptr(out["g_v0"]), _ptr(out["g_kr"]),
                         _ptr(out["g_ka"]), _ptr(out["g_c"]), _ptr(out["sig"]))
    return out


GRAD_NAMES = [("v0", 0), ("v0", 1), ("v0", 2), ("k_r", None), ("k_a", None),
              ("c", 0), ("c", 1), ("c", 2)]


def grad_vector(adj: dict, i: int) -> np.ndarray:
    """The 8 gradient entries of agent i in GRAD_NAMES order."""
    return np.array([adj["g_v0"][0, i], adj["g_v0"][1, i], adj["g_v0"][2, i], adj["g_kr"][i],
                     adj["g_ka"][i], adj["g_c"][0, i], adj["g_c"][1, i], adj["g_c"][2, i]])


def fd_gradient(obs_xyz, r_O, agents: dict, prm, agent_ids, h: float = 1e-6) -> dict:
    """Central finite differences (step h) of each listed agent's cost with
    respect to v0 (3), k_r, k_a and c (3), perturbing one agent parameter at
    a time (agents are independent, so every perturbed copy is one more
    agent of a single oracle run).  Returns per agent (gradient[8],
    valid[8]); an entry is valid only when both perturbed runs have the
    unperturbed run's branch signature (no clamp, gate or nearest-obstacle
    change inside +-h: no kink crossed)."""
    ids = [int(i) for i in agent_ids]
    copies = []  # per listed agent: base, then (+h, -h) for each of the 8 parameters
    for i in ids:
        one = {k: (_f64(v)[:, i:i + 1] if _f64(v).ndim == 2 else _f64(v)[i:i + 1])
               for k, v in agents.items()}
        copies.append(one)
        for name, ax in GRAD_NAMES:
            for sgn in (+1, -1):
                a = {k: v.copy() for k, v in one.items()}
                if ax is None:
                    a[name][0] += sgn * h
                else:
                    a[name][ax, 0] += sgn * h
                copies.append(a)
    allc = {k: np.ascontiguousarray(np.concatenate([c[k] for c in copies], axis=-1))
            for k in copies[0]}
    r = adjoint(obs_xyz, r_O, allc, prm)
    per = 1 + 2 * len(GRAD_NAMES)
    out = {}
    for n, i in enumerate(ids):
        b = n * per
        g = np.zeros(8)
        ok = np.zeros(8, bool)
        for q in range(len(GRAD_NAMES)):
            up, dn = b + 1 + 2 * q, b + 2 + 2 * q
            g[q] = (r["cost"][up] - r["cost"][dn]) / (2 * h)
            ok[q] = r["sig"][up] == r["sig"][b] and r["sig"][dn] == r["sig"][b]
        out[i] = (g, ok)
    return out
