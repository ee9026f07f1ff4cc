"""B300-native G-MAPP hot path: Python binding of libgmapp.so.

Argument marshalling only: every step of the path runs in the CUDA kernels
behind the C ABI (include/gmapp.h).  PyTorch supplies device memory and the
current stream.  There is no CPU fallback: on a machine without the library
or a CUDA device every compute call raises.

    ctx  = Context(0)
    obs  = filter_cloud(xyz, T, workspace)               # Sec. IV-B / V-A
    ro   = rollout_agents(obs, agents, params)           # Sec. IV-A, Eq. (mfi), Alg. 1
    sel  = score_and_select(ro, params, weights)         # Sec. IV-A cost, selection
"""

from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass

from . import _abi
from ._abi import check

__all__ = ["Context", "context", "Obstacles", "filter_cloud", "filter_clouds",
           "filter_cloud_noalloc", "filter_cloud_noalloc_status",
           "filter_workspace_bytes", "rollout_agents", "rollout_ensemble", "score_and_select",
           "score_and_select4", "grid_index", "rollout_agents_culled",
           "pick_tuning", "autotune_rollout", "autotune_ensemble", "rollout_adjoint", "GMappRollout", "sync", "GmappError",
           "FilterBatch", "Batch", "Server", "measure_peaks"]

GmappError = _abi.GmappError


def _torch():
    import torch
    return torch


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _stream(stream) -> C.c_void_p:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Context:
    """One library context per CUDA device (owns the device error word)."""

    def __init__(self, device: int = 0):
        lib = _abi.load()
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2606_12579_b300 needs a CUDA device (no CPU fallback)")
        torch.cuda.init()
        h = C.c_void_p()
        check(lib.gmapp_create(C.byref(h), int(device)), "gmapp_create")
        self.handle = h
        self.device = int(device)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _abi._lib is not None:
            _abi._lib.gmapp_destroy(h)
            self.handle = None

    def sync(self, stream=None) -> None:
        """Wait for the stream and raise if a kernel flagged a device error."""
        check(_abi.load().gmapp_sync(self.handle, _stream(stream)), "gmapp_sync")

    def set_wait_limit(self, polls: int) -> None:
        """Cap the polls of the rollout kernels' bounded waits (0 = defaults);
        a wait that gives up is reported as GMAPP_ERR_TIMEOUT by sync()."""
        check(_abi.load().gmapp_set_wait_limit(self.handle, int(polls)), "gmapp_set_wait_limit")

    def device_error_bits(self) -> int:
        b = C.c_uint32()
        check(_abi.load().gmapp_peek_device_error(self.handle, C.byref(b)), "peek")
        return int(b.value)


_contexts: dict = {}


def context(device: int | None = None) -> Context:
    torch = _torch()
    d = torch.cuda.current_device() if device is None else int(device)
    if d not in _contexts:
        _contexts[d] = Context(d)
    return _contexts[d]


def sync(stream=None, device: int | None = None) -> None:
    context(device).sync(stream)


# ---------------------------------------------------------------------------
# Obstacles (the sphere world S_W)
# ---------------------------------------------------------------------------

@dataclass
class Obstacles:
    x: object
    y: object
    z: object
    keys: object
    counts: object
    rep_idx: object
    n: object          # device int32 [1]
    cap: int
    r_O: float

    @staticmethod
    def empty(cap: int, device=None) -> "Obstacles":
        torch = _torch()
        cap = max(4, (int(cap) + 3) // 4 * 4)
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        f = lambda: torch.empty(cap, dtype=torch.float32, device=dev)  # noqa: E731
        u = lambda: torch.empty(cap, dtype=torch.int32, device=dev)    # noqa: E731
        return Obstacles(f(), f(), f(), u(), u(), u(), torch.zeros(1, dtype=torch.int32, device=dev),
                         cap, 0.0)

    @staticmethod
    def from_points(xyz, r_O: float, cap: int | None = None) -> "Obstacles":
        """Obstacle set from a [3, N] tensor of centres (copied to device)."""
        torch = _torch()
        n = int(xyz.shape[1])
        o = Obstacles.empty(max(n, 1) if cap is None else cap)
        if n > o.cap:
            raise ValueError(f"{n} obstacles exceed cap {o.cap}")
        src = xyz.to(device=o.x.device, dtype=torch.float32)
        o.x[:n].copy_(src[0])
        o.y[:n].copy_(src[1])
        o.z[:n].copy_(src[2])
        o.n.fill_(n)
        o.r_O = float(r_O)
        return o

    def count(self) -> int:
        return int(self.n.item())

    def centres(self):
        """[3, N_O] view of the valid centres (reads N_O from the device)."""
        torch = _torch()
        k = min(self.count(), self.cap)
        return torch.stack([self.x[:k], self.y[:k], self.z[:k]])

    def _struct(self) -> _abi.Obstacles:
        s = _abi.Obstacles()
        s.x, s.y, s.z = self.x.data_ptr(), self.y.data_ptr(), self.z.data_ptr()
        s.keys = self.keys.data_ptr() if self.keys is not None else None
        s.counts = self.counts.data_ptr() if self.counts is not None else None
        s.rep_idx = self.rep_idx.data_ptr() if self.rep_idx is not None else None
        s.n = self.n.data_ptr()
        s.cap = int(self.cap)
        s.r_O = float(self.r_O)
        return s


def _ws_struct(ws) -> _abi.Workspace:
    s = _abi.Workspace()
    for a in range(3):
        s.lo[a] = float(ws.lo[a])
        s.dims[a] = int(ws.dims[a])
    s.voxel = float(ws.voxel)
    s.min_pts = int(getattr(ws, "min_pts", 1))
    return s


def measure_peaks(reps: int = 5) -> dict:
    """Measured FP32 FMA (packed and scalar) and SFU rates of the current GPU
    (gmapp_measure_peaks): the denominators of the force kernel's roofline."""
    context()
    p = _abi.Peaks()
    check(_abi.load().gmapp_measure_peaks(int(reps), C.byref(p)), "gmapp_measure_peaks")
    return {f: getattr(p, f) for f, _ in _abi.Peaks._fields_}


def filter_workspace_bytes(n_raw: int, ws) -> int:
    return int(_abi.load().gmapp_filter_workspace_bytes(int(n_raw), C.byref(_ws_struct(ws))))


def filter_cloud(xyz, T, ws, out: Obstacles | None = None, cap: int | None = None,
                 workspace=None, stream=None) -> Obstacles:
    """Camera-frame cloud [N, 3] (float32, device) -> S_W (Sec. IV-B, V-A).

    ``T`` is the 3x4 row-major camera-to-world transform (12 numbers), ``ws``
    any object with ``lo``, ``voxel``, ``dims`` (and ``min_pts``).  The
    obstacle count stays on the device (``out.n``) until asked for."""
    torch = _torch()
    ctx = context()
    n = int(xyz.shape[0])
    if out is None:
        out = Obstacles.empty(cap if cap is not None else max(n, 4))
    wss = _ws_struct(ws)
    need = int(_abi.load().gmapp_filter_workspace_bytes(n, C.byref(wss)))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=xyz.device)
    Tc = (C.c_float * 12)(*[float(v) for v in list(T)])
    ob = out._struct()
    check(_abi.load().filter_cloud(ctx.handle, _ptr(xyz), n, C.byref(Tc), C.byref(wss),
                                   C.byref(ob), _ptr(workspace), int(workspace.numel()),
                                   _stream(stream)), "filter_cloud")
    out.r_O = float(ob.r_O)
    return out


def filter_clouds(clouds, ws, out: Obstacles | None = None, cap: int | None = None,
                  workspace=None, stream=None) -> Obstacles:
    """Several sensors fused into one S_W (Sec. IV-B): ``clouds`` is a list
    of (xyz [N_s, 3] float32 device tensor, T 12 numbers) pairs; point i of
    sensor s has the index N_0 + ... + N_{s-1} + i."""
    torch = _torch()
    ctx = context()
    arr = (_abi.SensorCloud * len(clouds))()
    for s, (xyz, T) in enumerate(clouds):
        arr[s].xyz = xyz.data_ptr() if xyz.numel() else None
        arr[s].n_raw = int(xyz.shape[0])
        for i, v in enumerate(list(T)):
            arr[s].T[i] = float(v)
    total = sum(int(x.shape[0]) for x, _ in clouds)
    if out is None:
        out = Obstacles.empty(cap if cap is not None else max(total, 4))
    wss = _ws_struct(ws)
    lib = _abi.load()
    need = int(lib.gmapp_filter_clouds_workspace_bytes(arr, len(clouds), C.byref(wss)))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=out.x.device)
    ob = out._struct()
    check(lib.filter_clouds(ctx.handle, arr, len(clouds), C.byref(wss), C.byref(ob),
                            _ptr(workspace), int(workspace.numel()), _stream(stream)),
          "filter_clouds")
    out.r_O = float(ob.r_O)
    return out


def filter_cloud_noalloc(xyz, T, ws, out: Obstacles, stream=None) -> Obstacles:
    """filter_cloud whose scratch is the library's fixed 16 MiB device array:
    no workspace and no allocation inside the call (``out`` is the caller's).
    For callers that may not allocate once running.  Calls that overlap on
    the GPU share the array and race; the first call on a device should come
    before any stream capture."""
    n = int(xyz.shape[0])
    Tc = (C.c_float * 12)(*[float(v) for v in list(T)])
    wss = _ws_struct(ws)
    ob = out._struct()
    check(_abi.load().filter_cloud_noalloc(_ptr(xyz), n, C.byref(Tc), C.byref(wss), C.byref(ob),
                                           _stream(stream)), "filter_cloud_noalloc")
    out.r_O = float(ob.r_O)
    return out


def filter_cloud_noalloc_status(stream=None) -> None:
    """Waits for ``stream`` and raises GmappError (GMAPP_ERR_CAPACITY) when the
    latest filter_cloud_noalloc call found more voxels than ``out.cap``."""
    check(_abi.load().filter_cloud_noalloc_status(_stream(stream)), "filter_cloud_noalloc_status")


# ---------------------------------------------------------------------------
# Rollout and selection
# ---------------------------------------------------------------------------

AGENT_KEYS = ("p0", "v0", "c", "k_r", "k_a", "r_d", "r_a")


def _agents_struct(agents: dict) -> _abi.Agents:
    s = _abi.Agents()
    for k in AGENT_KEYS:
        t = agents[k]
        if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float32"):
            raise ValueError(f"agent array {k} must be a contiguous float32 CUDA tensor")
        setattr(s, k, t.data_ptr())
    s.n = int(agents["k_r"].numel())
    return s


def _params_struct(prm) -> _abi.RolloutParams:
    s = _abi.RolloutParams()
    for a in range(3):
        s.goal[a] = float(prm.goal[a])
    s.dt, s.n_steps = float(prm.dt), int(prm.n_steps)
    s.damping, s.inv_mass, s.rho = float(prm.damping), float(prm.inv_mass), float(prm.rho)
    s.eps, s.vel_half = float(prm.eps), float(prm.vel_half)
    s.clear_margin, s.clear_beta = float(prm.clear_margin), float(prm.clear_beta)
    s.ckpt_every = int(getattr(prm, "ckpt_every", 0))
    s.cost_radius = float(getattr(prm, "cost_radius", 0.05))
    return s


def alloc_rollout_out(n_agents: int, n_steps: int, want_traj=True, want_trace=False,
                      want_clear=True, device=None, want_cost4=False) -> dict:
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    f = lambda *s: torch.empty(*s, dtype=torch.float32, device=dev)  # noqa: E731
    out = {"p_final": f(3, n_agents), "v_final": f(3, n_agents), "path_len": f(n_agents),
           "clear_pen": f(n_agents) if want_clear else None,
           "min_clear": f(n_agents) if want_clear else None,
           "traj": f(n_agents, n_steps + 1, 3) if want_traj else None,
           "w_trace": f(n_agents, n_steps) if want_trace else None,
           "m_trace": f(n_agents, n_steps) if want_trace else None,
           "f_trace": f(n_agents, n_steps, 3) if want_trace else None,
           "ckpt": None, "cost_terms": f(5, n_agents) if want_cost4 else None,
           "n_agents": n_agents, "n_steps": n_steps}
    return out


def _out_struct(out: dict) -> _abi.RolloutOut:
    s = _abi.RolloutOut()
    for k in ("traj", "p_final", "v_final", "path_len", "clear_pen", "min_clear", "w_trace",
              "m_trace", "f_trace", "ckpt", "cost_terms", "heur_pairs"):
        t = out.get(k)
        setattr(s, k, t.data_ptr() if t is not None else None)
    return s


def pick_tuning(obs_cap: int, n_agents: int) -> tuple:
    t = _abi.Tuning()
    check(_abi.load().gmapp_pick_tuning(context().handle, int(obs_cap), int(n_agents),
                                        C.byref(t)), "gmapp_pick_tuning")
    return (t.cluster, t.agents_per_cta, t.threads, t.exchange)


def autotune_rollout(obs: Obstacles, agents: dict, prm, out: dict | None = None,
                     candidates: int = 12, probe_steps: int = 60, stream=None):
    """Measure up to ``candidates`` launch shapes on these inputs and cache
    the fastest for later rollouts of the same sizes; returns
    ((cluster, agents_per_cta, threads, exchange), ms scaled to the full
    horizon)."""
    ctx = context()
    na = int(agents["k_r"].numel())
    if out is None:
        out = alloc_rollout_out(na, int(prm.n_steps))
    ob, ag, pr, os_ = obs._struct(), _agents_struct(agents), _params_struct(prm), _out_struct(out)
    t = _abi.Tuning()
    ms = C.c_float()
    check(_abi.load().gmapp_autotune_rollout(ctx.handle, C.byref(ob), C.byref(ag), C.byref(pr),
                                             C.byref(os_), int(candidates), int(probe_steps),
                                             C.byref(t), C.byref(ms), _stream(stream)),
          "gmapp_autotune_rollout")
    return (t.cluster, t.agents_per_cta, t.threads, t.exchange), float(ms.value)


def autotune_ensemble(obs: Obstacles, agents: dict, n_apf: int, prm, out: dict | None = None,
                      candidates: int = 12, probe_steps: int = 60, stream=None, n_proj: int = 0):
    """autotune_rollout for an ensemble whose last ``n_apf`` agents use APF;
    later rollout_ensemble calls of the same sizes without ``tuning`` use
    the shape it caches."""
    ctx = context()
    na = int(agents["k_r"].numel())
    if out is None:
        out = alloc_rollout_out(na, int(prm.n_steps))
    ob, ag, pr, os_ = obs._struct(), _agents_struct(agents), _params_struct(prm), _out_struct(out)
    t = _abi.Tuning()
    ms = C.c_float()
    check(_abi.load().gmapp_autotune_ensemble(ctx.handle, C.byref(ob), C.byref(ag), int(n_proj),
                                              int(n_apf),
                                              C.byref(pr), C.byref(os_), int(candidates),
                                              int(probe_steps), C.byref(t), C.byref(ms),
                                              _stream(stream)),
          "gmapp_autotune_ensemble")
    return (t.cluster, t.agents_per_cta, t.threads, t.exchange), float(ms.value)


def rollout_agents(obs: Obstacles, agents: dict, prm, out: dict | None = None,
                   want_traj: bool = True, want_trace: bool = False, want_clear: bool = True,
                   tuning=None, stream=None) -> dict:
    """Roll every agent N_k steps in one launch (Sec. IV-A, Eq. mfi, Alg. 1).

    ``agents``: dict of contiguous float32 CUDA tensors p0, v0, c [3, N_a] and
    k_r, k_a, r_d, r_a [N_a].  ``prm``: object with goal, dt, n_steps,
    damping, inv_mass, rho, eps, vel_half, clear_margin, clear_beta.
    ``tuning``: optional (cluster, agents_per_cta, threads[, exchange]);
    exchange 0 = cluster/DSMEM (default), 1 = cooperative grid."""
    ctx = context()
    na = int(agents["k_r"].numel())
    if out is None:
        out = alloc_rollout_out(na, int(prm.n_steps), want_traj, want_trace, want_clear)
    ob, ag, pr, os_ = obs._struct(), _agents_struct(agents), _params_struct(prm), _out_struct(out)
    lib = _abi.load()
    if tuning is None:
        st = lib.rollout_agents(ctx.handle, C.byref(ob), C.byref(ag), C.byref(pr), C.byref(os_),
                                _stream(stream))
    else:
        t = _abi.Tuning(*[int(v) for v in tuning])
        st = lib.rollout_agents_tuned(ctx.handle, C.byref(ob), C.byref(ag), C.byref(pr),
                                      C.byref(os_), C.byref(t), _stream(stream))
    check(st, "rollout_agents")
    return out


def rollout_agents_blockcull(obs: Obstacles, agents: dict, prm, out: dict | None = None,
                             want_traj: bool = True, want_trace: bool = False,
                             want_clear: bool = True, tuning=None, stream=None) -> dict:
    """rollout_agents visiting, each step, only the blocks of 128
    key-sorted obstacles whose bounding box lies within an agent's gate
    (spatial culling, Alg. 1's gate); W and the trajectories equal
    rollout_agents' at the same launch shape bit for bit."""
    ctx = context()
    na = int(agents["k_r"].numel())
    if out is None:
        out = alloc_rollout_out(na, int(prm.n_steps), want_traj, want_trace, want_clear)
    ob, ag, pr, os_ = obs._struct(), _agents_struct(agents), _params_struct(prm), _out_struct(out)
    t = _abi.Tuning(*[int(v) for v in tuning]) if tuning is not None else None
    check(_abi.load().rollout_agents_blockcull(ctx.handle, C.byref(ob), C.byref(ag), C.byref(pr),
                                               C.byref(os_), C.byref(t) if t is not None else None,
                                               _stream(stream)), "rollout_agents_blockcull")
    return out


def rollout_ensemble(obs: Obstacles, agents: dict, n_apf: int, prm, out: dict | None = None,
                     want_traj: bool = True, want_trace: bool = False, want_clear: bool = True,
                     tuning=None, stream=None, n_proj: int = 0, cull: bool = False) -> dict:
    """Heterogeneous ensemble in one launch: the last ``n_apf`` agents follow
    the APF heuristic (Eq. apf), the ``n_proj`` before them MFI with the
    per-obstacle projected current, the others the MFI field with their own
    current (Eq. mfi); agent groups are homogeneous.  Arguments and outputs
    as rollout_agents.  ``cull``: rollout_ensemble_blockcull (each group
    visits only the obstacle blocks whose bounding box meets a gate; the same
    forces and trajectories bit for bit)."""
    ctx = context()
    na = int(agents["k_r"].numel())
    if out is None:
        out = alloc_rollout_out(na, int(prm.n_steps), want_traj, want_trace, want_clear)
    ob, ag, pr, os_ = obs._struct(), _agents_struct(agents), _params_struct(prm), _out_struct(out)
    t = C.byref(_abi.Tuning(*[int(v) for v in tuning])) if tuning is not None else None
    lib = _abi.load()
    fn, name = ((lib.rollout_ensemble_blockcull, "rollout_ensemble_blockcull") if cull
                else (lib.rollout_ensemble, "rollout_ensemble"))
    check(fn(ctx.handle, C.byref(ob), C.byref(ag), int(n_proj), int(n_apf), C.byref(pr),
             C.byref(os_), t, _stream(stream)), name)
    return out


def grid_index(obs: Obstacles, ws, index=None, stream=None):
    """Neighbour index of ``obs`` on the grid ``ws`` (device uint32 tensor
    [ceil(cells/32) + 1]) for rollout_agents_culled."""
    torch = _torch()
    ctx = context()
    wss = _ws_struct(ws)
    lib = _abi.load()
    need = int(lib.gmapp_grid_index_bytes(C.byref(wss)))
    if index is None or index.numel() * 4 < need:
        index = torch.empty(need // 4, dtype=torch.int32, device=obs.x.device)
    ob = obs._struct()
    check(lib.gmapp_grid_index(ctx.handle, C.byref(ob), C.byref(wss), _ptr(index),
                               int(index.numel() * 4), _stream(stream)), "gmapp_grid_index")
    return index


def rollout_agents_culled(obs: Obstacles, ws, index, agents: dict, prm, out: dict | None = None,
                          want_traj: bool = True, want_trace: bool = False,
                          want_clear: bool = True, stream=None) -> dict:
    """rollout_agents visiting only the obstacles within each agent's gate
    (the voxel grid ``ws`` of ``obs`` as a neighbour grid; ``index`` from
    grid_index)."""
    ctx = context()
    na = int(agents["k_r"].numel())
    if out is None:
        out = alloc_rollout_out(na, int(prm.n_steps), want_traj, want_trace, want_clear)
        out["f_trace"] = None
    ob, ag, pr, os_ = obs._struct(), _agents_struct(agents), _params_struct(prm), _out_struct(out)
    wss = _ws_struct(ws)
    check(_abi.load().rollout_agents_culled(ctx.handle, C.byref(ob), C.byref(wss), _ptr(index),
                                            C.byref(ag), C.byref(pr), C.byref(os_),
                                            _stream(stream)), "rollout_agents_culled")
    return out


def score_and_select(ro: dict, prm, weights=None, prev_best_cost: float = math.nan,
                     alpha: float = 1.0, best_traj: bool = True, out: dict | None = None,
                     stream=None) -> dict:
    """Costs C_i and the selected agent i* (Sec. IV-A cost and selection).
    Returns device tensors ``costs`` [N_a], ``best`` [1] (int32, -1 = keep
    the previous path) and ``best_traj`` [N_k+1, 3]."""
    torch = _torch()
    ctx = context()
    na = int(ro["p_final"].shape[1])
    dev = ro["p_final"].device
    if out is None:
        out = {"costs": torch.empty(na, dtype=torch.float32, device=dev),
               "best": torch.empty(1, dtype=torch.int32, device=dev),
               "best_traj": (torch.empty(int(prm.n_steps) + 1, 3, dtype=torch.float32, device=dev)
                             if best_traj and ro.get("traj") is not None else None)}
    w = weights if weights is not None else prm
    cw = _abi.CostWeights(float(w.w_path), float(w.w_goal), float(w.w_clear))
    os_, pr = _out_struct(ro), _params_struct(prm)
    check(_abi.load().score_and_select(ctx.handle, C.byref(os_), na, C.byref(pr), C.byref(cw),
                                       float(prev_best_cost), float(alpha), _ptr(out["costs"]),
                                       _ptr(out["best"]), _ptr(out.get("best_traj")),
                                       _stream(stream)), "score_and_select")
    return out


def score_and_select4(ro: dict, prm, c_best=None, alpha: float = 1.0, best_traj: bool = True,
                      out: dict | None = None, stream=None) -> dict:
    """The paper's four-term cost (Eq. cost_function) from ``ro["cost_terms"]``
    (a rollout with ``want_cost4``) and the selection against the cost of
    the current plan: ``c_best`` is a device float32 tensor [1] (NaN = no
    plan), updated in place when an agent is selected; None = plain argmin.
    Weights from prm.w4 = (w_goal, w_obs, w_path, w_smooth) and prm.a_max."""
    torch = _torch()
    ctx = context()
    na = int(ro["p_final"].shape[1])
    dev = ro["p_final"].device
    if out is None:
        out = {"costs": torch.empty(na, dtype=torch.float32, device=dev),
               "best": torch.empty(1, dtype=torch.int32, device=dev),
               "best_traj": (torch.empty(int(prm.n_steps) + 1, 3, dtype=torch.float32, device=dev)
                             if best_traj and ro.get("traj") is not None else None)}
    w4 = tuple(float(v) for v in prm.w4)
    cw = _abi.Cost4(w4[0], w4[1], w4[2], w4[3], float(prm.a_max))
    os_, pr = _out_struct(ro), _params_struct(prm)
    check(_abi.load().score_and_select4(ctx.handle, C.byref(os_), na, C.byref(pr), C.byref(cw),
                                        _ptr(c_best), float(alpha), _ptr(out["costs"]),
                                        _ptr(out["best"]), _ptr(out.get("best_traj")),
                                        _stream(stream)), "score_and_select4")
    return out


# ---------------------------------------------------------------------------
# Differentiable rollout
# ---------------------------------------------------------------------------

def rollout_adjoint(obs: Obstacles, agents: dict, prm, ckpt, grad_cost=None, weights=None,
                    want_cost: bool = False, workspace=None, stream=None) -> dict:
    """dC_i/d(v0, k_r, k_a, c) by the adjoint kernel, from the checkpoints of
    a forward rollout_agents call (``out["ckpt"]`` with prm.ckpt_every = K).
    ``grad_cost`` ([N_a], device) scales each agent's gradient."""
    torch = _torch()
    ctx = context()
    na = int(agents["k_r"].numel())
    dev = agents["k_r"].device
    f = lambda *s: torch.empty(*s, dtype=torch.float32, device=dev)  # noqa: E731
    out = {"g_v0": f(3, na), "g_kr": f(na), "g_ka": f(na), "g_c": f(3, na),
           "cost": f(na) if want_cost else None}
    pr = _params_struct(prm)
    need = int(_abi.load().gmapp_adjoint_workspace_bytes(na, C.byref(pr)))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    w = weights if weights is not None else prm
    cw = _abi.CostWeights(float(w.w_path), float(w.w_goal), float(w.w_clear))
    ao = _abi.AdjointOut(*[out[k].data_ptr() if out[k] is not None else None
                           for k in ("g_v0", "g_kr", "g_ka", "g_c", "cost")])
    if grad_cost is not None:
        grad_cost = grad_cost.to(dtype=torch.float32).contiguous()
    check(_abi.load().rollout_adjoint(ctx.handle, C.byref(obs._struct()), C.byref(_agents_struct(agents)),
                                      C.byref(pr), C.byref(cw), _ptr(ckpt), _ptr(grad_cost),
                                      C.byref(ao), _ptr(workspace), int(workspace.numel()),
                                      _stream(stream)), "rollout_adjoint")
    return out


def _autograd_function():
    torch = _torch()

    class GMappRollout(torch.autograd.Function):
        """costs = GMappRollout.apply(v0, k_r, k_a, c, obstacles, agents, prm)

        Forward: rollout_agents with checkpoints every prm.ckpt_every steps,
        then the per-agent plan cost C_i (score_and_select).  Backward:
        rollout_adjoint with grad_cost = dLoss/dC_i, giving gradients for
        v0 [3, N_a], k_r, k_a [N_a] and c [3, N_a].  ``agents`` supplies the
        remaining agent arrays (p0, r_d, r_a)."""

        @staticmethod
        def forward(fctx, v0, k_r, k_a, c, obstacles, agents, prm):
            ag = dict(agents)
            ag.update(v0=v0.detach().contiguous(), k_r=k_r.detach().contiguous(),
                      k_a=k_a.detach().contiguous(), c=c.detach().contiguous())
            na, K = int(k_r.numel()), int(prm.ckpt_every)
            out = alloc_rollout_out(na, int(prm.n_steps), want_traj=True,
                                    want_clear=float(prm.w_clear) != 0.0)
            out["ckpt"] = torch.empty((int(prm.n_steps) + K - 1) // K, 6, na,
                                      dtype=torch.float32, device=v0.device)
            rollout_agents(obstacles, ag, prm, out=out)
            sel = score_and_select(out, prm, best_traj=False)
            fctx.save_for_backward(out["ckpt"])
            fctx.obstacles, fctx.agents, fctx.prm = obstacles, ag, prm
            return sel["costs"].clone()

        @staticmethod
        def backward(fctx, grad_costs):
            (ckpt,) = fctx.saved_tensors
            g = rollout_adjoint(fctx.obstacles, fctx.agents, fctx.prm, ckpt,
                                grad_cost=grad_costs.contiguous())
            return g["g_v0"], g["g_kr"], g["g_ka"], g["g_c"], None, None, None

    return GMappRollout


_GMappRollout = None


def __getattr__(name):
    global _GMappRollout
    if name == "GMappRollout":
        if _GMappRollout is None:
            _GMappRollout = _autograd_function()
        return _GMappRollout
    raise AttributeError(name)


# ---------------------------------------------------------------------------
# Batched uneven queries
# ---------------------------------------------------------------------------

class FilterBatch:
    """Many clouds through one batched filter (waves of clouds whose scratch
    fits in L2, three launches per wave on the batch's streams; results
    bit-identical to filter_cloud per cloud).  ``clouds``: list of
    device [N, 3] float32 tensors (kept, not copied: refill them in place
    between runs); ``T`` and ``ws`` are shared by all clouds, or lists of one
    per cloud.  ``outs[q]`` is cloud q's obstacle set after run()."""

    def __init__(self, clouds: list, T, ws, caps=None):
        ctx = context()
        n = len(clouds)
        import numpy as np
        Ts = list(T) if np.ndim(T) == 2 else [T] * n
        wss = ws if isinstance(ws, (list, tuple)) else [ws] * n
        self._keep = list(clouds)
        self.outs = []
        arr = (_abi.CloudJob * n)()
        for q, xyz in enumerate(clouds):
            cap = int(caps[q]) if caps is not None else max(4, (int(xyz.shape[0]) + 3) // 4 * 4)
            out = Obstacles.empty(cap)
            out.r_O = 0.5 * float(wss[q].voxel)
            self.outs.append(out)
            J = arr[q]
            J.xyz = xyz.data_ptr()
            J.n_raw = int(xyz.shape[0])
            for i, v in enumerate(list(Ts[q])):
                J.T[i] = float(v)
            J.ws = _ws_struct(wss[q])
            J.out = out._struct()
        h = C.c_void_p()
        check(_abi.load().gmapp_filter_batch_create(ctx.handle, arr, n, C.byref(h)),
              "gmapp_filter_batch_create")
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _abi._lib is not None:
            _abi._lib.gmapp_filter_batch_destroy(h)
            self.handle = None

    def run(self, stream=None) -> None:
        check(_abi.load().filter_cloud_batch(self.handle, _stream(stream)), "filter_cloud_batch")


class Batch:
    """Many planning queries through one fixed launch sequence (batched
    filter, planner, one persistent rollout launch, batched select), with
    optional CUDA-graph replay and an autotuner of the work-item size.

    ``queries``: list of dicts with ``xyz`` (device [N, 3] float32), ``T``,
    ``ws``, ``agents`` (device arrays), ``prm`` and optionally ``obs_cap``
    (default: the raw point count rounded up to 4), ``want_traj`` and
    ``cost4`` (score by the paper's four-term cost with prm.w4, prm.a_max,
    prm.cost_radius; ``alpha`` and ``c_best``, a device float32 tensor [1]
    holding the current plan's cost, give the selection's hysteresis).
    Outputs are allocated here; ``results[q]`` holds the query's obstacle
    set, rollout outputs, ``costs``, ``best`` and ``best_traj``."""

    def __init__(self, queries: list, want_traj: bool = True, want_clear: bool = False):
        torch = _torch()
        ctx = context()
        self._keep = []
        self.results = []
        arr = (_abi.Query * len(queries))()
        for q, spec in enumerate(queries):
            xyz = spec["xyz"]
            prm = spec["prm"]
            na = int(spec["agents"]["k_r"].numel())
            cap = int(spec.get("obs_cap", max(4, (int(xyz.shape[0]) + 3) // 4 * 4)))
            obs = Obstacles.empty(cap)
            obs.r_O = 0.5 * float(spec["ws"].voxel)
            cost4 = bool(spec.get("cost4", False))
            out = alloc_rollout_out(na, int(prm.n_steps), want_traj=spec.get("want_traj", want_traj),
                                    want_clear=want_clear, want_cost4=cost4)
            dev = xyz.device
            res = {"obs": obs, "out": out, "costs": torch.empty(na, dtype=torch.float32, device=dev),
                   "best": torch.empty(1, dtype=torch.int32, device=dev),
                   "best_traj": (torch.empty(int(prm.n_steps) + 1, 3, dtype=torch.float32, device=dev)
                                 if out["traj"] is not None else None)}
            self.results.append(res)
            self._keep.append((xyz, spec["agents"]))
            Q = arr[q]
            Q.xyz = xyz.data_ptr()
            Q.n_raw = int(xyz.shape[0])
            for i, v in enumerate(list(spec["T"])):
                Q.T[i] = float(v)
            Q.ws = _ws_struct(spec["ws"])
            Q.agents = _agents_struct(spec["agents"])
            Q.prm = _params_struct(prm)
            Q.w = _abi.CostWeights(float(prm.w_path), float(prm.w_goal), float(prm.w_clear))
            Q.obs = obs._struct()
            Q.out = _out_struct(out)
            Q.costs = res["costs"].data_ptr()
            Q.best = res["best"].data_ptr()
            Q.best_traj = res["best_traj"].data_ptr() if res["best_traj"] is not None else None
            if cost4:
                w4 = tuple(float(v) for v in prm.w4)
                Q.w4 = _abi.Cost4(w4[0], w4[1], w4[2], w4[3], float(prm.a_max))
                Q.alpha = float(spec.get("alpha", 1.0))
                cb = spec.get("c_best")
                Q.c_best = cb.data_ptr() if cb is not None else None
                self._keep.append(cb)
        h = C.c_void_p()
        check(_abi.load().gmapp_batch_create(ctx.handle, arr, len(queries), C.byref(h)),
              "gmapp_batch_create")
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _abi._lib is not None:
            _abi._lib.gmapp_batch_destroy(h)
            self.handle = None

    def run(self, stream=None) -> None:
        check(_abi.load().rollout_batch(self.handle, _stream(stream)), "rollout_batch")

    def launch_graph(self, stream) -> None:
        check(_abi.load().gmapp_batch_launch_graph(self.handle, _stream(stream)),
              "gmapp_batch_launch_graph")

    def set_tuning(self, agents_per_item: int, threads: int) -> None:
        check(_abi.load().gmapp_batch_set_tuning(self.handle, int(agents_per_item), int(threads)),
              "gmapp_batch_set_tuning")

    def set_culling(self, on: bool) -> None:
        """Block culling in the rollout kernel (results unchanged)."""
        check(_abi.load().gmapp_batch_set_culling(self.handle, int(bool(on))),
              "gmapp_batch_set_culling")

    def autotune(self, stream=None):
        t = _abi.Tuning()
        ms = C.c_float()
        check(_abi.load().gmapp_batch_autotune(self.handle, _stream(stream), C.byref(t), C.byref(ms)),
              "gmapp_batch_autotune")
        return (t.agents_per_cta, t.threads), float(ms.value)


# ---------------------------------------------------------------------------
# Served control loop (continuous batching)
# ---------------------------------------------------------------------------

def _host_ptr(a):
    """Address of a contiguous float32 host array (numpy or CPU torch)."""
    import numpy as np
    if hasattr(a, "data_ptr"):
        if a.is_cuda or not a.is_contiguous() or str(a.dtype) != "torch.float32":
            raise ValueError("request arrays must be contiguous float32 host tensors")
        return a.data_ptr()
    if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]):
        raise ValueError("request arrays must be contiguous float32 host arrays")
    return a.ctypes.data


class Server:
    """Control-rate request server: requests (host clouds and agents) are
    admitted as arena memory frees up, advanced M steps per tick together in
    one launch, scored and returned; see include/gmapp.h.  ``culled``:
    False (all pairs), True (voxel-grid culling, one agent per work item) or
    "blocks" (block culling in the chunk kernel; results equal all pairs)."""

    def __init__(self, max_slots=16, max_agents=1024, max_steps=300, obs_cap=32768,
                 arena_bytes=4 << 30, chunk_steps=50, agents_per_item=8, threads=256,
                 culled=False, admit_bypass=0, four_term=False, max_plan_streams=0):
        """``admit_bypass``: 0 admits in arrival order; k > 0 first fit over
        the queue with an aging bound of k overtakes.  ``four_term``: the
        chunk kernel computes the clearance and the four-term cost sums, so
        requests may use ``cost4=True``; ``max_plan_streams`` C_best slots
        on the device for request streams (``plan_stream``)."""
        ctx = context()
        cfg = _abi.ServerConfig(int(max_slots), int(max_agents), int(max_steps), int(obs_cap),
                                int(arena_bytes), int(chunk_steps), int(agents_per_item),
                                int(threads), 2 if culled == "blocks" else int(bool(culled)),
                                int(admit_bypass), int(bool(four_term)), int(max_plan_streams))
        h = C.c_void_p()
        check(_abi.load().gmapp_server_create(ctx.handle, C.byref(cfg), C.byref(h)),
              "gmapp_server_create")
        self.handle = h
        self._keep = {}

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _abi._lib is not None:
            _abi._lib.gmapp_server_destroy(h)
            self.handle = None

    def submit(self, xyz, T, ws, agents: dict, prm, cost4: bool = False, alpha: float = 1.0,
               plan_stream: int = -1) -> int:
        """Queue a request.  ``cost4``: score with the paper's four-term cost
        (weights prm.w4, prm.a_max, radius prm.cost_radius) and select against
        the C_best of request stream ``plan_stream`` with hysteresis ``alpha``
        (-1: plain argmin); needs a server created with four_term=True."""
        r = _abi.Request()
        r.xyz = _host_ptr(xyz)
        r.n_raw = int(xyz.shape[0])
        for i, v in enumerate(list(T)):
            r.T[i] = float(v)
        r.ws = _ws_struct(ws)
        for k in AGENT_KEYS:
            setattr(r, k, _host_ptr(agents[k]))
        r.n_agents = int(agents["k_r"].shape[0])
        r.prm = _params_struct(prm)
        r.w = _abi.CostWeights(float(prm.w_path), float(prm.w_goal), float(prm.w_clear))
        r.cost_mode = 1 if cost4 else 0
        if cost4:
            w4 = tuple(float(v) for v in prm.w4)
            r.w4 = _abi.Cost4(w4[0], w4[1], w4[2], w4[3], float(prm.a_max))
            r.alpha = float(alpha)
            r.plan_stream = int(plan_stream)
        else:
            r.plan_stream = -1
        t = C.c_int64()
        check(_abi.load().gmapp_server_submit(self.handle, C.byref(r), C.byref(t)),
              "gmapp_server_submit")
        self._keep[t.value] = (xyz, agents, int(prm.n_steps))
        return int(t.value)

    def tick(self) -> int:
        n = C.c_int32()
        check(_abi.load().gmapp_server_tick(self.handle, C.byref(n)), "gmapp_server_tick")
        return int(n.value)

    def poll(self, ticket: int):
        """None until done, then a dict with the selected agent, its cost, the
        costs, the chosen trajectory [N_k+1, 3], N_O and timestamps."""
        import numpy as np
        res = _abi.Result()
        st = _abi.load().gmapp_server_poll(self.handle, int(ticket), C.byref(res))
        if st == _abi.ERR_NOT_READY:
            return None
        check(st, "gmapp_server_poll")
        _, agents, nk = self._keep[ticket]
        na = int(agents["k_r"].shape[0])
        return {"best": int(res.best), "best_cost": float(res.best_cost), "n_obs": int(res.n_obs),
                "best_traj": np.ctypeslib.as_array(res.best_traj, shape=((nk + 1) * 3,)).reshape(-1, 3).copy(),
                "costs": np.ctypeslib.as_array(res.costs, shape=(na,)).copy(),
                "t_submit": res.t_submit, "t_admit": res.t_admit, "t_done": res.t_done}

    def release(self, ticket: int) -> None:
        check(_abi.load().gmapp_server_release(self.handle, int(ticket)), "gmapp_server_release")
        self._keep.pop(ticket, None)

    def stats(self) -> dict:
        s = _abi.ServerStats()
        check(_abi.load().gmapp_server_stats(self.handle, C.byref(s)), "gmapp_server_stats")
        return {"active": s.active, "pending": s.pending, "completed": s.completed,
                "arena_free_bytes": s.arena_free_bytes, "shard_cap": s.shard_cap}
