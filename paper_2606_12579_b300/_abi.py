"""ctypes mirror of include/gmapp.h (and include/gmapp_peaks.h): structures, status codes, prototypes.

Loading the library needs no GPU (the CUDA runtime is linked statically and
binds to the driver on the first CUDA call); every compute call does.
"""

from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# GMAPP_BOUNDS_CHECK=1 selects the bounds-checked build (index checks that
# set GMAPP_DEVERR_BOUNDS; see build.py)
LIB_PATH = os.path.join(HERE, "libgmapp_bc.so" if os.environ.get("GMAPP_BOUNDS_CHECK") == "1"
                        else "libgmapp.so")

OK, ERR_INVALID_ARG, ERR_CAPACITY, ERR_CUDA, ERR_TIMEOUT, ERR_NOT_READY = range(6)
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CAPACITY", 3: "CUDA", 4: "TIMEOUT", 5: "NOT_READY"}
DEVERR_CAPACITY, DEVERR_TIMEOUT, DEVERR_BOUNDS = 0x1, 0x2, 0x4

P = C.c_void_p


class Workspace(C.Structure):
    _fields_ = [("lo", C.c_float * 3), ("voxel", C.c_float), ("dims", C.c_int32 * 3),
                ("min_pts", C.c_int32)]


class Obstacles(C.Structure):
    _fields_ = [("x", P), ("y", P), ("z", P), ("keys", P), ("counts", P), ("rep_idx", P),
                ("n", P), ("cap", C.c_int64), ("r_O", C.c_float)]


class SensorCloud(C.Structure):
    _fields_ = [("xyz", P), ("n_raw", C.c_int64), ("T", C.c_float * 12)]


class CloudJob(C.Structure):
    _fields_ = [("xyz", P), ("n_raw", C.c_int64), ("T", C.c_float * 12), ("ws", Workspace),
                ("out", Obstacles)]


class Agents(C.Structure):
    _fields_ = [("p0", P), ("v0", P), ("c", P), ("k_r", P), ("k_a", P), ("r_d", P), ("r_a", P),
                ("n", C.c_int32)]


class RolloutParams(C.Structure):
    _fields_ = [("goal", C.c_float * 3), ("dt", C.c_float), ("n_steps", C.c_int32),
                ("damping", C.c_float), ("inv_mass", C.c_float), ("rho", C.c_float),
                ("eps", C.c_float), ("vel_half", C.c_float), ("clear_margin", C.c_float),
                ("clear_beta", C.c_float), ("ckpt_every", C.c_int32), ("cost_radius", C.c_float)]


class RolloutOut(C.Structure):
    _fields_ = [("traj", P), ("p_final", P), ("v_final", P), ("path_len", P), ("clear_pen", P),
                ("min_clear", P), ("w_trace", P), ("m_trace", P), ("f_trace", P), ("ckpt", P),
                ("cost_terms", P), ("heur_pairs", P)]


class AdjointOut(C.Structure):
    _fields_ = [("g_v0", P), ("g_kr", P), ("g_ka", P), ("g_c", P), ("cost", P)]


class Tuning(C.Structure):
    _fields_ = [("cluster", C.c_int32), ("agents_per_cta", C.c_int32), ("threads", C.c_int32),
                ("exchange", C.c_int32)]


class CostWeights(C.Structure):
    _fields_ = [("w_path", C.c_float), ("w_goal", C.c_float), ("w_clear", C.c_float)]


class Cost4(C.Structure):
    _fields_ = [("w_goal", C.c_float), ("w_obs", C.c_float), ("w_path", C.c_float),
                ("w_smooth", C.c_float), ("a_max", C.c_float)]


class Query(C.Structure):
    _fields_ = [("xyz", P), ("n_raw", C.c_int64), ("T", C.c_float * 12), ("ws", Workspace),
                ("agents", Agents), ("prm", RolloutParams), ("w", CostWeights),
                ("obs", Obstacles), ("out", RolloutOut), ("costs", P), ("best", P),
                ("best_traj", P), ("w4", Cost4), ("alpha", C.c_float), ("c_best", P)]


class ServerConfig(C.Structure):
    _fields_ = [("max_slots", C.c_int32), ("max_agents", C.c_int32), ("max_steps", C.c_int32),
                ("obs_cap", C.c_int64), ("arena_bytes", C.c_int64), ("chunk_steps", C.c_int32),
                ("agents_per_item", C.c_int32), ("threads", C.c_int32), ("culled", C.c_int32),
                ("admit_bypass", C.c_int32), ("four_term", C.c_int32),
                ("max_plan_streams", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("xyz", P), ("n_raw", C.c_int64), ("T", C.c_float * 12), ("ws", Workspace),
                ("p0", P), ("v0", P), ("c", P), ("k_r", P), ("k_a", P), ("r_d", P), ("r_a", P),
                ("n_agents", C.c_int32), ("prm", RolloutParams), ("w", CostWeights),
                ("cost_mode", C.c_int32), ("w4", Cost4), ("alpha", C.c_float),
                ("plan_stream", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("done", C.c_int32), ("best", C.c_int32), ("best_cost", C.c_float),
                ("n_obs", C.c_int32), ("best_traj", C.POINTER(C.c_float)),
                ("costs", C.POINTER(C.c_float)), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double)]


class Peaks(C.Structure):
    """gmapp_peaks (include/gmapp_peaks.h)."""
    _fields_ = [("fp32_tflops", C.c_double), ("fp32_tflops_scalar", C.c_double),
                ("fma_lanes_per_clk_sm", C.c_double), ("fma_lanes_per_clk_sm_scalar", C.c_double),
                ("sfu_lanes_per_clk_sm", C.c_double), ("sfu_gops", C.c_double),
                ("mix_fma_busy", C.c_double), ("mix_sfu_busy", C.c_double),
                ("sm_mhz", C.c_double), ("sm_count", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("active", C.c_int32), ("pending", C.c_int32), ("completed", C.c_int64),
                ("arena_free_bytes", C.c_int64), ("shard_cap", C.c_int32)]


# name -> (restype, argtypes); every entry point declared in include/gmapp.h
PROTOTYPES = {
    "gmapp_create": (C.c_int, [C.POINTER(P), C.c_int]),
    "gmapp_destroy": (None, [P]),
    "gmapp_last_error": (C.c_char_p, []),
    "gmapp_sync": (C.c_int, [P, P]),
    "gmapp_set_wait_limit": (C.c_int, [P, C.c_uint32]),
    "gmapp_peek_device_error": (C.c_int, [P, C.POINTER(C.c_uint32)]),
    "gmapp_filter_workspace_bytes": (C.c_size_t, [C.c_int64, C.POINTER(Workspace)]),
    "filter_cloud": (C.c_int, [P, P, C.c_int64, C.POINTER(C.c_float * 12), C.POINTER(Workspace),
                               C.POINTER(Obstacles), P, C.c_size_t, P]),
    "gmapp_filter_clouds_workspace_bytes": (C.c_size_t, [C.POINTER(SensorCloud), C.c_int32,
                                                         C.POINTER(Workspace)]),
    "filter_clouds": (C.c_int, [P, C.POINTER(SensorCloud), C.c_int32, C.POINTER(Workspace),
                                C.POINTER(Obstacles), P, C.c_size_t, P]),
    "filter_cloud_noalloc": (C.c_int, [P, C.c_int64, C.POINTER(C.c_float * 12),
                                       C.POINTER(Workspace), C.POINTER(Obstacles), P]),
    "filter_cloud_noalloc_status": (C.c_int, [P]),
    "gmapp_measure_peaks": (C.c_int, [C.c_int32, C.POINTER(Peaks)]),
    "rollout_agents": (C.c_int, [P, C.POINTER(Obstacles), C.POINTER(Agents),
                                 C.POINTER(RolloutParams), C.POINTER(RolloutOut), P]),
    "rollout_agents_tuned": (C.c_int, [P, C.POINTER(Obstacles), C.POINTER(Agents),
                                       C.POINTER(RolloutParams), C.POINTER(RolloutOut),
                                       C.POINTER(Tuning), P]),
    "rollout_ensemble_blockcull": (C.c_int, [P, C.POINTER(Obstacles), C.POINTER(Agents),
                                             C.c_int32, C.c_int32, C.POINTER(RolloutParams),
                                             C.POINTER(RolloutOut), C.POINTER(Tuning), P]),
    "rollout_agents_blockcull": (C.c_int, [P, C.POINTER(Obstacles), C.POINTER(Agents),
                                           C.POINTER(RolloutParams), C.POINTER(RolloutOut),
                                           C.POINTER(Tuning), P]),
    "rollout_ensemble": (C.c_int, [P, C.POINTER(Obstacles), C.POINTER(Agents), C.c_int32, C.c_int32,
                                   C.POINTER(RolloutParams), C.POINTER(RolloutOut),
                                   C.POINTER(Tuning), P]),
    "gmapp_pick_tuning": (C.c_int, [P, C.c_int64, C.c_int32, C.POINTER(Tuning)]),
    "gmapp_grid_index_bytes": (C.c_size_t, [C.POINTER(Workspace)]),
    "gmapp_grid_index": (C.c_int, [P, C.POINTER(Obstacles), C.POINTER(Workspace), P, C.c_size_t, P]),
    "rollout_agents_culled": (C.c_int, [P, C.POINTER(Obstacles), C.POINTER(Workspace), P,
                                        C.POINTER(Agents), C.POINTER(RolloutParams),
                                        C.POINTER(RolloutOut), P]),
    "gmapp_autotune_rollout": (C.c_int, [P, C.POINTER(Obstacles), C.POINTER(Agents),
                                         C.POINTER(RolloutParams), C.POINTER(RolloutOut),
                                         C.c_int32, C.c_int32, C.POINTER(Tuning),
                                         C.POINTER(C.c_float), P]),
    "gmapp_autotune_ensemble": (C.c_int, [P, C.POINTER(Obstacles), C.POINTER(Agents), C.c_int32,
                                          C.c_int32,
                                          C.POINTER(RolloutParams), C.POINTER(RolloutOut),
                                          C.c_int32, C.c_int32, C.POINTER(Tuning),
                                          C.POINTER(C.c_float), P]),
    "gmapp_adjoint_workspace_bytes": (C.c_size_t, [C.c_int32, C.POINTER(RolloutParams)]),
    "rollout_adjoint": (C.c_int, [P, C.POINTER(Obstacles), C.POINTER(Agents),
                                  C.POINTER(RolloutParams), C.POINTER(CostWeights), P, P,
                                  C.POINTER(AdjointOut), P, C.c_size_t, P]),
    "gmapp_filter_batch_create": (C.c_int, [P, C.POINTER(CloudJob), C.c_int32, C.POINTER(P)]),
    "gmapp_filter_batch_destroy": (None, [P]),
    "filter_cloud_batch": (C.c_int, [P, P]),
    "gmapp_batch_create": (C.c_int, [P, C.POINTER(Query), C.c_int32, C.POINTER(P)]),
    "gmapp_batch_destroy": (None, [P]),
    "gmapp_batch_set_tuning": (C.c_int, [P, C.c_int32, C.c_int32]),
    "gmapp_batch_set_culling": (C.c_int, [P, C.c_int32]),
    "rollout_batch": (C.c_int, [P, P]),
    "gmapp_batch_launch_graph": (C.c_int, [P, P]),
    "gmapp_batch_autotune": (C.c_int, [P, P, C.POINTER(Tuning), C.POINTER(C.c_float)]),
    "gmapp_server_create": (C.c_int, [P, C.POINTER(ServerConfig), C.POINTER(P)]),
    "gmapp_server_destroy": (None, [P]),
    "gmapp_server_submit": (C.c_int, [P, C.POINTER(Request), C.POINTER(C.c_int64)]),
    "gmapp_server_tick": (C.c_int, [P, C.POINTER(C.c_int32)]),
    "gmapp_server_poll": (C.c_int, [P, C.c_int64, C.POINTER(Result)]),
    "gmapp_server_release": (C.c_int, [P, C.c_int64]),
    "gmapp_server_stats": (C.c_int, [P, C.POINTER(ServerStats)]),
    "score_and_select": (C.c_int, [P, C.POINTER(RolloutOut), C.c_int32, C.POINTER(RolloutParams),
                                   C.POINTER(CostWeights), C.c_float, C.c_float, P, P, P, P]),
    "score_and_select4": (C.c_int, [P, C.POINTER(RolloutOut), C.c_int32, C.POINTER(RolloutParams),
                                    C.POINTER(Cost4), P, C.c_float, P, P, P, P]),
}

_lib = None


def load():
    """Load libgmapp.so and bind every prototype; raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with paper_2606_12579_b300/build.py "
                "(there is no CPU fallback)")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class GmappError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().gmapp_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int, where: str) -> None:
    if status != OK:
        raise GmappError(status, where)
