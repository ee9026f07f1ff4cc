#!/usr/bin/env python3
"""Benchmark of the B300 G-MAPP hot path.

One step = one planning query of the tabletop workload: a 640x480 depth
frame (307,200 points, 2 mm noise, 5% NaN) goes through filter_cloud
(workspace 1 x 1 x 0.8 m, 5 mm voxels -> N_O obstacles), rollout_agents
(256 agents x 500 steps under the circular field) and score_and_select.
The metric is agent-obstacle interactions per second, N_a * N_O * N_k per
step, over the whole job.  The inputs are a ring of distinct frames (sensor
noise and dropouts differ per frame) larger than L2, resident in HBM before
timing; ``e2e`` repeats the step through the same public calls with every
frame copied from pinned host memory and every chosen plan copied back, the
next frame's upload overlapping the current step on a copy stream (the
serial figure, one step at a time, is ``e2e.serial_value``; its per-step
wall times give ``latency_ms``).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs independent queries (replicas: the
path has no exchange step) on its own frames; the job time is the maximum
over ranks.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "agent-obstacle interactions/s (% FP32 peak) and p50/p99 plan latency vs plain rollout"
UNIT = "interactions/s"
FLOPS_PER_INTERACTION = 13      # 3 sub, 5 for |d|^2, rsqrt, mul, sub, rcp, accumulate
BLOCK_TEST_FLOPS = 6            # expanded distance |o|^2 - 2 p.o: 3 FMAs per pair
OBSTACLE_NORM_FLOPS = 5         # |o|^2 per obstacle and pass over a half-group
# APF pair (Eq. apf): 3 sub, 5 for |d|^2, rsqrt, 1/rho - 1/r_d, 3 mul for the
# coefficient, 3 accumulating FMAs (6); clamp/gate selects not counted
APF_FLOPS_PER_INTERACTION = 19
# projected-current MFI pair: 3 sub, 5 for |d|^2, rsqrt, 2 for s = |d|^2 r - R,
# rcp, 5 for t = d . v, 3 mul for a = w r^2 t, 4 accumulating FMAs (8)
PROJ_FLOPS_PER_INTERACTION = 28
ADJOINT_FLOPS_PER_INTERACTION = 26  # recompute 13 + grad W: 3 mul, 3 FMA, d(1/s) ~ 7
FP32_LANES_PER_SM = 128
OBS_CAP = 131072
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "rollout_tabletop_256x500.md")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_over_ranks(times, counts, ws, device):
    """Whole-job totals of a replicas-only run: every time is the maximum
    over ranks (the job ends with its slowest rank) and every count of work
    is the sum over ranks.  A single process returns its own values."""
    times, counts = [float(v) for v in times], [float(v) for v in counts]
    if ws <= 1:
        return times, counts
    import torch
    import torch.distributed as dist
    t = torch.tensor(times, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor(counts, dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return t.tolist(), c.tolist()


def _measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) == 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# Workload
# ---------------------------------------------------------------------------

def make_workload(n_frames: int, rank: int):
    import synth
    base = synth.tabletop_workload()           # scene, agents, params of the tabletop query
    frames = []
    for f in range(n_frames):
        w = synth.tabletop_workload(frame_seed=7_000_000 + 1000 * rank + f, n_agents=1, n_steps=1)
        frames.append(w["xyz"])
    return base, frames


def oracle_step(base, xyz, n_agents_sample: int):
    """The oracle on a bounded sample of one step: the full frame's filter,
    then n_agents_sample agents over all obstacles and all N_k steps."""
    import oracle
    f = oracle.filter_cloud(xyz, base["T"], base["workspace"])
    obs = np.stack([f["x"], f["y"], f["z"]])
    ag = {k: np.ascontiguousarray(v[..., :n_agents_sample]) for k, v in base["agents"].items()}
    ro = oracle.rollout(obs, f["r_O"], ag, base["params"], want_traj=True)
    c = oracle.costs(ro, base["params"])
    oracle.select(c)
    return n_agents_sample * f["n"] * int(base["params"].n_steps)


def run_reference(args, ws, rank):
    """--impl reference: the FP64 oracle as it stands on the host cores."""
    if rank != 0:
        return 0
    import oracle
    base, frames = make_workload(max(2, min(args.frames, 4)), rank)
    sample = args.ref_agents
    for i in range(args.warmup):
        oracle_step(base, frames[i % len(frames)], sample)
    t0 = time.perf_counter()
    inter = 0
    for i in range(args.steps):
        inter += oracle_step(base, frames[i % len(frames)], sample)
    dt = time.perf_counter() - t0
    value = inter / dt
    cores = oracle.max_threads()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": _config(base, args, ws),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "cpu_model": _cpu_model(),
                             "sample": f"per step: full-frame filter + {sample} of "
                                       f"{base['agents']['k_r'].size} agents x all obstacles x "
                                       f"{base['params'].n_steps} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or "unknown"


def _config(base, args, ws):
    return {"workload": "tabletop 640x480 depth frame -> 5 mm voxels; 256 agents x 500 steps",
            "n_raw": int(base["xyz"].shape[0]), "n_agents": int(base["agents"]["k_r"].size),
            "n_steps": int(base["params"].n_steps), "voxel_m": base["workspace"].voxel,
            "frames_in_ring": args.frames,
            "l2": f"inputs larger than L2: a ring of {args.frames} distinct frames "
                  f"({args.frames * base['xyz'].nbytes / 1e6:.0f} MB) resident in HBM",
            "parallelism": f"replicas x{ws}"}


def _traffic_from_profile():
    """Per-launch DRAM bytes of the rollout kernel from the committed ncu
    summary (the line 'traffic_bytes_per_launch: N'), if present."""
    if not os.path.exists(PROFILE_SUMMARY):
        return None
    with open(PROFILE_SUMMARY) as f:
        for line in f:
            if line.strip().startswith("traffic_bytes_per_launch:"):
                v = line.split(":", 1)[1].strip()
                return None if v in ("", "null") else float(v)
    return None


def run_ours(args, ws, rank, local):
    import torch
    import torch.distributed as dist
    import paper_2606_12579_b300 as gm

    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    base, frames_np = make_workload(args.frames, rank)
    prm = base["params"]
    na, nk = int(base["agents"]["k_r"].size), int(prm.n_steps)
    stream = torch.cuda.current_stream()
    ctx = gm.context(local)

    # inputs resident in HBM
    frames = torch.from_numpy(np.stack(frames_np)).cuda()
    pinned = torch.from_numpy(np.stack(frames_np)).pin_memory()
    agents = {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda()
              for k, v in base["agents"].items()}
    wsp = torch.empty(gm.filter_workspace_bytes(frames.shape[1], base["workspace"]),
                      dtype=torch.uint8, device="cuda")
    obs_cap = args.obs_cap
    if obs_cap <= 0:
        # size S_W to the scene: the first frame's N_O plus 5% (sensor noise
        # changes N_O by well under that from frame to frame)
        probe = gm.filter_cloud(frames[0], base["T"], base["workspace"], cap=OBS_CAP, workspace=wsp)
        obs_cap = (int(probe.count() * 1.05) + 63) // 64 * 64
        del probe
    obs = gm.Obstacles.empty(obs_cap)
    ro = gm.alloc_rollout_out(na, nk, want_traj=True, want_clear=False)
    sel = gm.score_and_select(gm.rollout_agents(gm.filter_cloud(frames[0], base["T"], base["workspace"],
                                                                 out=obs, workspace=wsp),
                                                agents, prm, out=ro), prm)
    ctx.sync()
    if args.tuning:
        tuning = tuple(int(v) for v in args.tuning.split(","))
    else:
        tuning, _ = gm.autotune_rollout(obs, agents, prm, out=ro, candidates=16, probe_steps=100)

    # N_O per frame (for the interaction count), outside any timed region
    n_obs = []
    for f in range(args.frames):
        gm.filter_cloud(frames[f], base["T"], base["workspace"], out=obs, workspace=wsp)
        n_obs.append(obs.count())
    ctx.sync()

    def step(f, ev=None):
        gm.filter_cloud(frames[f], base["T"], base["workspace"], out=obs, workspace=wsp)
        if ev is not None:
            ev[0].record(stream)
        gm.rollout_agents(obs, agents, prm, out=ro, tuning=tuning)
        if ev is not None:
            ev[1].record(stream)
        gm.score_and_select(ro, prm, out=sel)

    for i in range(args.warmup):
        step(i % args.frames)
    torch.cuda.synchronize()
    # FP32 FMA / SFU rates of this GPU (event-timed probe kernels), the
    # denominators of the force kernel's roofline
    peaks_probe = gm.measure_peaks(reps=5)
    for i in range(args.warmup):
        step(i % args.frames)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.25)
    ev_step = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    ev_roll = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    inter = 0
    for i in range(args.steps):
        f = (args.warmup + i) % args.frames
        ev_step[i][0].record(stream)
        step(f, ev_roll[i])
        ev_step[i][1].record(stream)
        inter += na * n_obs[f] * nk
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    ctx.sync()
    step_ms = [a.elapsed_time(b) for a, b in ev_step]
    roll_ms = [a.elapsed_time(b) for a, b in ev_roll]
    t_dev = sum(step_ms) / 1e3

    # end to end through the same calls: pinned host frame -> device, plan -> host
    host_best = torch.empty(1, dtype=torch.int32).pin_memory()
    host_traj = torch.empty(nk + 1, 3, dtype=torch.float32).pin_memory()
    dev_frame = torch.empty_like(frames[0])
    lat = []
    e2e_inter = 0
    for i in range(args.warmup + args.steps):
        f = i % args.frames
        t0 = time.perf_counter()
        dev_frame.copy_(pinned[f], non_blocking=True)
        gm.filter_cloud(dev_frame, base["T"], base["workspace"], out=obs, workspace=wsp)
        gm.rollout_agents(obs, agents, prm, out=ro, tuning=tuning)
        gm.score_and_select(ro, prm, out=sel)
        host_best.copy_(sel["best"], non_blocking=True)
        host_traj.copy_(sel["best_traj"], non_blocking=True)
        stream.synchronize()
        if i >= args.warmup:
            lat.append(time.perf_counter() - t0)
            e2e_inter += na * n_obs[f] * nk
    ctx.sync()

    # the same, streamed: the next frame's upload (copy stream, two device
    # frame buffers) overlaps the current step; every step still copies its
    # frame in and its plan out inside the timed region
    copy = torch.cuda.Stream()
    bufs = [torch.empty_like(frames[0]) for _ in range(2)]
    up = [torch.cuda.Event() for _ in range(2)]
    used = [torch.cuda.Event() for _ in range(2)]
    n_tot = args.warmup + args.steps
    h_best = torch.empty(n_tot, dtype=torch.int32).pin_memory()
    h_traj = torch.empty(n_tot, nk + 1, 3, dtype=torch.float32).pin_memory()
    for ev in used:
        ev.record(stream)

    def upload(i):
        b = i % 2
        with torch.cuda.stream(copy):
            copy.wait_event(used[b])
            bufs[b].copy_(pinned[i % args.frames], non_blocking=True)
            up[b].record(copy)

    def streamed(i0, i1):
        upload(i0)
        for i in range(i0, i1):
            b = i % 2
            if i + 1 < i1:
                upload(i + 1)
            stream.wait_event(up[b])
            gm.filter_cloud(bufs[b], base["T"], base["workspace"], out=obs, workspace=wsp)
            used[b].record(stream)
            gm.rollout_agents(obs, agents, prm, out=ro, tuning=tuning)
            gm.score_and_select(ro, prm, out=sel)
            h_best[i:i + 1].copy_(sel["best"], non_blocking=True)
            h_traj[i].copy_(sel["best_traj"], non_blocking=True)

    streamed(0, args.warmup)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    streamed(args.warmup, n_tot)
    torch.cuda.synchronize()
    e2e_stream_time = time.perf_counter() - t0
    ctx.sync()

    # executed work (untimed re-run of the timed frames): the kernel counts
    # the pairs whose heuristic terms it evaluated (Alg. 1's branch, taken per
    # block of 64 obstacles); every other pair costs the block test only
    hp = torch.zeros(1, dtype=torch.int64, device="cuda")
    ro["heur_pairs"] = hp
    for i in range(args.steps):
        gm.filter_cloud(frames[(args.warmup + i) % args.frames], base["T"], base["workspace"],
                        out=obs, workspace=wsp)
        gm.rollout_agents(obs, agents, prm, out=ro, tuning=tuning)
    ctx.sync()
    ro["heur_pairs"] = None
    heur_per_launch = hp.item() / args.steps

    # job time = max over ranks, work = sum over ranks
    (t_job, e2e_serial_time, e2e_time), (inter, e2e_inter) = reduce_over_ranks(
        [t_dev, sum(lat), e2e_stream_time], [inter, e2e_inter], ws, "cuda")

    result = None
    if rank == 0:
        props = torch.cuda.get_device_properties(local)
        peaks = _measured_peaks()
        sm_max = (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2032.0
        peak_nominal = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        # the faster of the packed and the scalar FMA probe
        peak_tflops = max(peaks_probe["fp32_tflops"], peaks_probe["fp32_tflops_scalar"])
        mean_roll = statistics.mean(roll_ms) / 1e3
        per_launch_inter = na * statistics.mean(
            [n_obs[(args.warmup + i) % args.frames] for i in range(args.steps)]) * nk
        achieved = per_launch_inter * FLOPS_PER_INTERACTION / mean_roll / 1e12
        # executed FP32 flops: every pair's block test (expanded distance, 3
        # FMAs) plus |o|^2 once per obstacle and half-group of AG/2 agents;
        # the pairs of evaluated blocks add the exact |d|^2 (8) and the
        # heuristic terms (5)
        exec_per_pair = BLOCK_TEST_FLOPS + OBSTACLE_NORM_FLOPS * 2.0 / tuning[1]
        exec_flops = per_launch_inter * exec_per_pair + heur_per_launch * FLOPS_PER_INTERACTION
        exec_tflops = exec_flops / mean_roll / 1e12
        cpu = cpu_baseline(base, frames_np, args.cpu_agents) if not args.no_cpu else None
        result = {
            "metric": METRIC, "value": inter / t_job, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_job / args.steps,
            "ms_per_step_median": float(np.median(step_ms)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": _config(base, args, ws),
            "n_obs_mean": float(np.mean(n_obs)), "tuning": list(tuning),
            "wall_s_timed": t_wall,
            "roofline": {"bound": "alu", "kernel": "k_rollout", "achieved": achieved,
                         "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                         "traffic": _traffic_from_profile(),
                         "flops_per_interaction": FLOPS_PER_INTERACTION,
                         "peak_source": "measured: gmapp_measure_peaks, the faster of "
                                        "fma.rn.f32x2 (12 chains) and fma.rn.f32 (16 chains), "
                                        "4 CTAs x 256 threads per SM, "
                                        f"at {peaks_probe['sm_mhz']:.0f} MHz",
                         "peak_nominal": peak_nominal,
                         "peak_nominal_source": f"{props.multi_processor_count} SMs x "
                                                f"{FP32_LANES_PER_SM} FP32 lanes x 2 x "
                                                f"{sm_max:.0f} MHz",
                         "frac_of_nominal": achieved / peak_nominal,
                         "peaks_measured": peaks_probe,
                         "rollout_ms_mean": 1e3 * mean_roll,
                         "rollout_ms_median": float(np.median(roll_ms)),
                         "executed": {
                             "note": "FP32 flops the kernel executes: the heuristic terms only "
                                     "for blocks of 64 obstacles where a pair passes the gate",
                             "heur_pair_fraction": heur_per_launch / per_launch_inter,
                             "flops_per_interaction": exec_flops / per_launch_inter,
                             "achieved": exec_tflops, "frac": exec_tflops / peak_tflops}},
            "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)),
                           "p99": 1e3 * float(np.percentile(lat, 99))},
            "e2e": {"value": e2e_inter / e2e_time, "unit": UNIT,
                    "h2d_bytes_per_step": int(frames[0].numel() * 4),
                    "d2h_bytes_per_step": int(host_best.numel() * 4 + host_traj.numel() * 4),
                    "mode": "streamed: frame i+1 uploads from pinned memory on a copy stream "
                            "while step i computes; the chosen index and plan of every step are "
                            "copied back",
                    "serial_value": e2e_inter / e2e_serial_time},
            "gpu_launches": args.steps * LAUNCHES_PER_STEP,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        result["config"]["obs_cap"] = obs_cap
        del frames, pinned, wsp, obs, ro, sel
        torch.cuda.empty_cache()
        if not args.no_patterns:
            result["patterns"] = {name: fn(gm, args) for name, fn in PATTERNS.items()
                                  if name != "filter_batched"}
            fs = result["patterns"]["filter_stream"]
        else:
            fs = bench_filter_stream(gm, args, with_fused=False, batched_only=True)
        result["roofline_filter"] = _filter_roofline(fs)
        print(json.dumps(result), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# filter_cloud (zero, keys, bitmap sums, emit, count) + rollout + select
LAUNCHES_PER_STEP = 5 + 1 + 1


def _events(torch, stream, fn, reps):
    """Mean device time (s) of fn() over reps runs, CUDA events on stream."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps


FILTER_PROFILE = os.path.join(ROOT, "profiles", "filter_stream_tabletop.md")


def _filter_roofline(fs: dict) -> dict:
    """Roofline line of the perception filter (A1-A3) from the filter-stream
    measurement: algorithmic bytes per frame / device time per frame against
    the measured HBM copy rate; DRAM traffic per frame from the committed
    ncu summary (line 'traffic_bytes_per_frame: N'), if present."""
    best = fs["stream"]
    traffic = None
    if os.path.exists(FILTER_PROFILE):
        with open(FILTER_PROFILE) as f:
            for line in f:
                if line.strip().startswith("traffic_bytes_per_frame:"):
                    v = line.split(":", 1)[1].strip()
                    traffic = None if v in ("", "null") else float(v)
    return {"bound": "hbm", "kernel": best.get("kernel", "filter_stream"),
            "achieved": best["GB_per_s"], "peak": fs["peak_GB_per_s"], "unit": "GB/s",
            "frac": best["hbm_frac"], "traffic": traffic,
            "algorithmic_bytes_per_frame": fs["algorithmic_bytes"] / fs["n_frames"],
            "us_per_frame": best["us_per_frame"], "workload": fs["workload"],
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}


def bench_filter_stream(gm, args, n_filters=256, n_distinct=64, n_streams=8, with_fused=True,
                        batched_only=False):
    """The perception filter alone (A1-A3) over a stream of 256 tabletop
    frames (307,200 points each, 944 MB read in total; 64 distinct frames,
    236 MB, cycled so that no frame is still in L2 when it comes back):
    through filter_cloud_batch, all 64 in one batch; and frame by frame
    through filter_cloud, on 8 CUDA streams with a workspace and an output
    each, and on one stream back to back (both graph-captured).  Algorithmic
    bytes per frame: 12 B per raw point read + 24 B per obstacle written
    (centres, key, count, index)."""
    import torch
    import synth
    base_frames = [synth.tabletop_workload(frame_seed=9_000_000 + f, n_agents=1, n_steps=1)
                   for f in range(8)]
    w0 = base_frames[0]
    g = np.random.Generator(np.random.PCG64(4242))
    host = []
    for i in range(n_distinct):
        xyz = base_frames[i % 8]["xyz"]
        host.append((xyz + g.normal(0.0, 1e-3, xyz.shape)).astype(np.float32))
    frames = torch.from_numpy(np.stack(host)).cuda()
    n_raw = frames.shape[1]
    wbytes = gm.filter_workspace_bytes(n_raw, w0["workspace"])
    streams = [torch.cuda.Stream() for _ in range(n_streams)]
    wsp = [torch.empty(wbytes, dtype=torch.uint8, device="cuda") for _ in range(n_streams)]
    outs = [gm.Obstacles.empty(131072) for _ in range(n_streams)]
    n_obs = []
    for i in range(n_distinct):   # N_O per distinct frame, outside timing
        gm.filter_cloud(frames[i], w0["T"], w0["workspace"], out=outs[0], workspace=wsp[0])
        n_obs.append(outs[0].count())
    torch.cuda.synchronize()

    def issue(ns):
        cur = torch.cuda.current_stream()
        for s in streams[:ns]:
            s.wait_stream(cur)
        for i in range(n_filters):
            k = i % ns
            with torch.cuda.stream(streams[k]):
                gm.filter_cloud(frames[i % n_distinct], w0["T"], w0["workspace"], out=outs[k],
                                workspace=wsp[k], stream=streams[k])
        for s in streams[:ns]:
            cur.wait_stream(s)

    def run(ns):
        # the 256 calls captured once in a CUDA graph, so the device time is
        # not bounded by the host issuing 1,280 launches
        issue(ns)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.graph(graph, stream=side):
            issue(ns)
        torch.cuda.synchronize()
        cur = torch.cuda.current_stream()
        best = None
        for _ in range(4):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(cur)
            graph.replay()
            e1.record(cur)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            best = t if best is None else min(best, t)
        return best

    byts = sum(12 * n_raw + 24 * n_obs[i % n_distinct] for i in range(n_filters))
    peak = _measured_peaks().get("hbm_gbs")
    res = {"workload": f"{n_filters} tabletop frames x {n_raw} points ({n_distinct} distinct, "
                       f"{n_distinct * n_raw * 12 / 1e6:.0f} MB), 5 mm voxels",
           "algorithmic_bytes": byts, "peak_GB_per_s": peak}

    def entry(t):
        gbs = byts / t / 1e9
        return {"ms": 1e3 * t, "us_per_frame": 1e6 * t / n_filters, "GB_per_s": gbs,
                "hbm_frac": gbs / peak if peak else None}

    # filter_cloud_batch: all 64 distinct frames in one batch (filtered in
    # L2-sized waves of a few frames on three streams), run four times
    per = n_distinct
    batches = [gm.FilterBatch([frames[i] for i in range(b, b + per)], w0["T"], w0["workspace"],
                              caps=[131072] * per) for b in range(0, n_distinct, per)]
    cur = torch.cuda.current_stream()
    for fb in batches:
        fb.run()
    torch.cuda.synchronize()
    for fb, b in zip(batches, range(0, n_distinct, per)):   # N_O agrees with filter_cloud
        assert [o.count() for o in fb.outs] == n_obs[b:b + per]
    best = None
    for _ in range(4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        for r in range(n_filters // per):
            batches[r % len(batches)].run()
        e1.record(cur)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        best = t if best is None else min(best, t)
    res["batched"] = entry(best)
    res["batched"]["frames_per_batch"] = per
    # the same runs captured once in a CUDA graph (the batch's side streams
    # join the capture), so launch latency is off the critical path
    side = torch.cuda.Stream()
    side.wait_stream(cur)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        for r in range(n_filters // per):
            batches[r % len(batches)].run(stream=side)
    torch.cuda.synchronize()
    bestg = None
    for _ in range(4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        graph.replay()
        e1.record(cur)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        bestg = t if bestg is None else min(bestg, t)
    for fb, b in zip(batches, range(0, n_distinct, per)):   # results unchanged by the replays
        assert [o.count() for o in fb.outs] == n_obs[b:b + per]
    res["batched_graph"] = entry(bestg)
    res["batched_graph"]["frames_per_batch"] = per
    res["n_frames"] = n_filters
    pick = "batched_graph" if bestg < best else "batched"
    res["stream"] = dict(res[pick], kernel="kf_points/kf_sums/kf_emit", mode=pick)
    del graph
    if batched_only:
        return res
    for ns in (n_streams, 1):
        res[f"per_frame_streams_{ns}"] = entry(run(ns))
    gm.sync()
    del batches, frames
    torch.cuda.empty_cache()
    if with_fused:
        res["fused_2_sensors"] = bench_fused(gm)
    return res


def bench_fused(gm, n_sets=24, reps=3):
    """filter_clouds: two 848x480 depth cameras fused into one obstacle set
    per call (Sec. IV-B), over a ring of n_sets distinct frame pairs resident
    in HBM (larger than L2); algorithmic bytes = 12 B per raw point + 24 B per
    obstacle."""
    import torch
    import synth
    sets = []
    n_obs = []
    for s in range(n_sets):
        m = synth.multi_sensor_frames(seed=9_000_000 + s, n_sensors=2)
        sets.append([(torch.from_numpy(x).cuda(), T) for x, T in m["clouds"]])
    ws = m["workspace"]
    out = gm.Obstacles.empty(262144)
    wsp = None
    for c in sets:
        gm.filter_clouds(c, ws, out=out)
        n_obs.append(out.count())
    need = sum(int(x.shape[0]) for x, _ in sets[0]) + 8
    wsp = torch.empty(int(gm.filter_workspace_bytes(need, ws)), dtype=torch.uint8, device="cuda")
    cur = torch.cuda.current_stream()
    for c in sets[:3]:
        gm.filter_clouds(c, ws, out=out, workspace=wsp)
    gm.sync()
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        for c in sets:
            gm.filter_clouds(c, ws, out=out, workspace=wsp)
        e1.record(cur)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / n_sets
        best = t if best is None else min(best, t)
    n_raw = sum(int(x.shape[0]) for x, _ in sets[0])
    byts = 12 * n_raw + 24 * float(np.mean(n_obs))
    peak = _measured_peaks().get("hbm_gbs")
    return {"workload": f"2 sensors x 848x480 ({n_raw} points), 5 mm voxels, {n_sets} distinct "
                        f"pairs ({n_sets * n_raw * 12 / 1e6:.0f} MB)",
            "n_obs_mean": float(np.mean(n_obs)), "us_per_call": 1e6 * best,
            "GB_per_s": byts / best / 1e9, "hbm_frac": byts / best / 1e9 / peak if peak else None,
            # k_zero, one key launch for both sensors, k_bitmap_sums, k_emit,
            # one count launch for both
            "launches_per_call": 5}


def bench_batched(gm, args, reps=3):
    """64 uneven sphere scenes: one batched launch sequence replayed from a
    CUDA graph vs the plain per-query path (filter_cloud, rollout_agents,
    score_and_select per query, one after another, same stream)."""
    import torch
    import synth
    ws_list = synth.batch_workloads()
    specs = [{"xyz": torch.from_numpy(w["xyz"]).cuda(), "T": w["T"], "ws": w["workspace"],
              "agents": {k: torch.from_numpy(v).cuda() for k, v in w["agents"].items()},
              "prm": w["params"], "obs_cap": 32768} for w in ws_list]
    b = gm.Batch(specs, want_traj=False)
    tune, _ = b.autotune()
    s = torch.cuda.Stream()
    b.launch_graph(s)
    s.synchronize()
    gm.sync()
    n_obs = [r["obs"].count() for r in b.results]
    inter = sum(int(w["agents"]["k_r"].size) * n * int(w["params"].n_steps)
                for w, n in zip(ws_list, n_obs))
    with torch.cuda.stream(s):
        t_batch = _events(torch, s, lambda: b.launch_graph(s), reps)
    gm.sync(s)
    # the same batch with block culling in the rollout kernel (same results;
    # plans/s only: culled pairs are not interactions)
    b.set_culling(True)
    b.launch_graph(s)
    gm.sync(s)
    t_cull = _events(torch, s, lambda: b.launch_graph(s), reps)
    gm.sync(s)
    b.set_culling(False)
    # plain per-query path
    outs = []
    for sp in specs:
        na = int(sp["agents"]["k_r"].numel())
        outs.append({"obs": gm.Obstacles.empty(32768),
                     "ro": gm.alloc_rollout_out(na, int(sp["prm"].n_steps), want_traj=False,
                                                want_clear=False),
                     "ws": torch.empty(gm.filter_workspace_bytes(sp["xyz"].shape[0], sp["ws"]),
                                       dtype=torch.uint8, device="cuda")})
    cur = torch.cuda.current_stream()

    def plain():
        for sp, o in zip(specs, outs):
            gm.filter_cloud(sp["xyz"], sp["T"], sp["ws"], out=o["obs"], workspace=o["ws"])
            gm.rollout_agents(o["obs"], sp["agents"], sp["prm"], out=o["ro"])
            gm.score_and_select(o["ro"], sp["prm"], best_traj=False)

    plain()
    gm.sync()
    t_plain = _events(torch, cur, plain, reps)
    gm.sync()
    return {"workload": "64 sphere scenes: raw 5k-300k points, voxel 4-10 mm, 32-1024 agents, "
                        "100-1000 steps", "interactions_per_batch": inter,
            "batched": {"plans_per_s": 64 / t_batch, "interactions_per_s": inter / t_batch,
                        "ms": 1e3 * t_batch, "tuning_agents_threads": list(tune),
                        "launches": 7, "graph": True},
            "plain": {"plans_per_s": 64 / t_plain, "interactions_per_s": inter / t_plain,
                      "ms": 1e3 * t_plain, "launches": 64 * LAUNCHES_PER_STEP},
            "batched_block_culled": {"plans_per_s": 64 / t_cull, "ms": 1e3 * t_cull},
            "speedup": t_plain / t_batch}


def bench_adjoint(gm, args, reps=3):
    """Differentiable rollout: 50,000 obstacles, 512 agents, 1000 steps,
    checkpoints every 50; forward (with checkpoints) + adjoint vs the plain
    forward rollout."""
    import torch
    import synth
    w = synth.adjoint_workload()
    prm = w["params"]
    o = gm.Obstacles.from_points(torch.from_numpy(w["obstacles"]), w["r_O"])
    ag = {k: torch.from_numpy(v).cuda() for k, v in w["agents"].items()}
    na, nk, K = 512, int(prm.n_steps), int(prm.ckpt_every)
    out = gm.alloc_rollout_out(na, nk, want_traj=False, want_clear=True)
    out["ckpt"] = torch.empty((nk + K - 1) // K, 6, na, device="cuda")
    plain_out = gm.alloc_rollout_out(na, nk, want_traj=False, want_clear=True)
    cur = torch.cuda.current_stream()
    ws = torch.empty(1 << 24, dtype=torch.uint8, device="cuda")
    gm.rollout_agents(o, ag, prm, out=out)
    gm.rollout_adjoint(o, ag, prm, out["ckpt"], workspace=ws)
    gm.rollout_agents(o, ag, prm, out=plain_out)
    gm.sync()
    # the forward's launch shape measured on these inputs (as the headline step)
    if getattr(args, "adjoint_tuning", ""):
        tuning = tuple(int(v) for v in args.adjoint_tuning.split(","))
    else:
        tuning, _ = gm.autotune_rollout(o, ag, prm, out=plain_out, candidates=16,
                                        probe_steps=100)
    t_fwd = _events(torch, cur, lambda: gm.rollout_agents(o, ag, prm, out=out, tuning=tuning),
                    reps)
    t_adj = _events(torch, cur, lambda: gm.rollout_adjoint(o, ag, prm, out["ckpt"], workspace=ws),
                    reps)
    t_plain = _events(torch, cur, lambda: gm.rollout_agents(o, ag, prm, out=plain_out,
                                                            tuning=tuning), reps)
    gm.sync()
    inter = na * w["obstacles"].shape[1] * nk
    peaks = gm.measure_peaks(reps=3)
    peak = max(peaks["fp32_tflops"], peaks["fp32_tflops_scalar"])
    # no detection gate: every pair runs the full terms, so the 13-flop
    # accounting is executed work
    fwd_tflops = inter * FLOPS_PER_INTERACTION / t_plain / 1e12
    return {"workload": "50,000 obstacles, 512 agents, 1000 steps, K = 50",
            "tuning": list(tuning),
            "forward_ms": 1e3 * t_fwd, "adjoint_ms": 1e3 * t_adj, "plain_forward_ms": 1e3 * t_plain,
            "forward_equivalent_interactions_per_s": inter / (t_fwd + t_adj),
            # raw flops: the forward's 13 per pair, and the adjoint's recompute
            # with the gradient of W (13 + 3 mul + 3 accumulating FMAs + the
            # derivative of 1/s, about 26 per pair)
            "adjoint_TFLOP_per_s": inter * ADJOINT_FLOPS_PER_INTERACTION / t_adj / 1e12,
            "forward_plus_adjoint_TFLOP_per_s":
                inter * (FLOPS_PER_INTERACTION + ADJOINT_FLOPS_PER_INTERACTION) / (t_fwd + t_adj) / 1e12,
            "gradient_cost_over_plain_forward": (t_fwd + t_adj) / t_plain,
            "plain_forward_fp32": {"achieved_TFLOP_per_s": fwd_tflops, "peak_TFLOP_per_s": peak,
                                   "frac": fwd_tflops / peak,
                                   "note": "every pair evaluated (r_d = inf): executed flops"}}


def bench_ensemble(gm, args, reps=5):
    """Heterogeneous ensemble (Eq. apf + Eq. mfi) on the tabletop query:
    256 agents x 500 steps, the last 128 on APF, in one launch; beside it
    the plain MFI rollout of the same 256 agents, an all-APF launch, an
    all-projected-current launch and a three-kind ensemble (86 MFI, 85
    projected, 85 APF), each in the launch shape the autotuner measures best
    for it."""
    import torch
    import synth
    w = synth.tabletop_workload()
    prm = w["params"]
    na, nk, n_apf = 256, int(prm.n_steps), 128
    xyz = torch.from_numpy(w["xyz"]).cuda()
    probe = gm.filter_cloud(xyz, w["T"], w["workspace"], cap=OBS_CAP)
    cap = (int(probe.count() * 1.05) + 63) // 64 * 64
    obs = gm.filter_cloud(xyz, w["T"], w["workspace"], cap=cap)
    n_o = obs.count()
    dev = lambda a: {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda()  # noqa: E731
                     for k, v in a.items()}
    mixed = dev(synth.ensemble_agents(w["agents"], n_apf))
    all_apf = dev(synth.ensemble_agents(w["agents"], na))
    mfi = dev(w["agents"])
    n3 = na // 3   # three kinds: 86 MFI, 85 projected current, 85 APF
    three = dev(synth.ensemble_agents(w["agents"], n3))
    out = gm.alloc_rollout_out(na, nk, want_traj=True, want_clear=False)
    shapes = {"ensemble": gm.autotune_ensemble(obs, mixed, n_apf, prm, out=out, candidates=16,
                                               probe_steps=nk)[0],
              "mfi": gm.autotune_rollout(obs, mfi, prm, out=out, candidates=16, probe_steps=nk)[0],
              "apf": gm.autotune_ensemble(obs, all_apf, na, prm, out=out, candidates=16,
                                          probe_steps=nk)[0],
              "proj": gm.autotune_ensemble(obs, mfi, 0, prm, out=out, candidates=16,
                                           probe_steps=nk, n_proj=na)[0],
              "three_kinds": gm.autotune_ensemble(obs, three, n3, prm, out=out, candidates=16,
                                                  probe_steps=nk, n_proj=n3)[0]}
    cur = torch.cuda.current_stream()
    runs = {"ensemble": lambda: gm.rollout_ensemble(obs, mixed, n_apf, prm, out=out,
                                                    tuning=shapes["ensemble"]),
            "mfi": lambda: gm.rollout_agents(obs, mfi, prm, out=out, tuning=shapes["mfi"]),
            "apf": lambda: gm.rollout_ensemble(obs, all_apf, na, prm, out=out,
                                               tuning=shapes["apf"]),
            "proj": lambda: gm.rollout_ensemble(obs, mfi, 0, prm, out=out, tuning=shapes["proj"],
                                                n_proj=na),
            "three_kinds": lambda: gm.rollout_ensemble(obs, three, n3, prm, out=out,
                                                       tuning=shapes["three_kinds"], n_proj=n3),
            # the mixed ensemble culled by the obstacle blocks' bounding boxes
            # (the same forces bit for bit; reported as time, not interactions)
            "ensemble_culled": lambda: gm.rollout_ensemble(obs, mixed, n_apf, prm, out=out,
                                                           tuning=shapes["ensemble"], cull=True)}
    shapes["ensemble_culled"] = shapes["ensemble"]
    for k, fn in runs.items():   # warm-up launches, one NVTX range each (for ncu)
        torch.cuda.nvtx.range_push(f"warm_{k}")
        fn()
        torch.cuda.nvtx.range_pop()
    gm.sync()
    times = {k: _events(torch, cur, fn, reps) for k, fn in runs.items()}
    gm.sync()
    # pairs whose heuristic terms ran (untimed re-run with the kernel's counter)
    heur = {}
    for k, fn in runs.items():
        hp = torch.zeros(1, dtype=torch.int64, device="cuda")
        out["heur_pairs"] = hp
        fn()
        gm.sync()
        heur[k] = hp.item()
    out["heur_pairs"] = None
    peaks = _measured_peaks()
    sm_max = peaks.get("sm_max_mhz") or 2032.0
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    pairs = n_o * nk
    flops = {"ensemble": pairs * ((na - n_apf) * FLOPS_PER_INTERACTION +
                                  n_apf * APF_FLOPS_PER_INTERACTION),
             "mfi": pairs * na * FLOPS_PER_INTERACTION,
             "apf": pairs * na * APF_FLOPS_PER_INTERACTION,
             "proj": pairs * na * PROJ_FLOPS_PER_INTERACTION,
             "three_kinds": pairs * ((na - 2 * n3) * FLOPS_PER_INTERACTION +
                                     n3 * PROJ_FLOPS_PER_INTERACTION +
                                     n3 * APF_FLOPS_PER_INTERACTION)}
    flops["ensemble_culled"] = flops["ensemble"]
    res = {"workload": f"tabletop 640x480 -> 5 mm voxels (N_O = {n_o}); 256 agents x 500 steps; "
                       f"ensemble = last {n_apf} agents APF (gain x 1e-3), r_d alternating 5/10 cm",
           "tuning": {k: list(v) for k, v in shapes.items()}, "peak_TFLOP_per_s": peak,
           "flops_per_interaction": {"mfi": FLOPS_PER_INTERACTION,
                                     "apf": APF_FLOPS_PER_INTERACTION,
                                     "proj": PROJ_FLOPS_PER_INTERACTION}}
    # executed flops: every pair's block test, plus the full terms of the
    # kind (its per-pair count) for the pairs of evaluated blocks; a mixed
    # launch weighs the kinds' counts by their agent shares (approximate)
    full = {"ensemble": ((na - n_apf) * FLOPS_PER_INTERACTION + n_apf * APF_FLOPS_PER_INTERACTION) / na,
            "mfi": FLOPS_PER_INTERACTION, "apf": APF_FLOPS_PER_INTERACTION,
            "proj": PROJ_FLOPS_PER_INTERACTION,
            "three_kinds": flops["three_kinds"] / (pairs * na)}
    full["ensemble_culled"] = full["ensemble"]
    for k, s in times.items():
        test = BLOCK_TEST_FLOPS + OBSTACLE_NORM_FLOPS * 2.0 / shapes[k][1]
        ex = pairs * na * test + heur[k] * full[k]
        res[k] = {"ms": 1e3 * s, "interactions_per_s": na * pairs / s,
                  "TFLOP_per_s": flops[k] / s / 1e12, "fp32_frac": flops[k] / s / 1e12 / peak,
                  "heur_pair_fraction": heur[k] / (pairs * na),
                  "executed_TFLOP_per_s": ex / s / 1e12, "executed_frac": ex / s / 1e12 / peak}
    res["note"] = ("fp32_frac counts every pair at its kind's full flop count (the paper's "
                   "per-interaction work); the kernels evaluate the terms only for blocks of 128 "
                   "obstacles where a pair passes a gate, so executed_frac is the FP32 work done")
    return res


def bench_replan(gm, args, n_frames=16, ticks=32, alpha=0.95):
    """Re-planning loop with the paper's four-term cost (Eq. cost_function)
    and hysteresis: per tick a new tabletop frame (a ring of distinct frames
    resident in HBM) -> filter_cloud -> rollout_agents accumulating the cost
    sums (256 agents x 500 steps, clearance reduced) -> score_and_select4
    against the device-resident C_best (alpha = 0.95), no host round trip
    inside a tick.  Beside it the same ticks with the plain cost (the
    headline step: no clearance, score_and_select)."""
    import dataclasses
    import torch
    base, frames_np = make_workload(n_frames, 0)
    prm = dataclasses.replace(base["params"], cost_radius=0.05, a_max=50.0)
    na, nk = int(base["agents"]["k_r"].size), int(prm.n_steps)
    frames = torch.from_numpy(np.stack(frames_np)).cuda()
    agents = {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda()
              for k, v in base["agents"].items()}
    wsp = torch.empty(gm.filter_workspace_bytes(frames.shape[1], base["workspace"]),
                      dtype=torch.uint8, device="cuda")
    n_obs = []
    probe = gm.Obstacles.empty(OBS_CAP)
    for f in range(n_frames):
        gm.filter_cloud(frames[f], base["T"], base["workspace"], out=probe, workspace=wsp)
        n_obs.append(probe.count())
    cap = (int(max(n_obs) * 1.05) + 63) // 64 * 64
    del probe
    obs = gm.Obstacles.empty(cap)
    gm.filter_cloud(frames[0], base["T"], base["workspace"], out=obs, workspace=wsp)
    out4 = gm.alloc_rollout_out(na, nk, want_traj=True, want_cost4=True)
    out = gm.alloc_rollout_out(na, nk, want_traj=True, want_clear=False)
    t4, _ = gm.autotune_rollout(obs, agents, prm, out=out4, candidates=16, probe_steps=100)
    t0, _ = gm.autotune_rollout(obs, agents, prm, out=out, candidates=16, probe_steps=100)
    c_best = torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")
    picks = torch.empty(ticks, dtype=torch.int32, device="cuda")
    sel4 = gm.score_and_select4(out4, prm)       # output buffers, reused
    sel = gm.score_and_select(out, prm)

    def tick4(i):
        gm.filter_cloud(frames[i % n_frames], base["T"], base["workspace"], out=obs, workspace=wsp)
        gm.rollout_agents(obs, agents, prm, out=out4, tuning=t4)
        gm.score_and_select4(out4, prm, c_best=c_best, alpha=alpha, out=sel4)
        picks[i % ticks].copy_(sel4["best"][0])

    def tick(i):
        gm.filter_cloud(frames[i % n_frames], base["T"], base["workspace"], out=obs, workspace=wsp)
        gm.rollout_agents(obs, agents, prm, out=out, tuning=t0)
        gm.score_and_select(out, prm, out=sel)

    cur = torch.cuda.current_stream()
    for i in range(3):
        tick4(i)
        tick(i)
    gm.sync()
    c_best.fill_(float("nan"))
    t_4 = _events(torch, cur, lambda it=iter(range(ticks)): tick4(next(it)), ticks)
    t_0 = _events(torch, cur, lambda it=iter(range(ticks)): tick(next(it)), ticks)
    gm.sync()
    pk = picks.cpu().numpy()
    inter = sum(na * n_obs[i % n_frames] * nk for i in range(ticks)) / ticks
    return {"workload": f"{ticks} ticks over {n_frames} tabletop frames; 256 agents x 500 steps; "
                        f"four-term cost (r_c 5 cm, a_max 50 m/s^2, w = 1,1,1,1), alpha = {alpha}",
            "tuning": {"four_term": list(t4), "plain": list(t0)},
            "four_term": {"ms_per_tick": 1e3 * t_4, "plans_per_s": 1.0 / t_4,
                          "interactions_per_s": inter / t_4,
                          "plan_switches": int((pk >= 0).sum()), "kept_plan": int((pk < 0).sum())},
            "plain_cost": {"ms_per_tick": 1e3 * t_0, "plans_per_s": 1.0 / t_0,
                           "interactions_per_s": inter / t_0},
            "overhead_of_four_term_cost": t_4 / t_0 - 1.0}


def bench_culled(gm, args, n_frames=16, ticks=32):
    """Plans with spatial culling vs the all-pairs plan on the tabletop
    query: per plan a new frame (a ring of distinct frames in HBM) ->
    filter_cloud -> [gmapp_grid_index -> rollout_agents_culled |
    rollout_agents_blockcull | rollout_agents] -> score_and_select, 256
    agents x 500 steps, r_d = 5 cm.  Culling skips the pairs beyond the
    gate, so it is reported as plans/s (interactions/s counts all pairs).
    The block-culled rollout takes the fastest of a few launch shapes."""
    import torch
    base, frames_np = make_workload(n_frames, 0)
    prm, ws = base["params"], base["workspace"]
    na, nk = int(base["agents"]["k_r"].size), int(prm.n_steps)
    frames = torch.from_numpy(np.stack(frames_np)).cuda()
    agents = {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda()
              for k, v in base["agents"].items()}
    wsp = torch.empty(gm.filter_workspace_bytes(frames.shape[1], ws), dtype=torch.uint8,
                      device="cuda")
    probe = gm.filter_cloud(frames[0], base["T"], ws, cap=OBS_CAP, workspace=wsp)
    cap = (int(probe.count() * 1.05) + 63) // 64 * 64
    del probe
    obs = gm.Obstacles.empty(cap)
    index = gm.grid_index(gm.filter_cloud(frames[0], base["T"], ws, out=obs, workspace=wsp), ws)
    out_c = gm.alloc_rollout_out(na, nk, want_traj=True, want_clear=False)
    out_c["f_trace"] = None
    out_a = gm.alloc_rollout_out(na, nk, want_traj=True, want_clear=False)
    tun, _ = gm.autotune_rollout(obs, agents, prm, out=out_a, candidates=16, probe_steps=100)
    sel_c, sel_a = gm.score_and_select(out_c, prm), gm.score_and_select(out_a, prm)

    def plan_culled(i):
        gm.filter_cloud(frames[i % n_frames], base["T"], ws, out=obs, workspace=wsp)
        gm.grid_index(obs, ws, index=index)
        gm.rollout_agents_culled(obs, ws, index, agents, prm, out=out_c)
        gm.score_and_select(out_c, prm, out=sel_c)

    def plan_all(i):
        gm.filter_cloud(frames[i % n_frames], base["T"], ws, out=obs, workspace=wsp)
        gm.rollout_agents(obs, agents, prm, out=out_a, tuning=tun)
        gm.score_and_select(out_a, prm, out=sel_a)

    # block culling: the per-step exchange sets its pace, so shapes with the
    # cluster exchange and more agents per group are among the candidates
    out_b = gm.alloc_rollout_out(na, nk, want_traj=True, want_clear=False)
    sel_b = gm.score_and_select(out_a, prm)
    cur = torch.cuda.current_stream()
    best_b = None
    for cand in [tuple(tun), (5, 9, 384, 0), (5, 10, 384, 0), (4, 8, 384, 0), (6, 11, 384, 1),
                 (8, 16, 256, 0), (8, 16, 256, 1)]:
        try:
            gm.rollout_agents_blockcull(obs, agents, prm, out=out_b, tuning=cand)
            gm.sync()
        except gm.GmappError:
            continue
        tb = _events(torch, cur, lambda c=cand: gm.rollout_agents_blockcull(
            obs, agents, prm, out=out_b, tuning=c), 3)
        if best_b is None or tb < best_b[0]:
            best_b = (tb, cand)
    tun_b = best_b[1]

    def plan_block(i):
        gm.filter_cloud(frames[i % n_frames], base["T"], ws, out=obs, workspace=wsp)
        gm.rollout_agents_blockcull(obs, agents, prm, out=out_b, tuning=tun_b)
        gm.score_and_select(out_b, prm, out=sel_b)

    for i in range(3):
        plan_culled(i)
        plan_all(i)
        plan_block(i)
    gm.sync()
    torch.cuda.nvtx.range_push("warm_blockcull")   # one launch in a range (for ncu)
    gm.rollout_agents_blockcull(obs, agents, prm, out=out_b, tuning=tun_b)
    torch.cuda.nvtx.range_pop()
    gm.sync()
    t_c = _events(torch, cur, lambda it=iter(range(ticks)): plan_culled(next(it)), ticks)
    t_a = _events(torch, cur, lambda it=iter(range(ticks)): plan_all(next(it)), ticks)
    t_b = _events(torch, cur, lambda it=iter(range(ticks)): plan_block(next(it)), ticks)
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    ev[0].record(cur)
    for _ in range(5):
        gm.rollout_agents_culled(obs, ws, index, agents, prm, out=out_c)
    ev[1].record(cur)
    torch.cuda.synchronize()
    t_roll = ev[0].elapsed_time(ev[1]) / 1e3 / 5
    gm.sync()
    same = int((sel_c["best"] == sel_a["best"]).item())
    same_b = int((sel_b["best"] == sel_a["best"]).item())
    return {"workload": f"{ticks} plans over {n_frames} tabletop frames; 256 agents x 500 steps, "
                        "r_d = 5 cm",
            "culled": {"ms_per_plan": 1e3 * t_c, "plans_per_s": 1.0 / t_c,
                       "rollout_ms": 1e3 * t_roll},
            "block_culled": {"ms_per_plan": 1e3 * t_b, "plans_per_s": 1.0 / t_b,
                             "rollout_ms": 1e3 * best_b[0], "tuning": list(tun_b),
                             "speedup_vs_all_pairs": t_a / t_b,
                             "last_plan_same_agent": bool(same_b)},
            "all_pairs": {"ms_per_plan": 1e3 * t_a, "plans_per_s": 1.0 / t_a,
                          "tuning": list(tun)},
            "speedup": t_a / t_c, "last_plan_same_agent": bool(same)}


def bench_served(gm, args):
    """1 kHz open-loop request stream over ``--serve-seconds`` (default 10 s:
    10,000 requests), each with its own 200k-point frame of the tabletop
    scene with 4 moving spheres at its arrival time (1 cm voxels, N_a in
    {64, 256, 1024}, N_k = 300), through the continuously batched server
    (first-fit admission with an aging bound) vs the same stream served one
    request at a time through the plain per-query calls.  The frames are
    rendered on the GPU before the stream starts (synth.stream_frames) and
    held in pinned host memory, as a sensor would deliver them; every request
    copies its frame host -> device.  The culled comparisons run the first
    ``--serve-cull-seconds`` of the same stream at several offered rates."""
    import torch
    import synth
    from synth.stream_frames import StreamFrames
    dur = float(args.serve_seconds)
    n_req = int(round(dur * 1000))
    arrivals_1k, na_choice, _ = synth.serve_stream(n_requests=n_req)
    renderer = StreamFrames(seed=1005, n_points=200000, device="cuda")
    frame_bytes = 200000 * 12
    avail = 64 << 30
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    # every request its own frame, as long as host memory holds them (a
    # quarter of the available memory at most); else frames are reused
    # cyclically and the output says how many were distinct
    n_frames = int(max(64, min(n_req, (avail // 4) // frame_bytes)))
    n_frames = (n_frames // 64) * 64 if n_frames < n_req else n_req
    frames = torch.empty(n_frames, 200000, 3, dtype=torch.float32, pin_memory=True)
    for c0 in range(0, n_frames, 512):
        c1 = min(n_frames, c0 + 512)
        frames[c0:c1].copy_(renderer.render(arrivals_1k[c0:c1], first=c0))
    torch.cuda.synchronize()
    T_cam = renderer.T
    Ts = [T_cam]
    base = synth.tabletop_workload(seed=1005, n_agents=1, n_steps=1, n_points=2000, voxel=0.01)
    ws_grid, prm = base["workspace"], base["params"]
    import dataclasses
    prm = dataclasses.replace(prm, n_steps=300)
    agents = {}
    for na in (64, 256, 1024):
        a = synth.agent_set(na, 77 + na, synth.workloads.TABLE_START, synth.workloads.TABLE_GOAL)
        agents[na] = {k: torch.from_numpy(v).pin_memory() for k, v in a.items()}
    frame_of = [r % n_frames for r in range(n_req)]
    Ts = [T_cam] * n_frames

    def lat_stats(lat, t_span, inter):
        lat = np.asarray(lat) * 1e3
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "plans_per_s": len(lat) / t_span, "interactions_per_s": inter / t_span}

    def run_served(culled, rate=1000.0, chunk=50, n=n_req, plan_streams=0, alpha=0.95):
        """The first ``n`` requests of the stream, offered at ``rate``
        requests/s, through the continuously batched server (``chunk`` steps
        of every active plan per tick; first-fit admission, a queued request
        overtaken at most 64 times).  With ``plan_streams`` > 0 the requests
        are re-planning ticks of that many robots (request r belongs to
        stream r mod plan_streams), scored by the paper's four-term cost and
        selected against their stream's C_best with hysteresis ``alpha``."""
        arrivals = arrivals_1k * (1000.0 / rate)
        srv = gm.Server(max_slots=48, max_agents=1024, max_steps=300, obs_cap=32768,
                        arena_bytes=2 << 30, chunk_steps=chunk, agents_per_item=8, threads=256,
                        culled=culled, admit_bypass=64, four_term=plan_streams > 0,
                        max_plan_streams=plan_streams)
        c4 = dict(cost4=True, alpha=alpha) if plan_streams else {}
        kept = 0
        for r in range(4):   # warm up (kernel loading, first admissions)
            t = srv.submit(frames[0], Ts[0], ws_grid, agents[int(na_choice[r])], prm)
            while srv.poll(t) is None:
                srv.tick()
            srv.release(t)
        lat, inter, done = [], 0, 0
        outstanding = {}
        t0 = time.perf_counter()
        nxt = 0
        while done < n:
            now = time.perf_counter() - t0
            while nxt < n and arrivals[nxt] <= now:
                na = int(na_choice[nxt])
                if plan_streams:
                    c4["plan_stream"] = nxt % plan_streams
                tk = srv.submit(frames[frame_of[nxt]], Ts[frame_of[nxt]], ws_grid, agents[na], prm,
                                **c4)
                outstanding[tk] = (nxt, na)
                nxt += 1
            if not outstanding:
                while time.perf_counter() - t0 < arrivals[nxt]:
                    pass
                continue
            srv.tick()
            for tk in list(outstanding):
                res = srv.poll(tk)
                if res is None:
                    continue
                r, na = outstanding.pop(tk)
                lat.append(time.perf_counter() - t0 - arrivals[r])
                inter += na * res["n_obs"] * prm.n_steps
                kept += res["best"] < 0
                srv.release(tk)
                done += 1
        t_span = time.perf_counter() - t0
        del srv
        out = lat_stats(lat, t_span, inter)
        if plan_streams:
            out.update(plan_streams=plan_streams, alpha=alpha, kept_current_plan=int(kept))
        return out

    cur = torch.cuda.current_stream()
    dev_frame = torch.empty(200000, 3, device="cuda")
    obs = gm.Obstacles.empty(32768)
    wsb = torch.empty(gm.filter_workspace_bytes(200000, ws_grid), dtype=torch.uint8, device="cuda")
    index = gm.grid_index(gm.filter_cloud(dev_frame.copy_(frames[0]), Ts[0], ws_grid, out=obs,
                                          workspace=wsb), ws_grid)
    dev_agents = {na: {k: v.cuda() for k, v in a.items()} for na, a in agents.items()}
    outs = {na: gm.alloc_rollout_out(na, 300, want_traj=True, want_clear=False) for na in agents}
    for o in outs.values():
        o["f_trace"] = None
    host_best = torch.empty(1, dtype=torch.int32).pin_memory()
    host_traj = torch.empty(301, 3).pin_memory()

    def plan(na, culled):
        if culled:
            gm.grid_index(obs, ws_grid, index=index)
            gm.rollout_agents_culled(obs, ws_grid, index, dev_agents[na], prm, out=outs[na])
        else:
            gm.rollout_agents(obs, dev_agents[na], prm, out=outs[na])
        return gm.score_and_select(outs[na], prm)

    def run_plain(culled, rate=1000.0, n=n_req):
        """The first ``n`` requests of the stream, offered at ``rate``
        requests/s, one request at a time through the per-query calls."""
        arrivals = arrivals_1k * (1000.0 / rate)
        for na in agents:  # warm up
            gm.filter_cloud(dev_frame.copy_(frames[0]), Ts[0], ws_grid, out=obs, workspace=wsb)
            plan(na, culled)
        gm.sync()
        lat, inter = [], 0
        t0 = time.perf_counter()
        for r in range(n):
            while time.perf_counter() - t0 < arrivals[r]:
                pass
            na = int(na_choice[r])
            dev_frame.copy_(frames[frame_of[r]], non_blocking=True)
            gm.filter_cloud(dev_frame, Ts[frame_of[r]], ws_grid, out=obs, workspace=wsb)
            sel = plan(na, culled)
            host_best.copy_(sel["best"], non_blocking=True)
            host_traj.copy_(sel["best_traj"], non_blocking=True)
            cur.synchronize()
            lat.append(time.perf_counter() - t0 - arrivals[r])
            inter += na * int(obs.count()) * 300
        t_span = time.perf_counter() - t0
        gm.sync()
        return lat_stats(lat, t_span, inter)

    served, plain = run_served(False), run_plain(False)
    # the re-planning form: 8 robots' plan streams, four-term cost, C_best
    # per stream on the device (the first --serve-cull-seconds of the stream)
    n_cull = min(n_req, int(round(float(args.serve_cull_seconds) * 1000)))
    replan = run_served(False, n=n_cull, plan_streams=8)
    culled = {}
    for rate in (float(r) for r in str(args.serve_cull_rates).split(",")):
        s = run_served(True, rate, int(args.serve_cull_chunk), n=n_cull)
        p = run_plain(True, rate, n=n_cull)
        sb = run_served("blocks", rate, int(args.serve_cull_chunk), n=n_cull)
        culled[f"{rate:g}_per_s"] = {"served": s, "plain": p, "p99_speedup": p["p99_ms"] / s["p99_ms"],
                                     "served_block_culled": sb}
    return {"workload": f"{n_req} requests at 1 kHz over {dur:g} s: each its own 200k-point "
                        "tabletop frame with 4 moving spheres at its arrival time, 1 cm voxels, "
                        "N_a in {64, 256, 1024}, N_k = 300",
            "offered_per_s": 1000.0, "served": served, "plain": plain,
            "p99_speedup": plain["p99_ms"] / served["p99_ms"],
            "plans_per_s_speedup": served["plans_per_s"] / plain["plans_per_s"],
            "served_four_term_replanning": dict(replan, requests=n_cull),
            "admission": "first fit over the queue, a request overtaken at most 64 times",
            "culled": {"note": "every agent visits only the obstacles within its reach "
                               "(interactions/s still counts all pairs); the first "
                               f"{n_cull} requests of the same stream at each rate",
                       "chunk_steps": int(args.serve_cull_chunk), **culled},
            "frames_distinct": n_frames, "frames_host_bytes": int(frames.numel() * 4)}


def cpu_baseline(base, frames, n_agents_sample, min_seconds=10.0, max_steps=8):
    """The oracle as it stands on the host cores (OpenMP over agents): whole
    steps (the frame's filter, then n_agents_sample agents x all obstacles x
    N_k) on successive frames until min_seconds have passed; and one thread
    on a sixteenth of the agents of one step."""
    import oracle
    cores = oracle.max_threads()
    t0 = time.perf_counter()
    inter, steps = 0, 0
    while steps < max_steps and (steps == 0 or time.perf_counter() - t0 < min_seconds):
        inter += oracle_step(base, frames[steps % len(frames)], n_agents_sample)
        steps += 1
    dt = time.perf_counter() - t0
    one = max(1, n_agents_sample // 16)
    oracle.set_threads(1)
    try:
        t1 = time.perf_counter()
        inter1 = oracle_step(base, frames[0], one)
        dt1 = time.perf_counter() - t1
    finally:
        oracle.set_threads(cores)
    return {"value": inter / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu_model": _cpu_model(),
            "sample": f"{steps} steps on distinct frames, each: full-frame filter + "
                      f"{n_agents_sample} of {base['agents']['k_r'].size} agents x all obstacles x "
                      f"{base['params'].n_steps} steps",
            "seconds": dt,
            "single_thread": {"value": inter1 / dt1, "agents": one, "seconds": dt1}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--frames", type=int, default=48)
    ap.add_argument("--cpu-agents", type=int, default=256,
                    help="agents per step of the oracle's cpu_baseline")
    ap.add_argument("--ref-agents", type=int, default=256,
                    help="agents per step of the --impl reference arm (all 256 by default, "
                         "so the oracle's OpenMP threads over agents all have work)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--obs-cap", type=int, default=0,
                    help="obstacle capacity of the S_W buffers (multiple of 4; 0 = from the scene)")
    ap.add_argument("--no-patterns", action="store_true",
                    help="skip the batched / adjoint / served measurements")
    ap.add_argument("--serve-cull-rates", default="1000,2000,4000",
                    help="offered request rates (Hz) of the culled serving comparison")
    ap.add_argument("--serve-cull-chunk", type=int, default=300,
                    help="steps per tick of the culled server")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="length of the 1 kHz request stream of the served loop")
    ap.add_argument("--serve-cull-seconds", type=float, default=3.0,
                    help="length of the stream prefix of the culled serving comparison")
    ap.add_argument("--tuning", default="",
                    help="rollout launch shape 'cluster,agents,threads[,exchange]' "
                         "(default: autotuned)")
    ap.add_argument("--adjoint-tuning", default="",
                    help="forward launch shape of the adjoint pattern "
                         "'cluster,agents,threads,exchange' (default: autotuned)")
    ap.add_argument("--pattern", choices=sorted(PATTERNS), default=None,
                    help="run only this pattern measurement and print its JSON")
    args = ap.parse_args()
    ws, rank, local = _dist()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.pattern:
        import torch
        import paper_2606_12579_b300 as gm
        torch.cuda.set_device(local)
        gm.context(local)
        print(json.dumps({args.pattern: PATTERNS[args.pattern](gm, args)}), flush=True)
        return 0
    return run_ours(args, ws, rank, local)


PATTERNS = {"filter_stream": lambda gm, a: bench_filter_stream(gm, a),
            "filter_batched": lambda gm, a: bench_filter_stream(gm, a, batched_only=True),
            "batched": lambda gm, a: bench_batched(gm, a),
            "adjoint": lambda gm, a: bench_adjoint(gm, a),
            "ensemble": lambda gm, a: bench_ensemble(gm, a),
            "replan": lambda gm, a: bench_replan(gm, a),
            "culled": lambda gm, a: bench_culled(gm, a),
            "served": lambda gm, a: bench_served(gm, a)}


if __name__ == "__main__":
    sys.exit(main())
