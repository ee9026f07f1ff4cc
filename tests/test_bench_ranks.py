"""The N > 1 path of bench.py on CPU: two gloo ranks combine their times by
maximum and their work by sum (replicas only, no data-path exchange), each
rank renders its own frames of the same scene, and the reference arm runs on
rank 0 alone."""

import os
import socket

import numpy as np
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        times, counts = bench.reduce_over_ranks([1.0 + rank, 5.0 - rank], [10 * (rank + 1), 7],
                                                ws, "cpu")
        dist.barrier()
        q.put((rank, times, counts))
    finally:
        dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, times, counts in got:
        assert times == [2.0, 5.0]        # max over ranks
        assert counts == [30.0, 14.0]     # sum over ranks


def test_single_process_is_identity():
    assert bench.reduce_over_ranks([3, 4], [5], 1, "cpu") == ([3.0, 4.0], [5.0])


def test_ranks_get_distinct_frames_of_one_scene():
    b0, f0 = bench.make_workload(1, 0)
    b1, f1 = bench.make_workload(1, 1)
    assert np.array_equal(b0["T"], b1["T"])
    for k in b0["agents"]:
        assert np.array_equal(b0["agents"][k], b1["agents"][k])
    assert f0[0].shape == f1[0].shape
    assert not np.array_equal(np.nan_to_num(f0[0]), np.nan_to_num(f1[0]))


def test_reference_arm_runs_on_rank0_only():
    class A:
        frames, warmup, steps, ref_agents = 2, 0, 1, 1
    assert bench.run_reference(A(), 2, 1) == 0
