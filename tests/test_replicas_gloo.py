"""The multi-GPU form of the benchmark is independent replicas (the method's
path has no exchange step on one mesh per GPU): the job's time is the maximum
over the ranks, and its throughput counts every replica's work. The host-side
logic runs here as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, loc = bench.dist_setup()
        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slower replica
        ms = bench.replica_max_ms(local_ms, dist, torch.device("cpu"))
        rate = bench.job_gdof_s(w, 1000, 4, ms)
        dist.barrier()
        q.put((r, w, loc, ms, rate))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_count_both():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 and o[2] == o[0] for o in out)
    # both ranks agree on the slowest replica's time
    assert all(o[3] == 15.0 for o in out)
    # 2 replicas x 5 stages x 1000 DOF x 4 steps in 15 ms
    expect = 2 * 5 * 1000 * 4 / 15e-3 / 1e9
    assert all(o[4] == pytest.approx(expect) for o in out)


def test_single_process_is_its_own_job():
    assert bench.replica_max_ms(7.5, None, None) == 7.5
    assert bench.job_gdof_s(1, 1000, 4, 10.0) == pytest.approx(5 * 1000 * 4 / 10e-3 / 1e9)
