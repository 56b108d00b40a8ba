"""The multi-rank host logic of bench.py on CPU, with two gloo ranks: rank
environment parsing, the max-over-ranks reduction of the timed region, the
whole-job rate, and the reference arm's other ranks exiting without work."""

import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    total_ms = 10.0 + 5.0 * r                 # rank 1 is the slower one
    m = bench.max_over_ranks(total_ms, w, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, r, w, local, m))


def test_two_gloo_ranks_take_the_slowest_timed_region():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, (r0, r, w, local, m) in enumerate(out):
        assert (r0, r, w, local) == (rank, rank, 2, rank)
        assert m == 15.0                     # both ranks see the slowest rank's time


def test_job_rate_counts_every_rank():
    import bench
    # two ranks of 100 steps each in 15 ms (the slowest rank): 200 steps / 15 ms
    assert bench.job_rate(2, 100, 15.0) == pytest.approx(200 / 0.015)
    assert bench.job_rate(1, 100, 15.0) == pytest.approx(100 / 0.015)
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5


def test_reference_arm_other_ranks_do_no_work():
    import argparse
    import bench
    args = argparse.Namespace(steps=1, warmup=1)
    assert bench.run_reference(args, 1, 2) == 0
