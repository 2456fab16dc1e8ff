"""The multi-rank path of bench.py on CPU: two gloo ranks, as torchrun would
launch them (one process per GPU, max-over-ranks timing, whole-job
throughput, a barrier), and the reference arm's rank > 0 no-op.  No GPU and
no data-path collective: the ranks only agree on the step time."""
import os
import socket

import pytest
import torch
import torch.distributed as tdist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_setup()
        assert (r, w, local) == (rank, world, rank)
        bench.barrier(world)
        local_ms = 3.0 if rank == 0 else 5.0  # rank 1 is the slow one
        ms, rate = bench.job_rate(local_ms, 10 ** 9, world, torch.device("cpu"))
        out[rank] = (ms, rate)
        bench.barrier(world)
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        ms, rate = out[rank]
        assert ms == pytest.approx(5.0)
        assert rate == pytest.approx(world * 10 ** 9 / 5e-3 / 1e9)  # 400 Gkeys/s: both ranks' keys / max time


def test_single_rank_needs_no_process_group():
    ms, rate = bench.job_rate(2.0, 10 ** 9, 1, torch.device("cpu"))
    assert ms == 2.0 and rate == pytest.approx(500.0)
    bench.barrier(1)  # no-op


def test_reference_arm_other_ranks_do_nothing(capsys):
    class A:
        pass

    args = A()
    args.workload, args.cpu_sample, args.warmup, args.steps, args.gpus = "plain_u32_1M", 1024, 0, 1, 2
    assert bench.run_reference(args, dict(bench.WORKLOADS["plain_u32_1M"]), 2, 1) == 0
    assert capsys.readouterr().out == ""
