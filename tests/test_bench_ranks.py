"""The multi-rank bookkeeping of bench.py (replicas, one per GPU): the job time is
the largest time over the ranks and the job throughput sums the replicas.  Runs
two gloo ranks on the CPU (no GPU involved)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 5.0 + 2.5 * rank            # rank 1 is the slow one
        ms = bench.max_over_ranks(ms_local)
        out[rank] = (ms, bench.job_gbs(4.0 * 1024 * 512, 3, world, ms))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 7.5
    expect = 4.0 * 1024 * 512 * 3 * world / 7.5e-3 / 1e9
    assert res[0][1] == pytest.approx(expect) and res[1][1] == pytest.approx(expect)


def test_single_process_is_identity():
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.job_gbs(1e9, 2, 1, 1000.0) == pytest.approx(2.0)
