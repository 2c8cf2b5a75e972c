"""The benchmark's N > 1 orchestration (one independent walker set per rank, no data-path
collective, barrier-bracketed timing, max over ranks) with two gloo ranks on the CPU."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    dist.barrier()
    ms = 100.0 + 50.0 * rank                     # rank 1 is the slow one
    got = bench.max_over_ranks(ms, world)
    out[rank] = (got, bench.job_rate(4096, world, got), bench.rank_seed(rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_distinct_seeds():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    r0, r1 = out[0], out[1]
    assert r0[0] == r1[0] == 150.0
    assert r0[1] == pytest.approx(2 * 4096 / 0.150)
    assert r0[2] != r1[2]


def test_reference_arm_other_ranks_do_nothing(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(bench.argparse.Namespace(steps=1, warmup=0, cpu_seconds=1.0, gpus=2))
    assert capsys.readouterr().out == ""
