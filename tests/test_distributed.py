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


def _acc_worker(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist
    import bench
    import oracle as O
    from tests.test_oracle import SYSTEMS, tiny
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    s = tiny(**SYSTEMS["1c2a2v"])
    o = O.Oracle.from_system(s)
    G = bench.groups_per_rank(world)
    acc = o.sample(64, 200, 20, seed=500 + rank, n_groups=G)      # each rank its own walkers and seed
    acc = {k: acc[k] for k in ("N", "U", "W", "E", "A", "B")}
    acc["type_steps"] = np.zeros(9, np.int64)
    acc["type_steps"][0] = 64 * 180
    acc["total_steps"] = 64 * 200
    objs = [None] * world
    dist.all_gather_object(objs, acc)
    merged = bench.merge_rank_accumulators(objs)
    in_order = all(np.array_equal(merged[k][r * G:(r + 1) * G], objs[r][k])
                   for k in ("N", "U", "W", "E", "A", "B") for r in range(world))
    out[rank] = (merged["N"].shape[0], merged["total_steps"], float(o.finalize(merged)["e2"]),
                 float(o.finalize(merged)["e2_sigma"]),
                 [float(o.finalize({k: v for k, v in a.items()})["e2"]) for a in objs], in_order,
                 int(merged["type_steps"][0]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_combine_their_walker_groups():
    """The cross-rank reduction: every rank's groups gathered, concatenated in rank order and
    finalized as one run; the union's estimate is the weighted combination of the ranks' (the
    sums add up) and both ranks see the same union."""
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_acc_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    g0, n0, e0, s0, per0, ord0, t0 = out[0]
    g1, n1, e1, s1, per1, ord1, t1 = out[1]
    assert ord0 and ord1 and t0 == t1 == 2 * 64 * 180
    import bench
    assert g0 == g1 == 2 * bench.groups_per_rank(2)
    assert n0 == n1 == 2 * 64 * 200
    assert e0 == e1 and s0 == s1 and s0 > 0
    assert per0 == per1 and per0[0] != per0[1]
    assert abs(e0 - 0.5 * sum(per0)) < 5 * s0


def test_groups_per_rank_keeps_the_union_within_64():
    import bench
    for w in (1, 2, 3, 4, 5, 8, 16, 64, 100):
        assert 1 <= bench.groups_per_rank(w) <= 16
        assert w * bench.groups_per_rank(w) <= 64 or bench.groups_per_rank(w) == 1


class _FakeCtx:
    """Stands in for a device context: fixed per-group sums, and it records what rank 0 loads."""

    def __init__(self, rank, G, L):
        import numpy as np
        rng = np.random.default_rng(100 + rank)
        self.acc = dict(N=rng.random((G, L)), U=rng.random((G, L)), W=rng.random(G), E=rng.random(G),
                        type_steps=np.full(9, rank + 1, np.int64))
        self.grad = (rng.random((G, L)), rng.random((G, L)))
        self.loaded = None

    def accumulators(self, G):
        return {k: v.copy() for k, v in self.acc.items()}

    def gradient_sums(self, G):
        return self.grad

    def load_accumulators(self, acc, total_steps=0):
        self.loaded = (acc, total_steps)

    def finalize(self):
        a, _ = self.loaded
        return dict(e2=float(a["E"].sum()), e2_sigma=1.0, e_var=float(a["W"].sum()), e_var_sigma=2.0)


def _combine_worker(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    G = bench.groups_per_rank(world)
    ctx = _FakeCtx(rank, G, 5)
    res = bench.combine_ranks(ctx, G, world, rank, total_steps=1000 * (rank + 1))
    if rank == 0:
        acc, steps = ctx.loaded
        others = [_FakeCtx(r, G, 5) for r in range(world)]
        ok = all(np.array_equal(acc["N"][r * G:(r + 1) * G], others[r].acc["N"]) and
                 np.array_equal(acc["A"][r * G:(r + 1) * G], others[r].grad[0]) for r in range(world))
        out[0] = (res, steps, ok, int(acc["type_steps"][0]))
    else:
        out[rank] = (res,)
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_loads_the_union_on_rank_zero_only():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_combine_worker, args=(3, port, out), nprocs=3, start_method="spawn", join=True)
    res, steps, ok, t0 = out[0]
    import bench
    assert ok and steps == 1000 + 2000 + 3000 and t0 == 1 + 2 + 3
    assert res["groups"] == 3 * bench.groups_per_rank(3) and res["walker_steps"] == 6000
    assert out[1] == (None,) and out[2] == (None,)
