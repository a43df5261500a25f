"""Multi-rank paths on CPU ranks (gloo, world size 2, 127.0.0.1).

* bench.py's weak-scaling coordination: each rank's problem shares L, W, R and has its
  own two-site tensor; the job time is the maximum over ranks;
* the row-sharded apply through bench.py's own step (``sharded_step``: zero y, write this
  rank's blocks, all-reduce): each rank plans its shard of y's left sectors and executes
  the plan's tables on the CPU (the table interpreter of the host tests) in place of the
  GPU apply; the all-reduced y equals the oracle's on every rank.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _bench_worker(rank, world, port):
    _init(rank, world, port)
    try:
        import bench
        assert bench.max_over_ranks(1.0 + rank, "cpu") == float(world)
        assert bench.sum_over_ranks(1.0 + rank, "cpu") == float(world * (world + 1) // 2)
        assert bench.rank_batch(rank) == rank
        # the ranks' two-site tensors differ, their environments agree
        _, lays, bufs = bench.make_problem("spin_m24", bench.rank_batch(rank))
        x = torch.from_numpy(np.asarray(bufs["x"]))
        L = torch.from_numpy(np.asarray(bufs["L"]))
        xs = [torch.zeros_like(x) for _ in range(world)]
        Ls = [torch.zeros_like(L) for _ in range(world)]
        dist.all_gather(xs, x)
        dist.all_gather(Ls, L)
        assert not torch.equal(xs[0], xs[1])
        assert torch.equal(Ls[0], Ls[1])
    finally:
        dist.destroy_process_group()


def _shard_worker(rank, world, port, name):
    _init(rank, world, port)
    try:
        import workloads as wl
        from oracle import heff as oh
        from paper_2007_05540_gb300 import heff
        from tests.helpers import library_problem, interpret_plan, oracle_flat
        w = wl.workload_by_name(name)
        lays, bufs = library_problem(w)
        xl = lays[4]
        import bench
        P = heff.Plan(*lays, bufs["W1"], bufs["W2"], "fp64", "f64", shard=(rank, world))

        def apply_shard(out):
            # the shard plan's tables executed on the CPU: this rank's y blocks only
            ys = interpret_plan(P, bufs, bufs["x"][0])
            keep = ~np.isnan(ys)
            out.numpy()[keep] = ys[keep]
        # bench.py's row-sharded step: zero y, this rank's blocks, all-reduce
        t = torch.full((xl.nelem,), float("nan"), dtype=torch.float64)
        bench.sharded_step(apply_shard, t)
        L, W1, W2, R, x = oh.problem_from_workload(w)
        y_ref = oracle_flat(xl, oh.heff_apply(L, W1, W2, R, x))
        err = np.abs(t.numpy() - y_ref).max() / np.abs(y_ref).max()
        assert err < 1e-12, err
        n = torch.tensor([len(heff.heff_plan_shard_sectors(P.handle))])
        dist.all_reduce(n)
        assert int(n) == len(w.alpha_d)
    finally:
        dist.destroy_process_group()


def test_bench_rank_coordination_gloo():
    import torch.multiprocessing as mp
    mp.spawn(_bench_worker, args=(2, _free_port()), nprocs=2, join=True)


@pytest.mark.parametrize("name", ["spin_m64", "electron_m40"])
def test_row_sharded_apply_allreduce_gloo(name):
    import torch.multiprocessing as mp
    mp.spawn(_shard_worker, args=(2, _free_port(), name), nprocs=2, join=True)
