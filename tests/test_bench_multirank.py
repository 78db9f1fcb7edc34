"""The multi-rank leg of bench.py on CPU: world size 2 over gloo.  Each rank
is an independent replica; the whole-job rate counts every rank's node
updates over the slowest rank's time."""
import os
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

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dt = 0.5 if rank == 0 else 2.0          # rank 1 is the slow one
        units = 1000 * (rank + 1)
        dtm, total = bench.aggregate(dt, units, dist)
        out[rank] = (dtm, total)
    finally:
        dist.destroy_process_group()


def test_aggregate_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(2):
            assert out[r] == (2.0, 3000.0)


def test_aggregate_single_process():
    import bench

    assert bench.aggregate(1.5, 42, None) == (1.5, 42)


def test_reference_arm_other_ranks_do_nothing(capsys):
    """Under torchrun only rank 0 runs and prints the reference line."""
    import argparse

    import bench

    args = argparse.Namespace(steps=1, warmup=3, lattice="d3q19", n=0, precision="fp32")
    bench.run_reference(args, rank=1, world=2)
    assert capsys.readouterr().out == ""
