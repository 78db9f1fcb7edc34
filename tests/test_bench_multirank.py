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


def test_reference_arm_line(capsys):
    """Rank 0 of the reference arm times the oracle on the host and prints
    one JSON line with the contract's keys (no GPU needed)."""
    import argparse
    import json

    import bench

    args = argparse.Namespace(steps=2, warmup=3, lattice="d3q19", n=0, precision="fp32")
    bench.run_reference(args, rank=0, world=1)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT
    assert line["metric"] == bench.METRIC and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_traffic_record_follows_the_kernel_sources(tmp_path, monkeypatch):
    """A DRAM traffic record counts only while the kernel sources hash to the
    value recorded with it."""
    import json

    import bench

    (tmp_path / "profiles").mkdir()
    rec = {"k": {"kernel_hash": bench.kernel_hash(), "dram_bytes_per_launch": 1}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    for p in bench.KERNEL_SOURCES:       # the same sources under the temporary root
        dst = tmp_path / p
        dst.parent.mkdir(parents=True, exist_ok=True)
        dst.write_bytes(open(os.path.join(os.path.dirname(os.path.dirname(
            os.path.abspath(__file__))), p), "rb").read())
    assert bench.traffic_record("k")["dram_bytes_per_launch"] == 1
    assert bench.traffic_record("missing") is None
    with open(tmp_path / bench.KERNEL_SOURCES[0], "ab") as fh:
        fh.write(b"\n// changed\n")
    assert bench.traffic_record("k") is None
