"""The multi-rank path of bench.py on CPU: world size 2 over gloo.

Each rank runs its own replica (weak scaling); the job's time is the slowest
rank's and the value counts the work of every rank.  The reference arm runs
on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.0 + rank, dist, device="cpu")
    out.put((rank, t, bench.job_value(world, 3, 100.0, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.0, 2.0]
    assert all(r[2] == pytest.approx(2 * 3 * 100.0 / 2.0) for r in res)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.job_value(1, 4, 10.0, 2.0) == 20.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import argparse

    import bench
    args = argparse.Namespace(workload="er4096", warmup=0, steps=1, gpus=2)
    bench.run_reference(args, rank=1, world=2)
    assert capsys.readouterr().out == ""


def test_traffic_record_only_for_its_workload_and_source():
    """roofline.traffic comes from profiles/traffic.json only for the workload
    and the kernel source it was captured on."""
    import hashlib
    import json

    import bench
    recs = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))["records"]
    assert recs
    for rec in recs:
        src = os.path.join(bench.ROOT, "paper_1408_6282_gb300", "csrc", rec["source"])
        current = hashlib.sha256(open(src, "rb").read()).hexdigest() == rec["source_sha256"]
        got = bench.traffic_record(rec["kernel"], rec["workload"])
        assert (got is not None) == current
        if got is not None:
            assert got["dram_bytes_per_launch"] == rec["dram_bytes_per_launch"]
        assert bench.traffic_record(rec["kernel"], rec["workload"] + "_other") is None
    assert bench.traffic_record("no_such_kernel", "rmat20_wc") is None
