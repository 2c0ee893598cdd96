"""The multi-rank path of bench.py on the CPU (gloo, world size 2): the
transfers do not shard, so N ranks run N independent replicas; the job's
time is the slowest rank's and its throughput counts every rank's units.
Also: under a multi-rank launch only rank 0 runs the reference arm."""
import contextlib
import io
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(rank, world, port, ms_by_rank, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        out[rank] = bench.job_throughput(torch, ms_by_rank[rank], 1000, 10, world, "cpu")
    finally:
        dist.destroy_process_group()


def test_job_throughput_takes_the_slowest_rank_and_all_units():
    world, port = 2, _free_port()
    ms_by_rank = [40.0, 50.0]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_replica, args=(world, port, ms_by_rank, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, value = res[rank]
        assert ms == 50.0                                    # max over ranks
        assert value == pytest.approx(1000 * 2 * 10 / 50e-3 / 1e6)   # units of both ranks


def test_job_throughput_single_rank_needs_no_process_group():
    ms, value = bench.job_throughput(torch, 20.0, 500, 4, 1, "cpu")
    assert ms == 20.0 and value == pytest.approx(500 * 4 / 20e-3 / 1e6)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2",
                                      "--steps", "1", "--warmup", "0"])
    args = bench.parse_args()
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.reference_arm(args) == 0
    assert buf.getvalue() == ""
