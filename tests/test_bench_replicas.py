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


def test_reference_arm_prints_the_contract_line(monkeypatch):
    """Rank 0 of the reference arm on a small grid: one JSON line with the
    contract's keys, the oracle's sample no larger than the scene, and the
    e2e and cpu_baseline objects describing the same run."""
    import json
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--n", "16",
                                      "--steps", "1", "--warmup", "0"])
    args = bench.parse_args()
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.reference_arm(args) == 0
    lines = [ln for ln in buf.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 0
    from paper_2308_01060_gb300 import scenes
    n_scene = scenes.dam_break_scene(n=16, R=27).fluid.n
    assert 0 < line["config"]["sample_particles_per_step"] <= n_scene
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


@pytest.mark.parametrize("n", [32, 128])
def test_bench_names_the_realised_dam_break_block(n):
    """The workload line's block (the corner block clipped to the 2-cell wall
    margin) times 8 particles per cell is the scene's particle count."""
    from paper_2308_01060_gb300 import scenes
    d = bench.block_cells(n)
    P = scenes.dam_break_scene(n=n, R=1).fluid.n
    assert d[0] * d[1] * d[2] * 8 == P
    text = bench.workload_name(n, P, 200)
    assert f"dam_break_{n}^3" in text and f"({P} particles)" in text
    assert "x".join(map(str, d)) + " cells" in text
