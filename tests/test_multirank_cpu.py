"""Multi-rank paths of bench.py on CPU: gloo, world size 2.

Ranks render independent replicas; the only collective is the timing
aggregation (max of the ranks' times, sum of their frames), and the
reference arm runs on rank 0 alone."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 10 + 5 r ms for 8 (r + 1) frames
        q.put((rank, bench.aggregate_over_ranks(10.0 + 5.0 * rank, 8 * (rank + 1), world, None)))
    finally:
        dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest time and the total frames
    assert got[0] == (15.0, 24) and got[1] == (15.0, 24)


def test_single_rank_aggregation_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(12.5, 7, 1) == (12.5, 7)


def test_reference_arm_runs_on_rank0_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference", "--gpus", "2"]) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_times_whole_frames(capsys):
    # rank 0 (no torchrun): whole oracle frames of a small scene; the timed steps fit
    # inside the call's own wall time, so the line's ms_per_step x steps is real
    import json
    import time
    sys.path.insert(0, ROOT)
    import bench
    t0 = time.perf_counter()
    assert bench.main(["--impl", "reference", "--gaussians", "3000", "--width", "96", "--height", "64",
                       "--steps", "2", "--warmup", "3"]) == 0
    wall_ms = (time.perf_counter() - t0) * 1e3
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 3
    assert line["value"] > 0 and line["unit"] == "frames/s"
    assert abs(line["value"] * line["ms_per_step"] * 1e-3 - 1.0) < 1e-9
    assert line["ms_per_step"] * line["steps"] <= wall_ms
    assert "whole" in line["cpu_baseline"]["sample"] and line["e2e"]["h2d_bytes_per_step"] == 0
