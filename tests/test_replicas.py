"""Host logic of multi-GPU runs (replicas, no data-path collective), on the
CPU with two gloo ranks: the whole-job rate is the units of all ranks over
the slowest rank's time, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        units = 100.0 * (rank + 1)      # 100 and 200 site updates
        seconds = 2.0 + 2.0 * rank      # 2 s and 4 s
        rate, slowest = bench.job_rate(dist, units, seconds, device="cpu")
        out.put((rank, rate, slowest))
    finally:
        dist.destroy_process_group()


def test_job_rate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(out.get(timeout=10) for _ in procs)
    for _, rate, slowest in got:
        assert slowest == 4.0
        assert rate == pytest.approx(300.0 / 4.0)


def test_job_rate_single_process():
    import bench

    assert bench.job_rate(None, 50.0, 2.0) == (25.0, 2.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = type("A", (), {"steps": 1, "warmup": 0})()
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""
