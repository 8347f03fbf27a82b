"""The multi-rank host logic of bench.py on CPU: two gloo ranks.

The path shards by realisation (independent problems, weak scaling): each
rank times its own replica, the job's time is the slowest rank's, and the
job's value counts the units of every rank.  The reference arm (the FP64
oracle) runs on rank 0 only; the other ranks leave without work.
"""
import os
import socket
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    sys.path.insert(0, str(ROOT))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        t = 1.0 + rank                      # rank 1 is the slow one
        t_max = bench._max_over_ranks(t, ws, "cpu")
        e2e = bench._max_over_ranks(10.0 - rank, ws, "cpu")
        q.put((rank, t_max, e2e, bench._job_value(1000.0, 4, ws, t_max)))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_the_slowest_time_and_count_every_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=90) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, t_max, e2e, value in got:
        assert t_max == 2.0 and e2e == 10.0
        assert value == 1000.0 * 4 * 2 / 2.0


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, str(ROOT))
    import bench
    assert bench._max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench._job_value(16384, 10, 1, 0.5) == 16384 * 10 / 0.5


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, str(ROOT))
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class A:
        steps, warmup = 1, 0

    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""


def test_gpus_flag_must_match_the_world_size():
    """bench.py --gpus N under a launcher with another WORLD_SIZE refuses to
    run instead of reporting the wrong n_gpus."""
    import subprocess
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    res = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--gpus", "2", "--steps", "1"],
                         capture_output=True, text=True, env=env, cwd=str(ROOT), timeout=120)
    assert res.returncode == 2, (res.returncode, res.stderr[-500:])
    assert "WORLD_SIZE=1" in res.stderr
