"""Host logic of bench.py's N > 1 path (independent replicas, no data-path collective):
two gloo ranks on CPU agree on the slowest rank's time, the whole-job throughput counts
every rank's keys, and the reference arm runs on rank 0 alone."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        ms = bench.max_over_ranks(torch, 1.0 + rank, world, "cpu")
        e2e = bench.e2e_over_ranks(torch, {"value": 0.0, "unit": bench.UNIT,
                                           "ms_per_step": 2.0 + 3.0 * rank,
                                           "keys_per_step": 1000}, world, "cpu")
        torch.distributed.barrier()
        q.put((rank, ms, e2e))
    finally:
        torch.distributed.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_count_every_rank():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, e2e in res:
        assert ms == 2.0, rank  # the slower rank's 2.0 ms, on both ranks
        assert e2e["ms_per_step"] == 5.0
        assert e2e["value"] == pytest.approx(2 * 1000 / 5e-3 / 1e9)


def test_one_rank_keeps_its_own_figures():
    import bench

    assert bench.max_over_ranks(None, 3.5, 1, "cpu") == 3.5
    e2e = {"value": 7.0, "ms_per_step": 2.0, "keys_per_step": 14_000_000}
    assert bench.e2e_over_ranks(None, e2e, 1, "cpu") is e2e
    assert bench.job_throughput(1 << 29, 4, 3.75) == pytest.approx(4 * (1 << 29) / 3.75e-3 / 1e9)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "3", "--warmup", "3"], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
