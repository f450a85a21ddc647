"""Replicas on several processes (the multi-GPU mode of the benchmark: one
independent evaluation per rank, no data-path collective): the timing is the
slowest rank's and the whole-job rate counts every rank's points.  Host logic
only, on world_size-2 gloo ranks on the CPU."""
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


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [2.0, 3.5][rank]
        dist.barrier()
        ms = bench._max_over_ranks(local_ms, dist, torch.device("cpu"))
        out.put((rank, ms, bench._whole_job_rate(bench.N_POINTS, world, ms)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    import bench

    for rank, ms, rate in res:
        assert ms == 3.5  # both ranks see the slowest rank's time
        assert rate == pytest.approx(2 * bench.N_POINTS / 3.5e-3 / 1e6)


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench._max_over_ranks(1.25, None, None) == 1.25
    assert bench._whole_job_rate(1_000_000, 1, 4.0) == pytest.approx(250.0)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the reference arm (the oracle on the host) runs on rank 0
    alone; the other ranks exit 0 without work or output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
