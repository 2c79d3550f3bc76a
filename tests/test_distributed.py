"""The multi-rank path of bench.py on CPU: independent replicas (one matrix per rank, no collective on the
data path), timed by the slowest rank, reported as whole-job throughput; gloo, world size 2."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    ms = 100.0 + 50.0 * rank          # rank 1 is the slow replica
    ms_max = bench.max_over_ranks(ms, w, "cpu")
    out.put((rank, r, w, local, ms_max, bench.replica_rate(2, w, ms_max)))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_time_by_slowest_rank_and_sum_throughput():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, w, local, ms_max, value in res:
        assert (r, w, local) == (rank, 2, rank)
        assert ms_max == 150.0                     # every rank sees the slowest replica's time
        assert abs(value - 2 * 2 / 0.150) < 1e-9   # all ranks' factorizations over that time


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(123.0, 1, "cpu") == 123.0
    assert bench.replica_rate(2, 1, 500.0) == 4.0


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
