"""Host-side logic of the multi-rank bench (replicas only: one independent replica per rank,
no collective on the data path) with two gloo ranks on the CPU: the job's time is the
slowest rank's, its work the sum over ranks, and every rank agrees; the reference arm runs
on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seconds = 2.0 + rank  # rank 1 is the slower one
    atom_steps = 1000 * (rank + 1)
    value, tmax = bench.job_throughput(seconds, atom_steps, dist)
    q.put((rank, value, tmax))
    dist.barrier()
    dist.destroy_process_group()


def test_job_throughput_takes_the_slowest_rank_and_sums_the_work():
    import torch.multiprocessing as mp

    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, tmax in out:
        assert tmax == pytest.approx(3.0)
        assert value == pytest.approx(3000 / 3.0)


def test_single_process_throughput_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.job_throughput(4.0, 100.0) == (25.0, 4.0)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the ranks other than 0 exit 0 without work or output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--gpus", "2"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
