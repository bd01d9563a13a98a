"""Multi-rank path of bench.py on CPU (gloo, world size 2).

The path does not shard on this pool (one GPU per box): N ranks run N
independent replicas of the workload, joined only by a barrier and the
max-over-ranks time.  These tests run that aggregation with two gloo ranks,
and the reference arm's rank rule (rank 0 alone times the oracle; the others
exit 0 without work)."""
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    dist.barrier()
    value, t = bench.replica_throughput(1.0 + rank, 5, world, "cpu")
    q.put((rank, value, t))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest replica's time; the job did 2 x 5 steps in it
    assert [t for _, _, t in out] == [2.0, 2.0]
    assert [v for _, v, _ in out] == [5.0, 5.0]


def test_replica_throughput_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_throughput(2.0, 4, 1, "cpu") == (2.0, 2.0)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
