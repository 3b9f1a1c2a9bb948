"""Multi-GPU path of bench.py (independent replicas), run as world-size-2 gloo
ranks on the CPU: rendezvous, barriers, maximum over ranks of the timed
region, whole-job throughput, and the reference arm running on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w, local = bench.dist_setup(world, backend="gloo")
    assert (r, w, local) == (rank, world, rank)
    bench.barrier(w)
    # each rank "timed" a different duration; the job time is the slowest
    ms_max = bench.barrier_max(w, 10.0 + 5.0 * r)
    value = bench.replica_value(1000, w, ms_max)
    q.put((r, ms_max, value))
    dist.destroy_process_group()


def test_two_replicas_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for r, ms_max, value in got:
        assert ms_max == 15.0
        assert value == pytest.approx(1000 * 2 / 0.015)


def test_reference_arm_rank_gate(monkeypatch):
    """Under torchrun only rank 0 runs the reference arm; others exit 0."""
    sys.path.insert(0, ROOT)
    import bench

    class A:
        workload = "rmat"
        steps = 1
        warmup = 0
        gpus = 2
    assert bench.run_reference(A(), 1, 2) == 0
