"""The multi-GPU path of bench.py runs independent replicas (galaxies do not
exchange anything): ranks meet only at barriers, the timing is the slowest
rank's, and the job's throughput counts every rank's galaxies.  Checked with
two gloo ranks on the CPU (the same helpers run over NCCL on GPUs)."""

import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        bench.barrier(world)
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world)   # rank 1 is the slow one
        q.put((rank, ms, bench.job_throughput(1000, world, ms)))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_count_both():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, ms, value in got:
        assert ms == 15.0, (rank, ms)
        assert abs(value - 2 * 1000 / 0.015) < 1e-6 * value


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    bench.barrier(1)
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_throughput(100, 1, 1000.0) == 100.0
