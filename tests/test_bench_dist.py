"""The multi-rank host logic of bench.py on CPU: under a world-size-2 gloo process
group each rank reports its own elapsed time and work; the aggregate is the
slowest rank's time and the sum of the work (weak scaling of independent
replicas, no data-path collective)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench.dist_env() == (world, rank, rank)
    ms, units = bench.reduce_timing(10.0 + 5.0 * rank, 4.0 * (rank + 1))
    bench.barrier()
    out.put((rank, ms, units))
    dist.destroy_process_group()


def test_reduce_timing_over_two_gloo_ranks():
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 15.0, 12.0), (1, 15.0, 12.0)]


def test_reduce_timing_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_timing(3.5, 7.0) == (3.5, 7.0)
