"""The benchmark's N > 1 path on the CPU: two gloo ranks, each with its own
(kept samples, seconds), aggregate to (sum of kept, max of seconds) -- the
replicas exchange nothing else."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    kept, secs = 1000.0 * (rank + 1), 2.0 + rank
    k, t = bench.gather_max_sum(dist, world, kept, secs, "cpu")
    out.put((rank, k, t, bench.aggregate([kept], [secs])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_kept_and_take_slowest():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, k, t, single in res:
        assert k == 3000.0 and t == 3.0
        assert single == (1000.0 * (rank + 1) / (2.0 + rank), 2.0 + rank)


def test_aggregate_single_rank():
    sys.path.insert(0, ROOT)
    import bench

    v, t = bench.aggregate([10.0, 30.0], [2.0, 4.0])
    assert (v, t) == (10.0, 4.0)
    assert bench.aggregate([1.0], [0.0]) == (0.0, 0.0)
    with pytest.raises(ValueError):
        bench.aggregate([], [])
