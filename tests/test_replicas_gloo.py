"""The multi-GPU path of bench.py is replicas only: every rank runs an
independent lattice, the ranks meet at a barrier, and the job's time is the
slowest rank's.  Checked here with world size 2 on the gloo backend (CPU):
the max-over-ranks reduction and the whole-job throughput."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = 1.5 + rank          # rank 1 is the slower replica
    tmax = bench.max_over_ranks(t, dist, "cpu")
    out.put((rank, tmax, bench.replica_throughput(world, 4, tmax)))
    dist.destroy_process_group()


def test_two_replicas_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, thr in res:
        assert tmax == pytest.approx(2.5)
        assert thr == pytest.approx(2 * 4 / 2.5)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    assert bench.replica_throughput(1, 2, 4.0) == pytest.approx(0.5)
