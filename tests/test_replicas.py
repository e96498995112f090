"""Host logic of the multi-process (replicas) benchmark path on CPU: two gloo
ranks, the max-over-ranks reduction of the timed region and the whole-job
throughput.  No GPU is involved."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MQR_DIST_BACKEND="gloo")
    import bench
    dist, r, w, local = bench.dist_setup(world)
    assert (r, w) == (rank, world)
    t = bench.reduce_max(dist, 10.0 + 5.0 * rank, None)       # rank 1 is the slower one
    value = w * 400_000 * 10 / (t / 1000.0)                    # queries/s of the whole job
    q.put((rank, t, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got[0][1] == got[1][1] == 15.0
    assert got[0][2] == pytest.approx(2 * 400_000 * 10 / 0.015)
