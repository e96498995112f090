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


def _replica_rank(rank, world, port, q):
    """One rank of the replicas path with the oracle standing in for the GPU
    tick: its own replica world (bench.replica_ticks), answered exactly, the
    timed region's max over ranks, the whole-job throughput."""
    import time

    import numpy as np
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MQR_DIST_BACKEND="gloo")
    import bench
    import oracle
    dist, r, w, local = bench.dist_setup(world)
    ticks = bench.replica_ticks("uniform16k", r, 3)
    st = oracle.State(ticks[0].ids.shape[0])
    bench.barrier(dist, None)
    t0 = time.perf_counter()
    answers = []
    for t in ticks:
        st.apply_updates(t.ids, t.xy)
        answers.append(oracle.count_grid(st, t.rects, cell_side=0.01))
    ms = 1000.0 * (time.perf_counter() - t0)
    bench.barrier(dist, None)
    t_max = bench.reduce_max(dist, ms, None)
    # the last tick answered again by brute force: exact for this rank's own world
    off, _ = oracle.join_brute(st, ticks[-1].rects)
    exact = bool(np.array_equal(np.diff(off.astype(np.int64)), answers[-1].astype(np.int64)))
    Q = sum(t.rects.shape[0] for t in ticks)
    q.put((r, ms, t_max, w * Q / (t_max / 1000.0), float(ticks[0].xy[0, 0]), exact))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_answer_independent_replica_worlds():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    (r0, ms0, max0, v0, x0, ok0), (r1, ms1, max1, v1, x1, ok1) = got
    assert ok0 and ok1                                   # each rank's answers are exact for its world
    assert x0 != x1                                      # the replicas are different worlds
    assert max0 == max1 == max(ms0, ms1)                 # the timed region is the slower rank's
    assert v0 == v1


def test_reference_arm_under_torchrun_prints_one_line():
    """`bench.py --impl reference` launched by torchrun with two ranks (gloo):
    rank 0 alone times the oracle and prints the JSON line; rank 1 exits 0."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, MQR_DIST_BACKEND="gloo")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(root, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--workload", "uniform16k", "--steps", "3", "--warmup", "3"]
    p = subprocess.run(cmd, cwd=root, env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
