"""Batched independent worlds in one index: every world's results must be the
oracle's for that world alone (and the same as a context holding only that
world), leaves must never span two worlds, and empty worlds / world counts
that are not powers of 4 must work."""
import numpy as np
import pytest

import oracle
from paper_1411_3212_gb300 import workloads
from tests.gpu_util import assert_same_csr, gpu_csr_sorted, gpu_pairs_as_csr, to_dev, torch_dev

pytestmark = pytest.mark.gpu


def world_oracle(tick, w):
    a, b = int(tick.obj_base[w]), int(tick.obj_base[w + 1])
    qa, qb = int(tick.q_base[w]), int(tick.q_base[w + 1])
    st = oracle.State(max(b - a, 1))
    if b > a:
        st.apply_updates(np.arange(b - a, dtype=np.uint32), tick.xy[a:b])
    off, ids = oracle.join_grid(st, tick.rects[qa:qb], cell_side=0.01)
    return off, ids + np.uint32(a)


@pytest.mark.parametrize("n_worlds,cap,seed", [(16, 32, 3), (5, 64, 4), (64, 16, 5)])
def test_each_world_alone_equals_batched(n_worlds, cap, seed):
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    bw = workloads.BatchedWorlds(n_worlds=n_worlds, n_lo=50, n_hi=4000, q_frac=0.2, side=0.02, seed=seed)
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=cap, max_objects=bw.n)
    idx.set_worlds(bw.obj_base)
    for tick_no in range(2):
        t = bw.next_tick()
        idx.set_query_worlds(t.q_base)
        idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
        off, ids = gpu_csr_sorted(idx, t.rects, dev)
        poff, pids = gpu_pairs_as_csr(idx, t.rects, dev)
        assert np.array_equal(off, poff) and np.array_equal(ids, pids)
        for w in range(n_worlds):
            qa, qb = int(t.q_base[w]), int(t.q_base[w + 1])
            got = (off[qa:qb + 1] - off[qa], ids[int(off[qa]):int(off[qb])])
            assert_same_csr(got, world_oracle(t, w), "world %d tick %d" % (w, tick_no))
        # no leaf spans two worlds
        lv = idx.leaves()
        _, sid = idx.sorted_objects()
        world_of_id = np.searchsorted(t.obj_base, sid, side="right") - 1
        for lvl, z, b, e in lv:
            assert world_of_id[b] == world_of_id[e - 1], (lvl, z)
        bits = 0
        while 4 ** bits < n_worlds:
            bits += 1
        assert lv[:, 0].min() >= bits
    # the same world alone in its own context
    w = 1
    a, b = int(t.obj_base[w]), int(t.obj_base[w + 1])
    qa, qb = int(t.q_base[w]), int(t.q_base[w + 1])
    alone = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=cap, max_objects=b - a)
    alone.apply_updates(to_dev(np.arange(b - a, dtype=np.uint32), dev), to_dev(t.xy[a:b], dev))
    aoff, aids = gpu_csr_sorted(alone, t.rects[qa:qb], dev)
    np.testing.assert_array_equal(aoff, off[qa:qb + 1] - off[qa])
    np.testing.assert_array_equal(aids + np.uint32(a), ids[int(off[qa]):int(off[qb])])
    alone.close()
    idx.close()


def test_worlds_with_empty_members_and_argument_checks():
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    # 4 worlds: world 1 has no objects, world 2 has no queries
    rng = np.random.default_rng(9)
    obj_base = np.array([0, 300, 300, 700, 1000], np.uint32)
    xy = rng.random((1000, 2)).astype(np.float32)
    q_base = np.array([0, 40, 80, 80, 120], np.uint32)
    c = rng.random((120, 2)).astype(np.float32)
    rects = workloads.squares_around(c, 0.1)
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=8, max_objects=1000)
    with pytest.raises(mqr.MqrError):
        idx.set_worlds(np.array([0, 10, 999], np.uint32))          # must end at max_objects
    with pytest.raises(mqr.MqrError):
        idx.set_worlds(np.array([0, 600, 500, 1000], np.uint32))   # decreasing
    with pytest.raises(mqr.MqrError):
        mqr.mqr_set_query_worlds(idx.ctx, q_base)                  # no worlds yet
    idx.set_worlds(obj_base)
    idx.apply_updates(to_dev(np.arange(1000, dtype=np.uint32), dev), to_dev(xy, dev))
    with pytest.raises(mqr.MqrError, match="Q must equal"):
        idx.tick(to_dev(rects, dev), kind="csr_sorted")           # query ranges not set
    idx.set_query_worlds(q_base)
    off, ids = gpu_csr_sorted(idx, rects, dev)
    tick = workloads.BatchedTick(np.arange(1000, dtype=np.uint32), xy, rects, obj_base, q_base)
    for w in range(4):
        qa, qb = int(q_base[w]), int(q_base[w + 1])
        got = (off[qa:qb + 1] - off[qa], ids[int(off[qa]):int(off[qb])])
        assert_same_csr(got, world_oracle(tick, w), "world %d" % w)
    # back to one world: the same objects answer as a single world
    idx.set_worlds(np.array([0, 1000], np.uint32))
    st = oracle.State(1000)
    st.apply_updates(np.arange(1000, dtype=np.uint32), xy)
    assert_same_csr(gpu_csr_sorted(idx, rects, dev), oracle.join_grid(st, rects, cell_side=0.01))
    idx.close()
