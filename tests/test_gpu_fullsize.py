"""Full-size parity, in the launch configurations bench.py times: the
4M-object hotspot workload with 400,000 queries per tick (leaf_cap 128,
quadtree, pair-list output), the 1M-object uniform walk (quadtree and the
uniform grid it is compared with), the 256 batched worlds (12.3M objects) and
the 10M-object served state with admission, and hotspot-4M under per-region
capacities.  Every query's result count is
compared with the oracle's, and the complete id lists of a random sample of
queries are compared exactly; covering-compressed outputs must give the same
counts.
"""
import multiprocessing
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

import oracle
from paper_1411_3212_gb300 import workloads
from tests.gpu_util import to_dev, torch_dev
from tests.result_hash import per_query_hash

pytestmark = pytest.mark.gpu


def _oracle_counts_and_hashes(n, ids, xy, rects):
    """One tick of the oracle in a worker process: every query's Def. 1
    result count and checksum (cell 0.002)."""
    st = oracle.State(n)
    st.apply_updates(ids, xy)
    return oracle.count_grid(st, rects, cell_side=0.002, with_hash=True)


def test_hotspot_4m_every_query_checksum_five_ticks():
    """Ticks 1-5 of hotspot-4M at the bench's launch configuration (leaf_cap
    128, quadtree, pair-list output): every query's result count and its
    order-independent checksum of (query, id) equal the oracle's, so every
    query's complete id set is compared.  The oracle's ticks run in spawned
    worker processes while the GPU answers."""
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    w = workloads.HotspotWalk(n=4_000_000, q=400_000, seed=0)
    ticks = [w.next_tick() for _ in range(5)]
    with ProcessPoolExecutor(max_workers=5, mp_context=multiprocessing.get_context("spawn")) as pool:
        futs = [pool.submit(_oracle_counts_and_hashes, w.n, t.ids, t.xy, t.rects) for t in ticks]
        idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=128, max_objects=w.n)
        got = []
        for t in ticks:
            idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
            pairs, offs = idx.tick(to_dev(t.rects, dev), kind="pairs")
            off = offs.cpu().numpy().view(np.uint64)
            p = pairs[: int(off[-1])].cpu().numpy().view(np.uint32)
            assert np.all(np.diff(p[:, 0].astype(np.int64)) >= 0)          # grouped by ascending query
            got.append((np.diff(off.astype(np.int64)), per_query_hash(p, off)))
            del pairs, p
        idx.close()
        for k, (f, (cnt, hs)) in enumerate(zip(futs, got)):
            want_cnt, want_hs = f.result()
            np.testing.assert_array_equal(cnt, want_cnt.astype(np.int64), err_msg="tick %d counts" % (k + 1))
            bad = np.nonzero(hs != want_hs)[0]
            assert bad.size == 0, "tick %d: %d queries' id sets differ, first %d" % (k + 1, bad.size, bad[:1])


def test_hotspot_4m_full_size_counts_and_sampled_lists():
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    w = workloads.HotspotWalk(n=4_000_000, q=400_000, seed=0)
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=128, max_objects=w.n)
    st = oracle.State(w.n)
    rng = np.random.default_rng(7)
    for tick in range(2):
        t = w.next_tick()
        idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
        st.apply_updates(t.ids, t.xy)
        rects_d = to_dev(t.rects, dev)
        pairs, offs = idx.tick(rects_d, kind="pairs")
        off = offs.cpu().numpy().view(np.uint64).astype(np.int64)
        R = int(off[-1])
        assert pairs.shape[0] == R
        # every query: result count
        want_cnt = oracle.count_grid(st, t.rects, cell_side=0.002).astype(np.int64)
        np.testing.assert_array_equal(np.diff(off), want_cnt)
        # grouping by query: qidx column non-decreasing and matching the offsets
        q_col = pairs[:, 0]
        assert bool((q_col[1:] >= q_col[:-1]).all().item())
        # sampled queries: exact id lists
        sample = np.sort(rng.choice(t.rects.shape[0], size=1500, replace=False))
        s_off, s_ids = oracle.join_grid(st, t.rects[sample], cell_side=0.002)
        for k, q in enumerate(sample):
            a, b = int(off[q]), int(off[q + 1])
            seg = pairs[a:b].cpu().numpy().view(np.uint32)
            assert np.all(seg[:, 0] == q)
            np.testing.assert_array_equal(np.sort(seg[:, 1]), s_ids[int(s_off[k]):int(s_off[k + 1])])
        s = idx.stats()
        assert s["n_results"] == R and s["n_objects"] == w.n
        assert s["n_results_covering"] <= R
        # covering-compressed output of the same tick: per-query counts
        elems, eoffs = idx.tick(rects_d, kind="runs")
        e = elems.cpu().numpy().view(np.uint32)
        eoff = eoffs.cpu().numpy().view(np.uint64).astype(np.int64)
        assert eoff[-1] == e.shape[0] == R - s["n_results_covering"] + 2 * s["n_covering_runs"]
        run = (e[:, 0] & 0x80000000) != 0
        heads = np.nonzero(run)[0]
        counts = np.ones(e.shape[0], np.int64)
        counts[heads] = e[heads + 1, 0]
        counts[heads + 1] = 0
        csum = np.concatenate([[0], np.cumsum(counts)])
        np.testing.assert_array_equal(csum[eoff[1:]] - csum[eoff[:-1]], want_cnt)
        del elems, e, counts, csum
    idx.close()


def _check_counts_and_sample(idx, st, rects, rects_d, off_cell, rng, n_sample, dev, what):
    pairs, offs = idx.tick(rects_d, kind="pairs")
    off = offs.cpu().numpy().view(np.uint64).astype(np.int64)
    want_cnt = oracle.count_grid(st, rects, cell_side=off_cell).astype(np.int64)
    np.testing.assert_array_equal(np.diff(off), want_cnt, err_msg=what)
    sample = np.sort(rng.choice(rects.shape[0], size=min(n_sample, rects.shape[0]), replace=False))
    s_off, s_ids = oracle.join_grid(st, rects[sample], cell_side=off_cell)
    for k, q in enumerate(sample):
        a, b = int(off[q]), int(off[q + 1])
        seg = pairs[a:b].cpu().numpy().view(np.uint32)
        assert np.all(seg[:, 0] == q), what
        np.testing.assert_array_equal(np.sort(seg[:, 1]), s_ids[int(s_off[k]):int(s_off[k + 1])], err_msg=what)
    return want_cnt


@pytest.mark.parametrize("index", ["quadtree", "grid"])
def test_uniform_1m_full_size(index):
    """1M uniform objects, 100,000 queries of side 0.002 per tick, 3 ticks of
    the random walk: the quadtree at leaf_cap 128 and the uniform grid the
    bench compares it with (level 8), counts of every query and sampled lists."""
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    w = workloads.UniformWalk(n=1_000_000, q=100_000, seed=0)
    if index == "quadtree":
        idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=128, max_objects=w.n)
    else:
        idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=1, max_objects=w.n, index_kind=1, grid_level=8)
    st = oracle.State(w.n)
    rng = np.random.default_rng(3)
    for tick in range(3):
        t = w.next_tick()
        idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
        st.apply_updates(t.ids, t.xy)
        _check_counts_and_sample(idx, st, t.rects, to_dev(t.rects, dev), 0.004, rng, 1000, dev,
                                 "%s tick %d" % (index, tick))
    idx.close()


def test_batched_256_worlds_full_size():
    """The batched-worlds workload at full size (256 worlds, 12.3M objects,
    1.23M queries): every query's count against the oracle run on its world
    alone, and sampled id lists of a few worlds."""
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    bw = workloads.BatchedWorlds(n_worlds=256, seed=0)
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=128, max_objects=bw.n)
    idx.set_worlds(bw.obj_base)
    t = bw.next_tick()
    idx.set_query_worlds(t.q_base)
    idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
    pairs, offs = idx.tick(to_dev(t.rects, dev), kind="pairs")
    off = offs.cpu().numpy().view(np.uint64).astype(np.int64)
    assert off[-1] == pairs.shape[0]
    rng = np.random.default_rng(11)
    check_lists = set(rng.choice(256, size=6, replace=False).tolist())
    for wd in range(256):
        a, b = int(t.obj_base[wd]), int(t.obj_base[wd + 1])
        qa, qb = int(t.q_base[wd]), int(t.q_base[wd + 1])
        if qb == qa:
            continue
        st = oracle.State(max(b - a, 1))
        if b > a:
            st.apply_updates(np.arange(b - a, dtype=np.uint32), t.xy[a:b])
        want = oracle.count_grid(st, t.rects[qa:qb], cell_side=0.004).astype(np.int64)
        np.testing.assert_array_equal(np.diff(off[qa:qb + 1]), want, err_msg="world %d" % wd)
        if wd in check_lists:
            sample = np.sort(rng.choice(qb - qa, size=min(40, qb - qa), replace=False))
            s_off, s_ids = oracle.join_grid(st, t.rects[qa:qb][sample], cell_side=0.004)
            for k, q in enumerate(sample):
                seg = pairs[int(off[qa + q]):int(off[qa + q + 1])].cpu().numpy().view(np.uint32)
                assert np.all(seg[:, 0] == qa + q)
                np.testing.assert_array_equal(np.sort(seg[:, 1]) - np.uint32(a),
                                              s_ids[int(s_off[k]):int(s_off[k + 1])])
    idx.close()


def test_served_10m_full_size_admission():
    """The served workload's state at full size (10M objects, 95% in 16
    hotspots): one tick's batch (Poisson arrivals at 5e6/s over 10 ms) with
    covering-compressed output and admission by an output budget of half the
    batch's output: the admitted prefix is the longest that fits, and its
    per-query counts, and those of the whole batch as pairs, equal the
    oracle's."""
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    world = workloads.ServedWorld(rate=5.0e6, dt=0.010, seed=0)
    t = world.next_tick()
    Q = t.rects.shape[0]
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=128, max_objects=world.n)
    idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
    st = oracle.State(world.n)
    st.apply_updates(t.ids, t.xy)
    rects_d = to_dev(t.rects, dev)
    want_cnt = _check_counts_and_sample(idx, st, t.rects, rects_d, 0.002, np.random.default_rng(5), 300, dev,
                                        "served pairs")
    _, full_offs = idx.tick(rects_d, kind="runs")              # the whole batch's element offsets
    full = full_offs.cpu().numpy().view(np.uint64).astype(np.int64)
    budget = int(full[-1]) // 2 * 8                              # room for about half of the output
    out = torch.empty(budget // 4, dtype=torch.int32, device=dev)
    offs = torch.empty(Q + 1, dtype=torch.int64, device=dev)
    adm, cnt = mqr.mqr_tick_admit(idx.ctx, rects_d, Q, mqr.MQR_OUT_RUNS, out, budget, offs)
    assert 0 < adm < Q and cnt * 8 <= budget
    assert cnt == full[adm] and full[adm + 1] * 8 > budget      # the longest prefix that fits
    e = out[: cnt * 2].cpu().numpy().view(np.uint32).reshape(-1, 2)
    eoff = offs[: adm + 1].cpu().numpy().view(np.uint64).astype(np.int64)
    assert eoff[adm] == cnt
    run = (e[:, 0] & 0x80000000) != 0
    heads = np.nonzero(run)[0]
    counts = np.ones(e.shape[0], np.int64)
    counts[heads] = e[heads + 1, 0]
    counts[heads + 1] = 0
    csum = np.concatenate([[0], np.cumsum(counts)])
    np.testing.assert_array_equal(csum[eoff[1:]] - csum[eoff[:-1]], want_cnt[:adm])
    idx.close()


def test_hotspot_4m_per_region_capacities_full_size():
    """The per-region thresholds the cost-model chooser settles on at
    hotspot-4M (regions of depth 3, capacity 2^(8 + 0.25 log2 density)): every
    query's count against the oracle, sampled lists, and the leaf table's
    capacity rule checked on the GPU's own leaves."""
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    from paper_1411_3212_gb300.costmodel import region_caps
    w = workloads.HotspotWalk(n=4_000_000, q=400_000, seed=0)
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=128, max_objects=w.n)
    st = oracle.State(w.n)
    rng = np.random.default_rng(9)
    t = w.next_tick()
    idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
    st.apply_updates(t.ids, t.xy)
    idx.tick(to_dev(t.rects, dev), kind="count")
    caps = region_caps(idx.region_counts(3), 3, 8, 0.25)
    idx.set_region_caps(3, caps)
    t = w.next_tick()
    idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
    st.apply_updates(t.ids, t.xy)
    _check_counts_and_sample(idx, st, t.rects, to_dev(t.rects, dev), 0.002, rng, 500, dev, "per-region caps")
    # capacity rule on the leaves: a leaf above l_max holds at most its region's capacity
    lv = idx.leaves().astype(np.int64)
    region = (lv[:, 1] << (2 * (15 - lv[:, 0]))) >> (2 * (15 - 3))
    size = lv[:, 3] - lv[:, 2]
    assert np.all((size <= caps[region]) | (lv[:, 0] == 15))
    assert lv[:, 0].min() >= 3
    idx.close()
