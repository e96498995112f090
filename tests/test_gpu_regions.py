"""Per-region split thresholds (Alg. 1's th_quad chosen per region of a fixed
quadtree level): the leaf table must be the oracle's Alg. 1 with the same
thresholds, exactly, and every output kind must stay the oracle's result
(Def. 1), whatever the thresholds; switching them between ticks, with the
captured-graph replay on, with batched worlds and with the uniform grid."""
import numpy as np
import pytest

import oracle
from paper_1411_3212_gb300 import workloads
from tests.gpu_util import (assert_same_csr, gpu_csr_sorted, gpu_pairs_as_csr, gpu_runs_as_csr, oracle_state,
                            to_dev, torch_dev)

pytestmark = pytest.mark.gpu


def random_caps(rng, region_bits):
    """Log-uniform thresholds in 1..16384, with the extremes present."""
    caps = np.exp2(rng.uniform(0, 14, 4 ** region_bits)).astype(np.uint32).clip(1, 16384)
    caps[rng.integers(0, caps.size)] = 1
    caps[rng.integers(0, caps.size)] = 16384
    return caps


def check_leaves(idx, st, n, region_bits, caps):
    ok = oracle.keys(st)
    order = np.argsort(ok, kind="stable")[:n]
    keys, ids = idx.sorted_objects()
    np.testing.assert_array_equal(keys, ok[order])
    want = oracle.quadtree(ok[order], 0, 15, region_bits=region_bits, region_caps=caps)
    want = want[want["begin"] != want["end"]]
    got = idx.leaves()
    np.testing.assert_array_equal(got, np.stack([want["level"], want["z"], want["begin"], want["end"]], 1))
    s = idx.stats()
    assert s["n_leaves"] == len(want) and s["max_level"] == int(want["level"].max())


@pytest.mark.parametrize("region_bits,n,seed", [(1, 70_000, 0), (2, 50_001, 1), (3, 120_000, 2), (4, 90_017, 3),
                                                (4, 3000, 4)])
def test_region_caps_leaves_and_results(region_bits, n, seed):
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    rng = np.random.default_rng(seed)
    w = workloads.HotspotWalk(n=n, q=1500, hotspots=6, side_lo=0.0005, side_hi=0.05, seed=seed)
    t = w.next_tick()
    xy = t.xy.copy()
    xy[: n // 40] = xy[0]                       # a pile of identical points (a level-15 leaf)
    nmax = n + 29                               # ragged: slots never updated
    caps = random_caps(rng, region_bits)
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=64, max_objects=nmax)
    idx.set_region_caps(region_bits, caps)
    idx.apply_updates(to_dev(t.ids, dev), to_dev(xy, dev))
    st = oracle_state(nmax, [(t.ids, xy)])
    want = oracle.join_grid(st, t.rects, cell_side=0.005)
    assert_same_csr(gpu_csr_sorted(idx, t.rects, dev), want, "csr_sorted")
    check_leaves(idx, st, n, region_bits, caps)
    assert idx.leaves()[:, 0].min() >= region_bits
    assert_same_csr(gpu_pairs_as_csr(idx, t.rects, dev), want, "pairs")
    go, gi, _ = gpu_runs_as_csr(idx, t.rects, dev)
    assert_same_csr((go, gi), want, "runs")
    idx.close()


def test_region_caps_switching_with_graph_replay():
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    rng = np.random.default_rng(7)
    n = 60_000
    w = workloads.HotspotWalk(n=n, q=2000, hotspots=5, side_lo=0.001, side_hi=0.03, seed=7)
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=128, max_objects=n)
    idx.set_graph(True)
    st = oracle.State(n)
    settings = [(2, random_caps(rng, 2)), (0, None), (3, random_caps(rng, 3)), (3, random_caps(rng, 3)),
                (1, np.array([1, 16384, 40, 7], np.uint32))]
    for k, (rb, caps) in enumerate(settings):
        t = w.next_tick()
        st.apply_updates(t.ids, t.xy)
        idx.set_region_caps(rb, caps)
        idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
        for rep in range(2):                    # the second tick replays the captured graph
            assert_same_csr(gpu_csr_sorted(idx, t.rects, dev), oracle.join_grid(st, t.rects, cell_side=0.005),
                            "setting %d rep %d" % (k, rep))
        if rb:
            check_leaves(idx, st, n, rb, caps)
        else:
            lv = oracle.quadtree(np.sort(oracle.keys(st)), 128, 15)
            assert idx.stats()["n_leaves"] == int((lv["begin"] != lv["end"]).sum())
    idx.close()


@pytest.mark.parametrize("region_bits", [1, 3])
def test_region_caps_with_batched_worlds(region_bits):
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    from tests.test_gpu_worlds import world_oracle
    rng = np.random.default_rng(region_bits)
    bw = workloads.BatchedWorlds(n_worlds=5, n_lo=50, n_hi=6000, q_frac=0.2, side=0.02, seed=11)
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=32, max_objects=bw.n)
    idx.set_worlds(bw.obj_base)
    idx.set_region_caps(region_bits, random_caps(rng, region_bits))
    t = bw.next_tick()
    idx.set_query_worlds(t.q_base)
    idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
    off, ids = gpu_csr_sorted(idx, t.rects, dev)
    for wd in range(5):
        qa, qb = int(t.q_base[wd]), int(t.q_base[wd + 1])
        got = (off[qa:qb + 1] - off[qa], ids[int(off[qa]):int(off[qb])])
        assert_same_csr(got, world_oracle(t, wd), "world %d" % wd)
    lv = idx.leaves()
    assert lv[:, 0].min() >= max(2, region_bits)          # 5 worlds: 2 levels above their roots
    _, sid = idx.sorted_objects()
    world_of_id = np.searchsorted(t.obj_base, sid, side="right") - 1
    for lvl, z, b, e in lv:
        assert world_of_id[b] == world_of_id[e - 1], (lvl, z)
    idx.close()


def test_region_caps_arguments_and_uniform_grid():
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    rng = np.random.default_rng(5)
    n = 20_000
    xy = rng.random((n, 2)).astype(np.float32)
    rects = workloads.squares_around(rng.random((500, 2)).astype(np.float32), 0.02)
    st = oracle_state(n, [(np.arange(n, dtype=np.uint32), xy)])
    want = oracle.join_grid(st, rects, cell_side=0.01)
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=16, max_objects=n)
    idx.apply_updates(to_dev(np.arange(n, dtype=np.uint32), dev), to_dev(xy, dev))
    with pytest.raises(mqr.MqrError):
        idx.set_region_caps(5, np.ones(4 ** 5, np.uint32))           # more than 4 levels
    with pytest.raises(mqr.MqrError):
        idx.set_region_caps(1, np.array([1, 0, 3, 4], np.uint32))    # a zero threshold
    with pytest.raises(mqr.MqrError):
        idx.set_region_caps(1, np.array([1, 16385, 3, 4], np.uint32))
    with pytest.raises(ValueError):
        idx.set_region_caps(2, np.ones(4, np.uint32))                # wrong length
    # a failed call leaves the single threshold in force
    assert_same_csr(gpu_csr_sorted(idx, rects, dev), want, "after errors")
    lv = oracle.quadtree(np.sort(oracle.keys(st)), 16, 15)
    assert idx.stats()["n_leaves"] == int((lv["begin"] != lv["end"]).sum())
    # the uniform grid ignores region thresholds
    idx.set_region_caps(2, np.full(16, 3, np.uint32))
    idx.set_index(1, grid_level=7)
    assert_same_csr(gpu_csr_sorted(idx, rects, dev), want, "grid")
    assert np.all(idx.leaves()[:, 0] == 7)
    idx.set_index(0, leaf_cap=16)
    assert_same_csr(gpu_csr_sorted(idx, rects, dev), want, "regions")
    check_leaves(idx, st, n, 2, np.full(16, 3, np.uint32))
    idx.close()


@pytest.mark.parametrize("region_bits", [1, 2, 3, 4])
def test_region_counts_match_sorted_keys(region_bits):
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    n = 40_000
    w = workloads.HotspotWalk(n=n, q=100, hotspots=3, seed=region_bits)
    t = w.next_tick()
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=32, max_objects=n + 5)
    with pytest.raises(mqr.MqrError):
        idx.region_counts(region_bits)                                # no tick yet
    idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
    idx.tick(to_dev(t.rects, dev), kind="count")
    st = oracle_state(n + 5, [(t.ids, t.xy)])
    k = oracle.keys(st)
    k = k[k != 0xFFFFFFFF]
    want = np.bincount(k >> (2 * (15 - region_bits)), minlength=4 ** region_bits)
    np.testing.assert_array_equal(idx.region_counts(region_bits), want)
    with pytest.raises(mqr.MqrError):
        idx.region_counts(0)
    with pytest.raises(mqr.MqrError):
        idx.region_counts(5)
    idx.close()


def test_chooser_applies_region_candidates_exactly():
    """A per-region candidate of the cost-model chooser configures the
    thresholds from the previous tick's densities; results stay the
    oracle's and the leaves are Alg. 1 with those thresholds."""
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    from paper_1411_3212_gb300.costmodel import QUAD, REGIONS, IndexChooser, region_caps
    n = 80_000
    w = workloads.HotspotWalk(n=n, q=2000, hotspots=6, side_lo=0.001, side_hi=0.03, seed=13)
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=128, max_objects=n)
    ch = IndexChooser(candidates=[(QUAD, 128), (REGIONS, 3, 7, 0.5)], seed=1)
    st = oracle.State(n)
    for k, cand in enumerate([(REGIONS, 3, 7, 0.5), (REGIONS, 3, 7, 0.5), (QUAD, 128), (REGIONS, 2, 6, -0.25)]):
        t = w.next_tick()
        st.apply_updates(t.ids, t.xy)
        caps = region_caps(idx.region_counts(cand[1]), cand[1], cand[2], cand[3]) \
            if cand[0] == REGIONS and k > 0 else None
        ch.apply(idx, cand)
        idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
        assert_same_csr(gpu_csr_sorted(idx, t.rects, dev), oracle.join_grid(st, t.rects, cell_side=0.005),
                        str(cand))
        if caps is not None:
            check_leaves(idx, st, n, cand[1], caps)
    ch.close()
    idx.close()


def oracle_region_work(st, rects, cap, region_bits):
    """The per-region statistics of mqr_region_work from the oracle: Alg. 1
    leaves, g(q) subqueries (Def. mapping functions), Def. 1 results."""
    R = 4 ** region_bits
    keys_slot = oracle.keys(st)
    order = np.argsort(keys_slot, kind="stable")
    n = int(st.present.sum())
    order = order[:n]
    keys = keys_slot[order]
    lv = oracle.quadtree(keys, cap, 15)
    lv = lv[lv["begin"] != lv["end"]]
    reg = (lv["z"].astype(np.int64) << (2 * (15 - lv["level"].astype(np.int64)))) >> (2 * (15 - region_bits))
    size = (lv["end"] - lv["begin"]).astype(np.int64)
    out = {k: np.zeros(R) for k in ("objects", "leaves", "queries", "side_log2_sum", "sub_intersecting",
                                    "sub_covering", "tests", "results_intersecting", "results_covering")}
    np.add.at(out["objects"], reg, size)
    np.add.at(out["leaves"], reg, 1)
    pos = st.pos[order]
    sc = oracle.scale(0.0, 1.0)
    for r in rects:
        li, cov = oracle.subqueries(lv, r)
        for l, c in zip(li, cov):
            g = reg[l]
            if c:
                out["sub_covering"][g] += 1
                out["results_covering"][g] += size[l]
            else:
                p = pos[lv["begin"][l]:lv["end"][l]]
                hit = (p[:, 0] >= r[0]) & (p[:, 0] <= r[2]) & (p[:, 1] >= r[1]) & (p[:, 1] <= r[3])
                out["sub_intersecting"][g] += 1
                out["tests"][g] += size[l]
                out["results_intersecting"][g] += int(hit.sum())
        if not (r[0] <= r[2] and r[1] <= r[3]) or not np.all(np.isfinite(r)):
            continue
        cx = np.float32(np.float32(0.5) * r[0] + np.float32(0.5) * r[2])
        cy = np.float32(np.float32(0.5) * r[1] + np.float32(0.5) * r[3])
        z = oracle.morton(oracle.cell(float(cx), 0.0, sc), oracle.cell(float(cy), 0.0, sc))
        g = z >> (2 * (15 - region_bits))
        out["queries"][g] += 1
        out["side_log2_sum"][g] += np.log2(max(float(max(r[2] - r[0], r[3] - r[1])), 1e-9))
    return out


@pytest.mark.parametrize("region_bits,cap", [(1, 16), (2, 32), (4, 8)])
def test_region_work_matches_oracle(region_bits, cap):
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    n = 20_000
    w = workloads.HotspotWalk(n=n, q=400, hotspots=4, side_lo=0.002, side_hi=0.08, seed=region_bits)
    t = w.next_tick()
    rects = t.rects.copy()
    rects[3] = [0.7, 0.7, 0.2, 0.9]                     # inverted: no subqueries, not counted
    rects[5, 1] = np.nan
    nmax = n + 11
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=cap, max_objects=nmax)
    idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
    r_d = to_dev(rects, dev)
    idx.tick(r_d, kind="pairs")
    got = idx.region_work(r_d, region_bits)
    st = oracle_state(nmax, [(t.ids, t.xy)])
    want = oracle_region_work(st, rects, cap, region_bits)
    for k in want:
        if k == "side_log2_sum":
            np.testing.assert_allclose(got[k], want[k], rtol=1e-5, atol=1e-3, err_msg=k)
        else:
            np.testing.assert_array_equal(got[k], want[k], err_msg=k)
    s = idx.stats()
    assert got["tests"].sum() == s["n_tests"] and got["results_covering"].sum() == s["n_results_covering"]
    with pytest.raises(mqr.MqrError):
        mqr.mqr_region_work(idx.ctx, r_d, 399, region_bits)          # not the last tick's Q
    idx.tick(r_d, kind="pairs_atomic")
    with pytest.raises(mqr.MqrError):
        idx.region_work(r_d, region_bits)                            # no per-subquery counts
    idx.close()


def test_region_chooser_on_real_ticks_stays_exact():
    """The node-level chooser logs each tick's region work and phase times,
    sets per-region capacities for the next tick, and every tick's result
    stays the oracle's; the leaves are Alg. 1 with the capacities chosen."""
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    from paper_1411_3212_gb300.costmodel import RegionChooser
    n = 60_000
    w = workloads.HotspotWalk(n=n, q=3000, hotspots=6, side_lo=0.001, side_hi=0.03, seed=17)
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=128, max_objects=n)
    ch = RegionChooser(region_bits=2, caps=(16, 64, 256, 1024), explore_rounds=1, retrain_every=1, epochs=100)
    st = oracle.State(n)
    for k in range(6):
        t = w.next_tick()
        st.apply_updates(t.ids, t.xy)
        ch.apply(idx)
        caps = ch.current.copy()
        idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
        r_d = to_dev(t.rects, dev)
        res, offs = idx.tick(r_d, kind="csr_sorted")
        got = (offs.cpu().numpy().view(np.uint64), res.cpu().numpy().view(np.uint32).copy())
        assert_same_csr(got, oracle.join_grid(st, t.rects, cell_side=0.005), "tick %d" % k)
        ch.record(idx, r_d)
        check_leaves(idx, st, n, 2, caps)
    assert ch.trained and len(ch.X) > 0
    cost = ch.region_costs(ch.last_work)
    assert cost.shape == (16,) and np.all(cost >= 0) and cost.sum() > 0
    ch.close()
    idx.close()
