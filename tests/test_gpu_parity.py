"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bit-exact: every comparison is on integer ids, keys and leaf records; the
containment test is an exact FP32 comparison on both sides (Def. 1).
"""
import numpy as np
import pytest

import oracle
from paper_1411_3212_gb300 import workloads
from tests.gpu_util import (assert_same_csr, gpu_atomic_as_csr, gpu_csr_sorted, gpu_pairs_as_csr, gpu_runs_as_csr, oracle_state,
                            to_dev, torch_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mqr():
    torch, dev = torch_dev()
    if not torch.cuda.is_available():
        pytest.fail("CUDA is not available")
    from paper_1411_3212_gb300 import mqr as m
    m.load()
    return m


def make_index(mqr, nmax, cap=64, **kw):
    return mqr.Index(bounds=kw.pop("bounds", (0.0, 0.0, 1.0, 1.0)), leaf_cap=cap, max_objects=nmax, **kw)


# ---------------------------------------------------------------------------
# 16K uniform objects, 1,024 queries of side 0.01, leaf_cap 64: bitmap +
# sorted per-query lists, bit-exact.
# ---------------------------------------------------------------------------
def test_uniform_16k_bitmap_and_sorted_lists(mqr):
    torch, dev = torch_dev()
    t = workloads.uniform_small(seed=0)
    n = t.ids.shape[0]
    idx = make_index(mqr, n, cap=64)
    idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
    st = oracle_state(n, [(t.ids, t.xy)])
    want = oracle.join_grid(st, t.rects, cell_side=0.01)

    assert_same_csr(gpu_csr_sorted(idx, t.rects, dev), want, "csr_sorted")
    assert_same_csr(gpu_pairs_as_csr(idx, t.rects, dev), want, "pairs")
    bm, offs = idx.tick(to_dev(t.rects, dev), kind="bitmap")
    np.testing.assert_array_equal(bm.cpu().numpy().view(np.uint32), oracle.bitmap(*want, n))
    np.testing.assert_array_equal(offs.cpu().numpy().view(np.uint64), want[0])
    s = idx.stats()
    assert s["n_results"] == want[1].shape[0]
    assert s["n_objects"] == n
    # self-inclusion (Def. 1 remark)
    for q, issuer in enumerate(t.issuers):
        assert issuer in want[1][int(want[0][q]):int(want[0][q + 1])]
    idx.close()


# ---------------------------------------------------------------------------
# Morton keys + radix sort (Alg. 1 GPUcalculateMortonHash / GPUradixSort) and
# the leaf table (Alg. 1), exact against the oracle.
# ---------------------------------------------------------------------------
# (65_499 and 65_500 objects + 37 absent slots: 16 and 17 sort tiles of 4,096,
# the largest sort run with look-back passes and the smallest without)
@pytest.mark.parametrize("n,cap,seed", [(16384, 64, 0), (50_001, 128, 1), (5000, 1, 2), (70_000, 2, 3),
                                        (3000, 5000, 4), (120_000, 20_000, 5), (65_499, 128, 6),
                                        (65_500, 128, 7)])
def test_sorted_keys_and_leaves(mqr, n, cap, seed):
    torch, dev = torch_dev()
    w = workloads.HotspotWalk(n=n, q=10, hotspots=8, seed=seed)
    t = w.next_tick()
    xy = t.xy.copy()
    xy[: n // 50] = xy[0]                        # a pile of identical points (level-15 leaf)
    nmax = n + 37                                # ragged: 37 slots never updated (absent)
    idx = make_index(mqr, nmax, cap=cap)
    idx.apply_updates(to_dev(t.ids, dev), to_dev(xy, dev))
    idx.tick(to_dev(t.rects, dev), kind="count")
    keys, ids = idx.sorted_objects()

    st = oracle_state(nmax, [(t.ids, xy)])
    ok = oracle.keys(st)
    order = np.argsort(ok, kind="stable")[:n]
    np.testing.assert_array_equal(keys, ok[order])
    np.testing.assert_array_equal(ids, order.astype(np.uint32))

    lv = idx.leaves()
    want = oracle.quadtree(ok[order], cap, 15)
    want = want[want["begin"] != want["end"]]
    got = np.stack([want["level"], want["z"], want["begin"], want["end"]], 1)
    np.testing.assert_array_equal(lv, got)
    s = idx.stats()
    assert s["n_leaves"] == len(want) and s["max_level"] == int(want["level"].max())
    idx.close()


# ---------------------------------------------------------------------------
# Query splitting counts (Def. "Mapping functions"): intersecting subqueries
# and covering leaves equal the oracle's g(q) over the non-empty leaves.
# ---------------------------------------------------------------------------
def test_subquery_counts_match_oracle(mqr):
    torch, dev = torch_dev()
    w = workloads.HotspotWalk(n=20000, q=300, hotspots=4, side_lo=0.001, side_hi=0.2, seed=9)
    t = w.next_tick()
    idx = make_index(mqr, 20000, cap=32)
    idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
    idx.tick(to_dev(t.rects, dev), kind="count")
    s = idx.stats()
    st = oracle_state(20000, [(t.ids, t.xy)])
    ok = oracle.keys(st)
    lv = oracle.quadtree(np.sort(ok), 32, 15)
    n_i = n_c = tests = 0
    for r in t.rects:
        li, cov = oracle.subqueries(lv, r)
        n_c += int(cov.sum())
        n_i += int(len(cov) - cov.sum())
        tests += int(sum(lv["end"][k] - lv["begin"][k] for k, c in zip(li, cov) if not c))
    assert s["n_sub_intersecting"] == n_i
    assert s["n_sub_covering"] == n_c
    assert s["n_tests"] == tests
    assert s["n_covering_runs"] <= n_c
    idx.close()


# ---------------------------------------------------------------------------
# Index independence: every leaf capacity, the uniform grid at several
# resolutions, covering on/off -> identical results.
# ---------------------------------------------------------------------------
CFGS = [dict(cap=1), dict(cap=2), dict(cap=64), dict(cap=128), dict(cap=512), dict(cap=20000),
        dict(cap=2 ** 31 - 1), dict(cap=128, covering=False),
        dict(cap=1, index_kind=1, grid_level=3), dict(cap=1, index_kind=1, grid_level=7),
        dict(cap=1, index_kind=1, grid_level=10)]


@pytest.fixture(scope="module")
def hotspot_case():
    w = workloads.HotspotWalk(n=60000, q=3000, hotspots=8, side_lo=0.0005, side_hi=0.05, seed=3)
    t = w.next_tick()
    st = oracle_state(60000, [(t.ids, t.xy)])
    return t, oracle.join_grid(st, t.rects, cell_side=0.005)


@pytest.mark.parametrize("cfg", CFGS, ids=[str(c) for c in CFGS])
def test_index_independence(mqr, hotspot_case, cfg):
    torch, dev = torch_dev()
    t, want = hotspot_case
    cfg = dict(cfg)
    cap = cfg.pop("cap")
    idx = make_index(mqr, 60000, cap=cap, **cfg)
    idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
    assert_same_csr(gpu_csr_sorted(idx, t.rects, dev), want, str(cfg))
    assert_same_csr(gpu_pairs_as_csr(idx, t.rects, dev), want, str(cfg))
    go, gi, e = gpu_runs_as_csr(idx, t.rects, dev)
    assert_same_csr((go, gi), want, "runs " + str(cfg))
    s = idx.stats()
    assert e.shape[0] == s["n_results"] - s["n_results_covering"] + 2 * s["n_covering_runs"]
    assert_same_csr(gpu_atomic_as_csr(idx, t.rects, dev), want, "atomic " + str(cfg))
    idx.close()


# ---------------------------------------------------------------------------
# Adversarial inputs: coordinates on query edges, duplicates, NaN/inf/-0,
# out-of-bounds points, absent objects, inverted / NaN / infinite queries,
# ragged sizes.
# ---------------------------------------------------------------------------
def adversarial(seed, n, q):
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 2)).astype(np.float32)
    lat = (np.round(rng.random((n, 2)) * 64) / 64).astype(np.float32)
    snap = rng.random(n) < 0.5
    pos[snap] = lat[snap]
    k = max(1, n // 16)
    pos[rng.integers(0, n, k)] = pos[rng.integers(0, n, k)]
    pos[rng.integers(0, n, k)] = rng.uniform(-0.5, 1.5, (k, 2)).astype(np.float32)
    specials = np.array([np.nan, np.inf, -np.inf, -0.0, 0.0, 1.0], np.float32)
    for _ in range(k):
        pos[rng.integers(0, n), rng.integers(0, 2)] = specials[rng.integers(0, len(specials))]
    present_ids = np.nonzero(rng.random(n) < 0.9)[0].astype(np.uint32)
    c = np.nan_to_num(pos[rng.integers(0, n, q)], nan=0.5, posinf=1.0, neginf=0.0)
    rects = workloads.squares_around(c, rng.choice([0.0, 1 / 64, 0.05, 0.2, 0.7], q))
    lq = (np.round(rng.random((q, 4)) * 64) / 64).astype(np.float32)
    pick = rng.random(q) < 0.5
    rects[pick] = np.sort(lq[pick].reshape(-1, 2, 2), axis=1).reshape(-1, 4)[:, [0, 2, 1, 3]]
    flip = rng.random(q) < 0.05
    rects[flip] = rects[flip][:, [2, 3, 0, 1]]
    rects[rng.integers(0, q, max(1, q // 32)), rng.integers(0, 4)] = np.nan
    rects[rng.integers(0, q, max(1, q // 32))] = [-np.inf, -np.inf, np.inf, np.inf]
    return present_ids, pos[present_ids], rects


@pytest.mark.parametrize("seed,n,q,cap", [(0, 1000, 200, 4), (1, 4097, 1025, 16), (2, 33_333, 2049, 64),
                                          (3, 100_003, 3001, 128)])
def test_adversarial(mqr, seed, n, q, cap):
    torch, dev = torch_dev()
    ids, xy, rects = adversarial(seed, n, q)
    idx = make_index(mqr, n, cap=cap)
    idx.apply_updates(to_dev(ids, dev), to_dev(xy, dev))
    st = oracle_state(n, [(ids, xy)])
    want = oracle.join_grid(st, rects, cell_side=0.01)
    assert_same_csr(gpu_csr_sorted(idx, rects, dev), want)
    assert_same_csr(gpu_pairs_as_csr(idx, rects, dev), want)
    go, gi, _ = gpu_runs_as_csr(idx, rects, dev)
    assert_same_csr((go, gi), want, "runs")
    assert_same_csr(gpu_atomic_as_csr(idx, rects, dev), want, "atomic")
    idx.close()


def test_last_update_wins_across_and_within_calls(mqr):
    torch, dev = torch_dev()
    rng = np.random.default_rng(5)
    nmax = 3000
    idx = make_index(mqr, nmax, cap=8)
    ups = []
    for _ in range(4):
        ids = rng.integers(0, nmax - 100, 2500).astype(np.uint32)      # duplicates inside a call
        xy = rng.random((2500, 2)).astype(np.float32)
        idx.apply_updates(to_dev(ids, dev), to_dev(xy, dev))
        ups.append((ids, xy))
    rects = workloads.squares_around(rng.random((400, 2)), 0.08)
    st = oracle_state(nmax, ups)
    want = oracle.join_grid(st, rects, cell_side=0.02)
    assert_same_csr(gpu_csr_sorted(idx, rects, dev), want)
    assert idx.stats()["n_objects"] == int(st.present.sum())
    idx.close()


def test_empty_and_degenerate(mqr):
    torch, dev = torch_dev()
    idx = make_index(mqr, 1000, cap=4)
    rects = np.array([[0, 0, 1, 1], [0.5, 0.5, 0.4, 0.6]], np.float32)
    off, ids = gpu_csr_sorted(idx, rects, dev)          # no object ever updated
    assert list(off) == [0, 0, 0] and ids.shape[0] == 0
    off, ids = gpu_csr_sorted(idx, np.zeros((0, 4), np.float32), dev)   # Q = 0
    assert list(off) == [0] and ids.shape[0] == 0
    # all objects at one point: a level-15 leaf far above the capacity
    xy = np.full((1000, 2), 0.25, np.float32)
    idx.apply_updates(to_dev(np.arange(1000, dtype=np.uint32), dev), to_dev(xy, dev))
    rects = np.array([[0.25, 0.25, 0.25, 0.25], [0, 0, 0.2, 0.2], [0.2, 0.2, 0.3, 0.3]], np.float32)
    off, ids = gpu_csr_sorted(idx, rects, dev)
    assert list(off) == [0, 1000, 1000, 2000]
    np.testing.assert_array_equal(ids[:1000], np.arange(1000))
    idx.close()


def test_uniform_walk_multi_tick(mqr):
    """1M uniform objects random-walking, 100K queries of side 0.002 per tick,
    leaf_cap 128, pair-list output; three ticks, full comparison."""
    torch, dev = torch_dev()
    w = workloads.UniformWalk(n=1_000_000, q=100_000, seed=0)
    idx = make_index(mqr, 1_000_000, cap=128)
    st = oracle.State(1_000_000)
    for _ in range(3):
        t = w.next_tick()
        idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
        st.apply_updates(t.ids, t.xy)
        want = oracle.join_grid(st, t.rects, cell_side=0.002)
        assert_same_csr(gpu_pairs_as_csr(idx, t.rects, dev), want)
    idx.close()


def test_overfull_leaf_of_identical_points(mqr):
    """120,000 objects on one point (a level-15 leaf of 120K objects: 469 filter
    chunks, multi-chunk counts, thousands of bitmap words per subquery) beside
    80,000 uniform ones; queries that cover the point, touch it on their
    boundary, and miss it; every output kind against the oracle."""
    torch, dev = torch_dev()
    rng = np.random.default_rng(17)
    n = 200_000
    xy = rng.random((n, 2)).astype(np.float32)
    xy[:120_000] = np.float32(0.3125)                  # exactly representable
    ids = rng.permutation(n).astype(np.uint32)          # the cluster's ids are scattered
    c = rng.random((300, 2)).astype(np.float32)
    rects = workloads.squares_around(c, rng.choice([0.001, 0.01, 0.1], 300))
    rects[:40] = workloads.squares_around(np.full((40, 2), 0.3125, np.float32), rng.choice([0.0, 0.001, 0.2], 40))
    rects[40:50] = [[0.3125, 0.3125, 0.5, 0.5]] * 10    # the point on the lower-left corner
    rects[50:60] = [[0.1, 0.1, 0.3125, 0.3125]] * 10    # ... and on the upper-right corner
    rects[60:70] = [[0.1, 0.1, 0.3124, 0.3124]] * 10    # just missing it
    idx = make_index(mqr, n, cap=64)
    idx.apply_updates(to_dev(ids, dev), to_dev(xy, dev))
    st = oracle_state(n, [(ids, xy)])
    want = oracle.join_grid(st, rects, cell_side=0.01)
    assert int(np.diff(want[0].astype(np.int64))[:60].min()) >= 120_000
    assert_same_csr(gpu_csr_sorted(idx, rects, dev), want)
    assert_same_csr(gpu_pairs_as_csr(idx, rects, dev), want)
    go, gi, _ = gpu_runs_as_csr(idx, rects, dev)
    assert_same_csr((go, gi), want, "runs")
    assert_same_csr(gpu_atomic_as_csr(idx, rects, dev), want, "atomic")
    lv = idx.leaves()
    assert (lv[:, 3] - lv[:, 2]).max() >= 120_000 and lv[:, 0].max() == 15
    idx.close()
