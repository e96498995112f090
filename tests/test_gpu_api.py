"""C-ABI behaviour on the GPU: output kinds, host-buffer entry points,
capacity and id errors, timing counters."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1411_3212_gb300 import workloads
from tests.gpu_util import (assert_same_csr, expand_runs, gpu_csr_sorted, gpu_pairs_as_csr, oracle_state,  # noqa: F401
                            to_dev, torch_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    w = workloads.HotspotWalk(n=30000, q=2000, hotspots=6, side_lo=0.001, side_hi=0.03, seed=21)
    t = w.next_tick()
    st = oracle_state(30000, [(t.ids, t.xy)])
    return t, oracle.join_grid(st, t.rects, cell_side=0.005)


def mk(n, cap=32):
    from paper_1411_3212_gb300 import mqr
    return mqr, mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=cap, max_objects=n)


def test_pairs_sorted_kind(case):
    torch, dev = torch_dev()
    t, (woff, wids) = case
    mqr, idx = mk(30000)
    idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
    res, offs = idx.tick(to_dev(t.rects, dev), kind="pairs_sorted")
    p = res.cpu().numpy().view(np.uint32)
    want_q = np.repeat(np.arange(t.rects.shape[0], dtype=np.uint32), np.diff(woff.astype(np.int64)))
    np.testing.assert_array_equal(p[:, 0], want_q)
    np.testing.assert_array_equal(p[:, 1], wids)
    np.testing.assert_array_equal(offs.cpu().numpy().view(np.uint64), woff)
    idx.close()


def test_csr_unsorted_kind_is_a_permutation_per_query(case):
    torch, dev = torch_dev()
    t, (woff, wids) = case
    mqr, idx = mk(30000)
    idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
    res, offs = idx.tick(to_dev(t.rects, dev), kind="csr")
    ids = res.cpu().numpy().view(np.uint32)
    off = offs.cpu().numpy().view(np.uint64)
    np.testing.assert_array_equal(off, woff)
    for q in range(t.rects.shape[0]):
        a, b = int(off[q]), int(off[q + 1])
        np.testing.assert_array_equal(np.sort(ids[a:b]), wids[a:b])
    idx.close()


def test_host_entry_points(case):
    torch, dev = torch_dev()
    t, want = case
    from paper_1411_3212_gb300 import mqr
    ctx = mqr.mqr_create((0.0, 0.0, 1.0, 1.0), 32, 30000)
    try:
        mqr.mqr_apply_updates_host(ctx, np.ascontiguousarray(t.ids), np.ascontiguousarray(t.xy))
        Q = t.rects.shape[0]
        offs = np.zeros(Q + 1, np.uint64)
        out = np.zeros(16, np.uint32)                    # far too small: CAPACITY with the size needed
        st, cnt = mqr.mqr_tick_host(ctx, np.ascontiguousarray(t.rects), Q, mqr.MQR_OUT_CSR_SORTED, out,
                                    out.nbytes, offs)
        assert st == mqr.MQR_ERR_CAPACITY and cnt == want[1].shape[0]
        out = np.zeros(cnt, np.uint32)
        st, cnt = mqr.mqr_tick_host(ctx, np.ascontiguousarray(t.rects), Q, mqr.MQR_OUT_CSR_SORTED, out,
                                    out.nbytes, offs)
        assert st == mqr.MQR_OK
        assert_same_csr((offs, out), want)
        bm = np.zeros((Q, (30000 + 31) // 32), np.uint32)
        st, cnt = mqr.mqr_tick_host(ctx, np.ascontiguousarray(t.rects), Q, mqr.MQR_OUT_BITMAP, bm, bm.nbytes)
        assert st == mqr.MQR_OK
        np.testing.assert_array_equal(bm, oracle.bitmap(*want, 30000))
    finally:
        mqr.mqr_destroy(ctx)


def test_runs_kind_through_host_entry_point(case):
    """Covering-compressed output through mqr_tick_host: every result exactly
    once, as a pair or inside a covering run of the tick's sorted ids."""
    torch, dev = torch_dev()
    t, want = case
    from paper_1411_3212_gb300 import mqr
    ctx = mqr.mqr_create((0.0, 0.0, 1.0, 1.0), 32, 30000)
    try:
        mqr.mqr_apply_updates_host(ctx, np.ascontiguousarray(t.ids), np.ascontiguousarray(t.xy))
        Q = t.rects.shape[0]
        offs = np.zeros(Q + 1, np.uint64)
        out = np.zeros((want[1].shape[0] + 16, 2), np.uint32)
        st, cnt = mqr.mqr_tick_host(ctx, np.ascontiguousarray(t.rects), Q, mqr.MQR_OUT_RUNS, out, out.nbytes,
                                    offs)
        assert st == mqr.MQR_OK and offs[-1] == cnt
        s = mqr.mqr_get_stats(ctx)
        assert s["n_covering_runs"] > 0
        assert cnt == s["n_results"] - s["n_results_covering"] + 2 * s["n_covering_runs"]
        _, sid = mqr.mqr_get_sorted(ctx)
        pairs, counts = expand_runs(out[:cnt], sid)
        per_q = np.array([counts[int(offs[q]):int(offs[q + 1])].sum() for q in range(Q)], np.int64)
        off = np.concatenate([[0], np.cumsum(per_q)]).astype(np.uint64)
        ids = pairs[:, 1].copy()
        for q in range(Q):
            ids[int(off[q]):int(off[q + 1])] = np.sort(ids[int(off[q]):int(off[q + 1])])
        assert_same_csr((off, ids), want)
    finally:
        mqr.mqr_destroy(ctx)


def test_atomic_baseline_capacity_then_retry(case):
    """The unordered atomic-append kind: a too-small buffer gives CAPACITY with
    the exact count (nothing past the buffer is written), then the full set."""
    torch, dev = torch_dev()
    t, (woff, wids) = case
    from paper_1411_3212_gb300 import mqr
    mqr_, idx = mk(30000)
    idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
    Q = t.rects.shape[0]
    rd = to_dev(t.rects, dev)
    guard = torch.full((4096,), -7, dtype=torch.int32, device=dev)
    small = guard[:1024]
    st, cnt = mqr.mqr_tick(idx.ctx, rd, Q, mqr.MQR_OUT_PAIRS_ATOMIC, small, small.numel() * 4)
    assert st == mqr.MQR_ERR_CAPACITY and cnt == wids.shape[0]
    assert bool((guard[1024:] == -7).all().item())
    with pytest.raises(mqr.MqrError, match="offsets"):
        mqr.mqr_tick(idx.ctx, rd, Q, mqr.MQR_OUT_PAIRS_ATOMIC, small, small.numel() * 4,
                     torch.empty(Q + 1, dtype=torch.int64, device=dev))
    big = torch.empty(2 * cnt + 16, dtype=torch.int32, device=dev)
    st, cnt2 = mqr.mqr_tick(idx.ctx, rd, Q, mqr.MQR_OUT_PAIRS_ATOMIC, big, big.numel() * 4)
    assert st == mqr.MQR_OK and cnt2 == cnt
    p = big[: 2 * cnt].cpu().numpy().view(np.uint32).reshape(-1, 2)
    p = p[np.lexsort((p[:, 1], p[:, 0]))]
    want_q = np.repeat(np.arange(Q, dtype=np.uint32), np.diff(woff.astype(np.int64)))
    np.testing.assert_array_equal(p[:, 0], want_q)
    np.testing.assert_array_equal(p[:, 1], wids)
    idx.close()


def test_device_capacity_error_then_retry(case):
    torch, dev = torch_dev()
    t, want = case
    from paper_1411_3212_gb300 import mqr
    mqr_, idx = mk(30000)
    idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
    Q = t.rects.shape[0]
    rd = to_dev(t.rects, dev)
    small = torch.empty(64, dtype=torch.int32, device=dev)
    st, cnt = mqr.mqr_tick(idx.ctx, rd, Q, mqr.MQR_OUT_PAIRS, small, small.numel() * 4)
    assert st == mqr.MQR_ERR_CAPACITY and cnt == want[1].shape[0]
    big = torch.empty(2 * cnt, dtype=torch.int32, device=dev)
    st, cnt2 = mqr.mqr_tick(idx.ctx, rd, Q, mqr.MQR_OUT_PAIRS, big, big.numel() * 4)
    assert st == mqr.MQR_OK and cnt2 == cnt
    idx.close()


def test_bad_update_id_is_reported_and_ignored():
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    mqr_, idx = mk(100, cap=4)
    ids = np.array([0, 1, 100, 2], np.uint32)             # 100 >= max_objects
    xy = np.array([[0.1, 0.1], [0.2, 0.2], [0.3, 0.3], [0.4, 0.4]], np.float32)
    idx.apply_updates(to_dev(ids, dev), to_dev(xy, dev))
    with pytest.raises(mqr.MqrError, match="max_objects"):
        idx.tick(to_dev(np.array([[0, 0, 1, 1]], np.float32), dev), kind="csr_sorted")
    # the error is reported once; the valid updates were applied
    res, offs = idx.tick(to_dev(np.array([[0, 0, 1, 1]], np.float32), dev), kind="csr_sorted")
    np.testing.assert_array_equal(res.cpu().numpy(), [0, 1, 2])
    idx.close()


def test_misaligned_output_rejected(case):
    torch, dev = torch_dev()
    t, want = case
    from paper_1411_3212_gb300 import mqr
    mqr_, idx = mk(30000)
    idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
    buf = torch.empty(1 << 20, dtype=torch.int32, device=dev)
    with pytest.raises(mqr.MqrError, match="aligned"):
        mqr.mqr_tick(idx.ctx, to_dev(t.rects, dev), t.rects.shape[0], mqr.MQR_OUT_PAIRS,
                     buf.data_ptr() + 4, buf.numel() * 4 - 4)
    idx.close()


def test_timing_counters(case):
    torch, dev = torch_dev()
    t, want = case
    mqr, idx = mk(30000)
    idx.set_timing(True)
    for _ in range(2):
        idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
        idx.tick(to_dev(t.rects, dev), kind="pairs")
    tm = idx.timing()
    assert tm["ticks"] >= 2
    for ph in ["updates", "keys", "sort", "leaves", "query_blocks", "candidates", "group", "filter",
               "result_scan", "emit"]:
        assert tm["launches"][ph] > 0 and tm["ms"][ph] > 0.0, ph
    idx.close()


def test_timing_of_selected_phases(case):
    """Timing only the emit phase: its device time is measured, the other
    phases get no events, and every phase's launches are still counted (the
    same counts as with all phases timed)."""
    torch, dev = torch_dev()
    t, want = case
    mqr, idx = mk(30000)
    idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
    idx.tick(to_dev(t.rects, dev), kind="pairs")          # buffers grown: no retries below
    counts = []
    for phases in (None, ["emit"]):
        idx.set_timing(True, phases=phases)
        for _ in range(2):
            idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
            idx.tick(to_dev(t.rects, dev), kind="pairs")
        tm = idx.timing()
        counts.append(tm["launches"])
    assert tm["ms"]["emit"] > 0.0
    for ph in ["updates", "keys", "sort", "leaves", "query_blocks", "candidates", "group", "filter", "result_scan"]:
        assert tm["ms"][ph] == 0.0, ph
    assert counts[0] == counts[1]
    idx.set_timing(False)
    idx.close()


def test_uniform_grid_subquery_counts_match_oracle(case):
    """The uniform-grid variant (every leaf at grid_level) splits queries
    exactly as g(q) over the grid's non-empty cells."""
    torch, dev = torch_dev()
    t, want = case
    from paper_1411_3212_gb300 import mqr
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=1, max_objects=30000, index_kind=1, grid_level=7)
    idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
    idx.tick(to_dev(t.rects, dev), kind="count")
    s = idx.stats()
    lv = idx.leaves()
    assert np.all(lv[:, 0] == 7)
    dt = np.dtype([("level", np.uint32), ("z", np.uint32), ("begin", np.uint32), ("end", np.uint32)])
    table = np.zeros(len(lv), dt)
    table["level"], table["z"], table["begin"], table["end"] = lv[:, 0], lv[:, 1], lv[:, 2], lv[:, 3]
    n_i = n_c = 0
    for r in t.rects[:500]:
        li, cov = oracle.subqueries(table, r)
        n_c += int(cov.sum())
        n_i += int(len(cov) - cov.sum())
    idx.tick(to_dev(t.rects[:500], dev), kind="count")
    s = idx.stats()
    assert s["n_sub_intersecting"] == n_i and s["n_sub_covering"] == n_c
    idx.close()


def test_leaf_cap_autotune_picks_a_capacity_with_identical_results(case):
    torch, dev = torch_dev()
    t, want = case
    from paper_1411_3212_gb300 import mqr
    from paper_1411_3212_gb300.autotune import tune_leaf_cap
    ticks = [(to_dev(t.ids, dev), to_dev(t.xy, dev), to_dev(t.rects, dev))]
    best, table = tune_leaf_cap(lambda cap: mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=cap, max_objects=30000),
                                ticks, caps=(8, 32, 128), reps=2)
    assert best in (8, 32, 128) and set(table) == {8, 32, 128}
    assert {v["results"] for v in table.values()} == {int(want[1].shape[0])}
    assert all(v["ms_per_tick"] > 0 for v in table.values())


def test_launch_config_changes_time_not_results(case):
    """Blocks per SM of the work-item kernels (down to one block per SM and up
    to 32): every shape gives the oracle's result; out-of-range values are
    rejected; the autotuner picks a shape among its options."""
    torch, dev = torch_dev()
    t, want = case
    from paper_1411_3212_gb300.autotune import tune_launch_config
    mqr, idx = mk(30000)
    idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
    for cfg in [dict(candidate=1, compact=1, filter=1, emit=1), dict(candidate=16, compact=2, filter=4, emit=32),
                dict()]:
        idx.set_launch_config(**cfg)
        assert_same_csr(gpu_csr_sorted(idx, t.rects, dev), want, str(cfg))
        assert_same_csr(gpu_pairs_as_csr(idx, t.rects, dev), want, str(cfg))
    with pytest.raises(mqr.MqrError):
        idx.set_launch_config(filter=65)
    ticks = [(to_dev(t.ids, dev), to_dev(t.xy, dev), to_dev(t.rects, dev))]
    best, table = tune_launch_config(idx, ticks, options=(2, 8), reps=1)
    assert set(best) == {"candidate", "compact", "filter", "emit"} and set(best.values()) <= {2, 8}
    assert len(table) == 8 and len({r for _, _, r in table}) == 1
    assert_same_csr(gpu_csr_sorted(idx, t.rects, dev), want, "tuned")
    idx.close()


def test_graph_mode_replays_identical_results():
    """Graph mode: the first tick of a shape is captured (including the
    buffer growth of a fresh context), later ticks replay it; a new Q or
    output buffer captures again; every tick equals the oracle and the plain
    launches bit for bit."""
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    w = workloads.HotspotWalk(n=20000, q=1500, hotspots=4, side_lo=0.002, side_hi=0.04, seed=31)
    ticks = [w.next_tick() for _ in range(4)]
    g = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=32, max_objects=20000)
    plain = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=32, max_objects=20000)
    g.set_graph(True)
    st = oracle.State(20000)
    for k, t in enumerate(ticks):
        rects = t.rects if k < 3 else t.rects[:700]            # the last tick has a new Q
        rd = to_dev(rects, dev)
        for idx in (g, plain):
            idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
        st.apply_updates(t.ids, t.xy)
        res_g, off_g = g.tick(rd, kind="pairs")
        a = (res_g.cpu().numpy().copy(), off_g.cpu().numpy().copy())
        res_p, off_p = plain.tick(rd, kind="pairs")
        np.testing.assert_array_equal(a[0], res_p.cpu().numpy())
        np.testing.assert_array_equal(a[1], off_p.cpu().numpy())
        woff, wids = oracle.join_grid(st, rects, cell_side=0.01)
        np.testing.assert_array_equal(a[1].view(np.uint64), woff)
        assert a[0].shape[0] == wids.shape[0]
    g.set_graph(False)
    g.close()
    plain.close()


def test_phase_timing_under_graph_replay():
    """Graph mode with phase timing: the timed phase's events are event nodes
    of the captured graph, so every replayed tick adds its time and launch
    counts (the same counts as plain launches), and the results stay those
    of the plain launches and the oracle."""
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    w = workloads.HotspotWalk(n=20000, q=1500, hotspots=4, side_lo=0.002, side_hi=0.04, seed=32)
    ticks = [w.next_tick() for _ in range(5)]
    g = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=32, max_objects=20000)
    plain = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=32, max_objects=20000)
    g.set_graph(True)
    for idx in (g, plain):
        idx.set_timing(True, phases=["emit"])
    st = oracle.State(20000)
    for k, t in enumerate(ticks):
        rd = to_dev(t.rects, dev)
        st.apply_updates(t.ids, t.xy)
        outs = []
        for idx in (g, plain):
            idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
            res, off = idx.tick(rd, kind="pairs")
            outs.append((res.cpu().numpy().copy(), off.cpu().numpy().copy()))
        np.testing.assert_array_equal(outs[0][0], outs[1][0])
        np.testing.assert_array_equal(outs[0][1], outs[1][1])
        woff, _ = oracle.join_grid(st, t.rects, cell_side=0.01)
        np.testing.assert_array_equal(outs[0][1].view(np.uint64), woff)
    tg, tp = g.timing(), plain.timing()
    assert tg["ticks"] == tp["ticks"] >= len(ticks)       # (an output buffer that grew answers a tick again)
    assert tg["launches"] == tp["launches"]
    assert tg["launches"]["emit"] >= len(ticks)
    assert tg["ms"]["emit"] > 0.0 and tg["ms"]["filter"] == 0.0     # only the timed phase has events
    g.set_graph(False)
    g.close()
    plain.close()


def test_async_host_ticks_overlap_and_match_the_oracle():
    """mqr_tick_host_async: four ticks in a row, each copying into its own
    page-locked host buffer while the next runs; after mqr_host_wait every
    buffer holds its tick's results (offsets and sorted lists = oracle)."""
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    w = workloads.HotspotWalk(n=30000, q=2000, hotspots=6, side_lo=0.001, side_hi=0.03, seed=44)
    ticks = [w.next_tick() for _ in range(4)]
    ctx = mqr.mqr_create((0.0, 0.0, 1.0, 1.0), 32, 30000)
    st = oracle.State(30000)
    wants, outs, offs, cnts = [], [], [], []
    try:
        for t in ticks:
            st.apply_updates(t.ids, t.xy)
            wants.append(oracle.join_grid(st, t.rects, cell_side=0.005))
            out = torch.zeros(2 * (wants[-1][1].shape[0] + 64), dtype=torch.int32).pin_memory()
            off = torch.zeros(t.rects.shape[0] + 1, dtype=torch.int64).pin_memory()
            mqr.mqr_apply_updates_host(ctx, np.ascontiguousarray(t.ids), np.ascontiguousarray(t.xy))
            s, cnt = mqr.mqr_tick_host_async(ctx, np.ascontiguousarray(t.rects), t.rects.shape[0], mqr.MQR_OUT_PAIRS,
                                             out.numpy(), out.numel() * 4, off.numpy())
            assert s == mqr.MQR_OK and cnt == wants[-1][1].shape[0]
            outs.append(out)
            offs.append(off)
            cnts.append(cnt)
        mqr.mqr_host_wait(ctx)
        for (woff, wids), out, off, cnt, t in zip(wants, outs, offs, cnts, ticks):
            p = out.numpy().view(np.uint32)[: 2 * cnt].reshape(-1, 2)
            o = off.numpy().view(np.uint64)
            np.testing.assert_array_equal(o, woff)
            ids = p[:, 1].copy()
            for q in range(t.rects.shape[0]):
                ids[int(o[q]):int(o[q + 1])] = np.sort(ids[int(o[q]):int(o[q + 1])])
            np.testing.assert_array_equal(ids, wids)
    finally:
        mqr.mqr_destroy(ctx)


def test_async_runs_with_async_sorted_ids():
    """RUNS output through mqr_tick_host_async + mqr_get_sorted_async on three
    ticks in a row: each tick's runs expand, with that tick's sorted ids, to
    the oracle's sets."""
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    w = workloads.HotspotWalk(n=30000, q=1500, hotspots=6, side_lo=0.002, side_hi=0.04, seed=45)
    ticks = [w.next_tick() for _ in range(3)]
    ctx = mqr.mqr_create((0.0, 0.0, 1.0, 1.0), 32, 30000)
    st = oracle.State(30000)
    keep = []
    try:
        for t in ticks:
            st.apply_updates(t.ids, t.xy)
            want = oracle.join_grid(st, t.rects, cell_side=0.005)
            out = torch.zeros(2 * (want[1].shape[0] + 64), dtype=torch.int32).pin_memory()
            off = torch.zeros(t.rects.shape[0] + 1, dtype=torch.int64).pin_memory()
            sid = torch.zeros(30000, dtype=torch.int32).pin_memory()
            mqr.mqr_apply_updates_host(ctx, np.ascontiguousarray(t.ids), np.ascontiguousarray(t.xy))
            s, cnt = mqr.mqr_tick_host_async(ctx, np.ascontiguousarray(t.rects), t.rects.shape[0], mqr.MQR_OUT_RUNS,
                                             out.numpy(), out.numel() * 4, off.numpy())
            assert s == mqr.MQR_OK
            assert mqr.mqr_get_sorted_async(ctx, sid.numpy().view(np.uint32)) == 30000
            keep.append((want, out, off, sid, cnt, t.rects.shape[0]))
        mqr.mqr_host_wait(ctx)
        for (woff, wids), out, off, sid, cnt, Q in keep:
            e = out.numpy().view(np.uint32)[: 2 * cnt].reshape(-1, 2)
            pairs, counts = expand_runs(e, sid.numpy().view(np.uint32))
            eo = off.numpy().view(np.uint64).astype(np.int64)
            per_q = np.array([counts[eo[q]:eo[q + 1]].sum() for q in range(Q)], np.int64)
            o = np.concatenate([[0], np.cumsum(per_q)]).astype(np.uint64)
            ids = pairs[:, 1].copy()
            for q in range(Q):
                ids[int(o[q]):int(o[q + 1])] = np.sort(ids[int(o[q]):int(o[q + 1])])
            assert_same_csr((o, ids), (woff, wids))
    finally:
        mqr.mqr_destroy(ctx)


def test_result_footprint_against_the_oracle(case):
    """mqr_result_footprint: the leaves holding at least one result object and
    the leaves with at least one intersecting subquery, with their objects,
    from the oracle's Alg. 1 leaves, g(q) and Def. 1 result sets."""
    torch, dev = torch_dev()
    t, want = case
    from paper_1411_3212_gb300 import mqr
    cap = 32
    mqr_, idx = mk(30000, cap)
    idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
    idx.tick(to_dev(t.rects, dev), kind="pairs")
    fp = idx.footprint()
    st = oracle_state(30000, [(t.ids, t.xy)])
    k = oracle.keys(st)
    order = np.argsort(k, kind="stable")
    leaves = oracle.quadtree(k[order], cap)
    pos = np.empty(30000, np.int64)
    pos[order] = np.arange(30000)
    size = (leaves["end"] - leaves["begin"]).astype(np.int64)
    res_leaf = np.zeros(len(leaves), bool)
    hit = np.searchsorted(leaves["begin"], pos[want[1]], side="right") - 1
    res_leaf[hit] = True
    tested = np.zeros(len(leaves), bool)
    for q in range(t.rects.shape[0]):
        lv, cov = oracle.subqueries(leaves, t.rects[q])
        tested[lv[cov == 0]] = True
    assert fp == {"result_leaves": int(res_leaf.sum()), "result_leaf_objects": int(size[res_leaf].sum()),
                  "tested_leaves": int(tested.sum()), "tested_leaf_objects": int(size[tested].sum())}
    idx.close()


def test_misaligned_update_arrays_rejected(case):
    torch, dev = torch_dev()
    t, want = case
    from paper_1411_3212_gb300 import mqr
    mqr_, idx = mk(30000)
    ids = to_dev(t.ids, dev)
    xy = torch.zeros(2 * 30000 + 2, dtype=torch.float32, device=dev)
    with pytest.raises(mqr.MqrError, match="aligned"):
        mqr.mqr_apply_updates(idx.ctx, ids, xy.data_ptr() + 4, 30000)
    with pytest.raises(mqr.MqrError, match="aligned"):
        mqr.mqr_apply_updates(idx.ctx, ids.data_ptr() + 2, xy, 30000)
    idx.close()
