"""Join slots (mqr_snapshot, mqr_slot_*): batches answered concurrently on
their own streams against one snapshot of the object state.  Every batch's
result in the overlapped mix must equal the oracle's Def. 1 result for the
snapshot's positions and the same batch answered alone by a plain tick, for
every output kind the slots support, with admission cuts, across ticks; the
served stream on slots must answer every query exactly once."""
import numpy as np
import pytest

import oracle
from paper_1411_3212_gb300 import workloads
from tests.gpu_util import expand_runs, oracle_state, to_dev, torch_dev

pytestmark = pytest.mark.gpu


def decode(mqr, kind, out, cnt, offs, admitted, sid):
    """A slot's output -> (per-query counts, sorted ids per query) of its
    admitted queries."""
    off = offs[: admitted + 1].astype(np.int64)
    if kind == mqr.MQR_OUT_CSR:
        ids = out[:cnt].view(np.uint32).copy()
        for q in range(admitted):
            ids[off[q]:off[q + 1]] = np.sort(ids[off[q]:off[q + 1]])
        return np.diff(off), ids
    e = out[: 2 * cnt].view(np.uint32).reshape(-1, 2)
    if kind == mqr.MQR_OUT_RUNS:
        pairs, _ = expand_runs(e, sid)
    else:
        pairs = e
    assert np.all(np.diff(pairs[:, 0].astype(np.int64)) >= 0)
    order = np.lexsort((pairs[:, 1], pairs[:, 0]))
    pairs = pairs[order]
    counts = np.bincount(pairs[:, 0].astype(np.int64), minlength=admitted)[:admitted]
    return counts, pairs[:, 1].copy()


def test_slots_overlap_and_match_alone_and_oracle():
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    n = 60_000
    w = workloads.HotspotWalk(n=n, q=6000, hotspots=6, side_lo=0.001, side_hi=0.03, seed=33)
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=32, max_objects=n)
    slots = [idx.slot() for _ in range(3)]
    kinds = [mqr.MQR_OUT_PAIRS, mqr.MQR_OUT_CSR, mqr.MQR_OUT_RUNS]
    # before any snapshot a slot cannot answer
    with pytest.raises(mqr.MqrError, match="snapshot"):
        slots[0].begin(to_dev(np.zeros((1, 4), np.float32), dev), "pairs",
                       torch.empty(16, dtype=torch.int32, device=dev), 64)
    rng = np.random.default_rng(4)
    for tick in range(3):
        t = w.next_tick()
        idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
        idx.snapshot()
        st = oracle_state(n, [(t.ids, t.xy)])
        Q = t.rects.shape[0]
        cuts = np.sort(rng.choice(np.arange(1, Q), size=2, replace=False))
        parts = [t.rects[:cuts[0]], t.rects[cuts[0]:cuts[1]], t.rects[cuts[1]:]]
        want = [oracle.join_grid(st, r, cell_side=0.01) for r in parts]
        outs, offs, caps, elems = [], [], [], []
        for i, r in enumerate(parts):
            R = int(want[i][0][-1])
            # the third tick cuts slot 1's output at about half of its results (admission)
            cap_elems = R // 2 + 1 if (tick == 2 and i == 1) else R + 64
            if kinds[i] == mqr.MQR_OUT_RUNS:
                cap_elems = 2 * R + 64
            outs.append(torch.full((2 * cap_elems + 16,), -1, dtype=torch.int32, device=dev))
            offs.append(torch.zeros(r.shape[0] + 1, dtype=torch.int64, device=dev))
            caps.append(cap_elems * (4 if kinds[i] == mqr.MQR_OUT_CSR else 8))
            elems.append(cap_elems)
        rect_d = [to_dev(r, dev) for r in parts]
        for i in range(3):              # all three joins in flight at once
            slots[i].begin(rect_d[i], kinds[i], outs[i], caps[i], offs[i])
        # while they run: another snapshot or a plain tick is refused, updates are accepted
        with pytest.raises(mqr.MqrError, match="pending"):
            idx.snapshot()
        with pytest.raises(mqr.MqrError, match="pending"):
            idx.tick(rect_d[0], kind="pairs")
        res = [slots[i].end() for i in range(3)]
        _, sid = idx.sorted_objects()
        for i in range(3):
            adm, cnt = res[i]
            wo, wi = want[i]
            wo = wo.astype(np.int64)
            if tick == 2 and i == 1:
                assert 0 < adm < parts[i].shape[0]           # a prefix was admitted
                assert wo[adm] <= elems[i] < wo[adm + 1]      # the longest prefix that fits
            else:
                assert adm == parts[i].shape[0]
            counts, ids = decode(mqr, kinds[i], outs[i].cpu().numpy(), cnt,
                                 offs[i].cpu().numpy().view(np.uint64), adm, sid)
            np.testing.assert_array_equal(counts, np.diff(wo)[:adm])
            np.testing.assert_array_equal(ids, wi[: wo[adm]])
            # the same batch alone, through a plain tick of the same state
            if adm == parts[i].shape[0]:
                alone, aoff = idx.tick(rect_d[i], kind="csr_sorted")
                np.testing.assert_array_equal(aoff.cpu().numpy().view(np.uint64)[: adm + 1].astype(np.int64),
                                              wo[: adm + 1])
                np.testing.assert_array_equal(alone.cpu().numpy().view(np.uint32), ids)
            s = slots[i].stats()
            assert s["n_queries"] == parts[i].shape[0]
    for sl in slots:
        sl.close()
    idx.close()


def test_served_stream_on_slots_answers_every_query_once():
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    from paper_1411_3212_gb300.serve import SlotBackend, TickServer

    n, dt, n_ticks = 50_000, 0.004, 6
    world = workloads.ServedWorld(n=n, rate=3.0e5, dt=dt, side_lo=0.002, side_hi=0.02, seed=8)
    ticks = [world.next_tick() for _ in range(n_ticks)]
    arrivals = np.concatenate([k * dt + t.arrivals for k, t in enumerate(ticks)])
    rects = np.concatenate([t.rects for t in ticks])
    pos = [t.xy for t in ticks]
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=64, max_objects=n)
    ids_d = to_dev(ticks[0].ids, dev)
    updates = [(ids_d, to_dev(p, dev)) for p in pos]
    rects_d = to_dev(rects, dev)
    answered = []            # (tick, lo, admitted, pairs relative to lo)

    class Checked(SlotBackend):
        def begin_tick(self, k):
            self.k = k
            super().begin_tick(k)

        def answer(self, lo, hi):
            adm, cnt, ev = super().answer(lo, hi)
            ev.synchronize()
            _, sid = mqr.mqr_get_sorted(self.idx.ctx)
            for a, padm, pcnt, i in self.last_parts:
                e = self.host[i][: pcnt * 2].numpy().view(np.uint32).reshape(-1, 2).copy()
                pairs, _ = expand_runs(e, sid)
                answered.append((self.k, a, padm, pairs))
            return adm, cnt, ev

    be = Checked(idx, updates, rects_d, kind="runs", budget_bytes=3 * 128 * 1024, n_slots=3)
    rep = TickServer(be, dt).run(arrivals, n_ticks=n_ticks, drain_ticks=200)
    be.close()
    assert rep["answered"] == rects.shape[0] and rep["rejected"] == []
    assert rep["deferred_batches"] > 0
    got = np.zeros(rects.shape[0], np.int64)
    for k, lo, adm, pairs in answered:
        got[lo:lo + adm] += 1
        st = oracle.State(n)
        st.apply_updates(ticks[0].ids, pos[k % len(pos)])
        woff, wids = oracle.join_grid(st, rects[lo:lo + adm], cell_side=0.01)
        qrel = pairs[:, 0].astype(np.int64)
        cnt = np.bincount(qrel, minlength=adm)
        np.testing.assert_array_equal(cnt, np.diff(woff.astype(np.int64)))
        order = np.lexsort((pairs[:, 1], qrel))
        np.testing.assert_array_equal(pairs[order, 1], wids)
    np.testing.assert_array_equal(got, 1)
    idx.close()


def test_slot_edge_cases_and_updates_during_a_join():
    """Q = 0 on a slot; end without begin and a second begin are refused;
    updates applied while a join runs belong to the next snapshot (the
    running join answers the snapshot's positions); a slot of a destroyed
    context refuses to answer."""
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    n = 20_000
    rng = np.random.default_rng(9)
    xy0 = rng.random((n, 2)).astype(np.float32)
    xy1 = rng.random((n, 2)).astype(np.float32)
    ids = np.arange(n, dtype=np.uint32)
    rects = workloads.squares_around(xy0[rng.integers(0, n, 500)], 0.03)
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=32, max_objects=n)
    sl = idx.slot()
    idx.apply_updates(to_dev(ids, dev), to_dev(xy0, dev))
    idx.snapshot()
    out = torch.empty(1 << 22, dtype=torch.int32, device=dev)
    with pytest.raises(mqr.MqrError, match="no join pending"):
        sl.end()
    sl.begin(to_dev(np.zeros((0, 4), np.float32), dev), "pairs", out, out.numel() * 4)
    assert sl.end() == (0, 0)
    offs = torch.zeros(rects.shape[0] + 1, dtype=torch.int64, device=dev)
    sl.begin(to_dev(rects, dev), "pairs", out, out.numel() * 4, offs)
    with pytest.raises(mqr.MqrError, match="pending"):
        sl.begin(to_dev(rects, dev), "pairs", out, out.numel() * 4)
    idx.apply_updates(to_dev(ids, dev), to_dev(xy1, dev))        # the next snapshot's positions
    adm, cnt = sl.end()
    want = oracle.join_grid(oracle_state(n, [(ids, xy0)]), rects, cell_side=0.03)
    assert adm == rects.shape[0] and cnt == int(want[0][-1])
    counts, got = decode(mqr, mqr.MQR_OUT_PAIRS, out.cpu().numpy(), cnt, offs.cpu().numpy().view(np.uint64), adm,
                         None)
    np.testing.assert_array_equal(got, want[1])
    # the updates show in the next snapshot
    idx.snapshot()
    sl.begin(to_dev(rects, dev), "pairs", out, out.numel() * 4, offs)
    adm, cnt = sl.end()
    want1 = oracle.join_grid(oracle_state(n, [(ids, xy1)]), rects, cell_side=0.03)
    counts, got = decode(mqr, mqr.MQR_OUT_PAIRS, out.cpu().numpy(), cnt, offs.cpu().numpy().view(np.uint64), adm,
                         None)
    np.testing.assert_array_equal(got, want1[1])
    idx.close()
    with pytest.raises(mqr.MqrError, match="destroyed"):
        sl.begin(to_dev(rects, dev), "pairs", out, out.numel() * 4)
    sl.close()


def test_graph_cache_alternating_outputs_and_eviction():
    """Graph mode keeps a few captured ticks: ticks alternating between five
    output buffers (more than it keeps, so captures are evicted and made
    again) all answer exactly."""
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    n = 20_000
    w = workloads.HotspotWalk(n=n, q=1200, hotspots=4, side_lo=0.002, side_hi=0.03, seed=41)
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=32, max_objects=n)
    idx.set_graph(True)
    outs = [torch.empty(1 << 21, dtype=torch.int32, device=dev) for _ in range(5)]
    offs = torch.zeros(1201, dtype=torch.int64, device=dev)
    st = oracle.State(n)
    for k in range(12):
        t = w.next_tick() if k % 3 == 0 else t
        if k % 3 == 0:
            idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
            st.apply_updates(t.ids, t.xy)
            want = oracle.join_grid(st, t.rects, cell_side=0.01)
        out = outs[(k * 2) % 5]
        status, cnt = mqr.mqr_tick(idx.ctx, to_dev(t.rects, dev), t.rects.shape[0], mqr.MQR_OUT_PAIRS, out,
                                   out.numel() * 4, offs)
        assert status == mqr.MQR_OK and cnt == int(want[0][-1])
        np.testing.assert_array_equal(offs.cpu().numpy().view(np.uint64), want[0])
        p = out[: 2 * cnt].cpu().numpy().view(np.uint32).reshape(-1, 2)
        order = np.lexsort((p[:, 1], p[:, 0]))
        np.testing.assert_array_equal(p[order, 1], want[1])
    idx.set_graph(False)
    idx.close()
