"""Served stream on the GPU: Poisson arrivals batched into ticks, admission by
output memory (small budget, so batches are split across ticks), results
copied out on a second stream.  Every query must be answered exactly once,
with the oracle's result set for the positions of the tick that answered it,
and a query answered alone (mqr_tick) must give the same set as in the mix."""
import numpy as np
import pytest

import oracle
from paper_1411_3212_gb300 import workloads
from tests.gpu_util import expand_runs, to_dev, torch_dev

pytestmark = pytest.mark.gpu


def test_served_stream_admission_and_isolation():
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    from paper_1411_3212_gb300.serve import GpuBackend, TickServer

    n, dt, n_ticks = 50_000, 0.004, 6
    world = workloads.ServedWorld(n=n, rate=3.0e5, dt=dt, side_lo=0.002, side_hi=0.02, seed=5)
    ticks = [world.next_tick() for _ in range(n_ticks)]
    arrivals = np.concatenate([k * dt + t.arrivals for k, t in enumerate(ticks)])
    rects = np.concatenate([t.rects for t in ticks])
    pos = [t.xy for t in ticks]
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=64, max_objects=n)
    ids_d = to_dev(ticks[0].ids, dev)
    updates = [(ids_d, to_dev(p, dev)) for p in pos]
    rects_d = to_dev(rects, dev)

    answered = []            # (tick, lo, admitted, pairs, per-query counts)

    class Checked(GpuBackend):
        def begin_tick(self, k):
            self.k = k
            super().begin_tick(k)

        def answer(self, lo, hi):
            adm, cnt, ev = super().answer(lo, hi)
            ev.synchronize()
            e = self.host[(self.n_answers - 1) & 1][: cnt * 2].numpy().view(np.uint32).reshape(-1, 2).copy()
            _, sid = mqr.mqr_get_sorted(self.idx.ctx)
            pairs, _ = expand_runs(e, sid)
            answered.append((self.k, lo, adm, pairs))
            # the same queries alone, against the same state
            for q in sorted({lo, lo + adm // 2, lo + max(adm - 1, 0)}):
                if adm == 0:
                    break
                one, offs = self.idx.tick(self.rects[q:q + 1], kind="csr_sorted")
                mine = np.sort(pairs[pairs[:, 0] == q - lo, 1])
                np.testing.assert_array_equal(one.cpu().numpy().view(np.uint32), mine)
            return adm, cnt, ev

    budget = 256 * 1024         # bytes: forces several batches to be split
    be = Checked(idx, updates, rects_d, kind="runs", budget_bytes=budget)
    rep = TickServer(be, dt).run(arrivals, n_ticks=n_ticks, drain_ticks=200)
    assert rep["answered"] == rects.shape[0] and rep["rejected"] == []
    assert rep["deferred_batches"] > 0
    # every query answered once, with the oracle's set at the answering tick's positions
    got = np.zeros(rects.shape[0], np.int64)
    for k, lo, adm, pairs in answered:
        got[lo:lo + adm] += 1
        st = oracle.State(n)
        st.apply_updates(ticks[0].ids, pos[k % len(pos)])
        woff, wids = oracle.join_grid(st, rects[lo:lo + adm], cell_side=0.01)
        qrel = pairs[:, 0].astype(np.int64)
        assert np.all(np.diff(qrel) >= 0)
        cnt = np.bincount(qrel, minlength=adm)
        np.testing.assert_array_equal(cnt, np.diff(woff.astype(np.int64)))
        order = np.lexsort((pairs[:, 1], qrel))
        np.testing.assert_array_equal(pairs[order, 1], wids)
    np.testing.assert_array_equal(got, 1)
    lat = rep["query_latency_ms"]
    assert lat["p50"] > 0 and lat["max"] >= lat["p99"] >= lat["p50"]
    idx.close()
