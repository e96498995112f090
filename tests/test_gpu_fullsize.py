"""Full-size parity: the 4M-object hotspot workload with 400,000 queries per
tick, in the launch configuration bench.py times (leaf_cap 128, quadtree,
pair-list output).  Every query's result count is compared with the oracle's,
and the complete id lists of a random sample of queries are compared exactly;
the covering-compressed output of the same ticks must give the same counts.
"""
import numpy as np
import pytest

import oracle
from paper_1411_3212_gb300 import workloads
from tests.gpu_util import to_dev, torch_dev

pytestmark = pytest.mark.gpu


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
