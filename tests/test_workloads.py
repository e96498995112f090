"""The synthetic input recipes (no GPU): determinism by seed, every query
containing the object that issued it (self-inclusion, Def. 1), values in
the unit square, and the structure each recipe states."""
import numpy as np
import pytest

from paper_1411_3212_gb300 import workloads


def issued_inside(t):
    xy = t.xy[t.issuers]
    r = t.rects
    return np.all((r[:, 0] <= xy[:, 0]) & (xy[:, 0] <= r[:, 2]) & (r[:, 1] <= xy[:, 1]) & (xy[:, 1] <= r[:, 3]))


@pytest.mark.parametrize("make", [
    lambda s: workloads.UniformWalk(n=5000, q=500, seed=s),
    lambda s: workloads.HotspotWalk(n=5000, q=500, hotspots=6, seed=s),
    lambda s: workloads.MixedDensity(n=5000, q_small=400, q_large=40, seed=s),
    lambda s: workloads.ServedWorld(n=5000, rate=2e5, dt=0.01, seed=s),
])
def test_walks_are_seeded_self_including_and_in_bounds(make):
    a, b, c = make(3), make(3), make(4)
    for _ in range(3):
        ta, tb, tc = a.next_tick(), b.next_tick(), c.next_tick()
        np.testing.assert_array_equal(ta.xy, tb.xy)
        np.testing.assert_array_equal(ta.rects, tb.rects)
        assert not np.array_equal(ta.xy, tc.xy)
        assert ta.xy.dtype == np.float32 and ta.rects.dtype == np.float32
        assert np.all((ta.xy >= 0) & (ta.xy < 1))
        assert issued_inside(ta)


def test_mixed_density_halves_and_query_sides():
    w = workloads.MixedDensity(n=20_000, q_small=2000, q_large=200, seed=1)
    for _ in range(4):
        t = w.next_tick()
    nd = w.n_dense
    assert nd == 15_000
    assert t.xy[:nd, 0].max() < 0.5 and t.xy[nd:, 0].min() >= 0.5           # each population in its half
    side = np.maximum(t.rects[:, 2] - t.rects[:, 0], t.rects[:, 3] - t.rects[:, 1])
    small, large = side[:2000], side[2000:]
    assert small.max() <= 0.001 * 1.001 and large.min() >= 0.01 * 0.999
    assert np.all(t.issuers[:2000] < nd) and np.all(t.issuers[2000:] >= nd)


def test_served_world_arrivals_are_sorted_inside_the_tick():
    w = workloads.ServedWorld(n=5000, rate=1e6, dt=0.01, seed=2)
    t = w.next_tick()
    assert t.arrivals.shape[0] == t.rects.shape[0]
    assert np.all(np.diff(t.arrivals) >= 0) and t.arrivals.min() >= 0 and t.arrivals.max() < 0.01
    assert abs(t.rects.shape[0] - 10_000) < 500                              # Poisson(rate x dt)


def test_batched_worlds_ranges():
    bw = workloads.BatchedWorlds(n_worlds=9, n_lo=50, n_hi=3000, seed=5)
    t = bw.next_tick()
    assert t.obj_base[0] == 0 and t.obj_base[-1] == bw.n == t.xy.shape[0]
    assert t.q_base[0] == 0 and t.q_base[-1] == t.rects.shape[0]
    assert np.all(np.diff(t.obj_base.astype(np.int64)) >= 50) and np.all(np.diff(t.q_base.astype(np.int64)) >= 1)
    # each world's queries are centred on its own objects
    for w in range(9):
        a, b = int(t.obj_base[w]), int(t.obj_base[w + 1])
        qa, qb = int(t.q_base[w]), int(t.q_base[w + 1])
        c = (t.rects[qa:qb, :2] + t.rects[qa:qb, 2:]) / 2
        pts = t.xy[a:b]
        d = np.min(np.abs(c[:, None, 0] - pts[None, :, 0]) + np.abs(c[:, None, 1] - pts[None, :, 1]), axis=1)
        assert np.all(d < 1e-5)


def test_alternating_queries_share_the_hotspot_positions():
    """The two query regimes alternate tick by tick on the objects of one
    hotspot world: positions equal HotspotWalk's of the same seed, query
    counts and sides follow the regime of the tick."""
    w = workloads.AlternatingQueries(n=30_000, q_small=3_000, small_lo=0.0002, small_hi=0.001, q_large=40,
                                     large_lo=0.005, large_hi=0.02, seed=4)
    ref = workloads.HotspotWalk(n=30_000, q=1, seed=4)
    for k in range(4):
        t, r = w.next_tick(), ref.next_tick()
        np.testing.assert_array_equal(t.xy, r.xy)
        side = np.maximum(t.rects[:, 2] - t.rects[:, 0], t.rects[:, 3] - t.rects[:, 1])
        if k % 2 == 0:
            assert t.rects.shape[0] == 3_000 and side.max() <= 0.00101
        else:
            assert t.rects.shape[0] == 40 and side.min() >= 0.00499
