"""The learned tick-cost model on the GPU against the double-precision
reference (oracle/cost_mlp.py): gradients, predictions and Adam training;
per-tick index switching keeps results identical; the chooser finds the
cheapest configuration of a known cost function."""
import numpy as np
import pytest

import oracle
from oracle import cost_mlp
from paper_1411_3212_gb300 import workloads
from tests.gpu_util import assert_same_csr, gpu_csr_sorted, to_dev, torch_dev

pytestmark = pytest.mark.gpu


def data(seed, n):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, size=(n, 5))
    y = 0.5 * X[:, 0] - X[:, 1] ** 2 + 0.3 * X[:, 2] * X[:, 3] + 0.1
    return X, y


@pytest.mark.parametrize("n", [1, 31, 200])
def test_gradient_and_prediction_match_float64(n):
    torch_dev()
    from paper_1411_3212_gb300 import mqr
    X, y = data(n, n)
    p0 = cost_mlp.init(7)
    m = mqr.CostModel(p0)
    g32, l32 = m.gradient(X, y)
    g64 = cost_mlp.grad(p0.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64),
                        y.astype(np.float32).astype(np.float64))
    scale = np.abs(g64).max()
    np.testing.assert_allclose(g32, g64, rtol=1e-3, atol=1e-5 * scale)
    assert l32 == pytest.approx(cost_mlp.loss(p0, X, y), rel=1e-4)
    out64, _ = cost_mlp.forward(p0, X)
    np.testing.assert_allclose(m.predict(X), out64, rtol=1e-4, atol=1e-4)
    m.close()


def test_adam_training_matches_reference_trajectory():
    torch_dev()
    from paper_1411_3212_gb300 import mqr
    X, y = data(3, 150)
    p0 = cost_mlp.init(11)
    m = mqr.CostModel(p0)
    l0 = cost_mlp.loss(p0, X, y)
    # a few steps: the parameters follow the float64 reference closely
    m.train(X, y, epochs=3, lr=1e-3)
    p_ref, _, _, _ = cost_mlp.adam(p0, X, y, epochs=3, lr=1e-3)
    moved = np.abs(p_ref - p0) > 1e-4                      # parameters the reference really moved
    np.testing.assert_allclose(m.params()[moved], p_ref[moved], atol=3e-4)
    # a longer run learns the target as the reference does
    m.set_params(p0)
    m.train(X, y, epochs=400, lr=3e-3)
    p_ref, _, _, _ = cost_mlp.adam(p0, X, y, epochs=400, lr=3e-3)
    l_gpu = cost_mlp.loss(m.params().astype(np.float64), X, y)
    assert l_gpu < 0.1 * l0
    assert l_gpu < 3.0 * cost_mlp.loss(p_ref, X, y) + 1e-3
    m.close()


def test_set_index_between_ticks_keeps_results():
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    w = workloads.HotspotWalk(n=30000, q=2000, hotspots=6, side_lo=0.001, side_hi=0.03, seed=21)
    t = w.next_tick()
    st = oracle.State(30000)
    st.apply_updates(t.ids, t.xy)
    want = oracle.join_grid(st, t.rects, cell_side=0.005)
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=128, max_objects=30000)
    idx.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
    for kind, v in [(0, 8), (1, 6), (0, 512), (1, 9), (0, 128)]:
        if kind == 0:
            idx.set_index(0, leaf_cap=v)
        else:
            idx.set_index(1, grid_level=v)
        assert_same_csr(gpu_csr_sorted(idx, t.rects, dev), want, str((kind, v)))
    with pytest.raises(mqr.MqrError):
        idx.set_index(0, leaf_cap=0)
    with pytest.raises(mqr.MqrError):
        idx.set_index(1, grid_level=16)
    idx.close()


def test_chooser_learns_the_cheapest_configuration():
    torch_dev()
    from paper_1411_3212_gb300.costmodel import QUAD, IndexChooser
    # a known cost: cheapest at leaf capacity 256 for these tick sizes
    cost = {64: 2.3, 128: 1.9, 256: 1.75, 512: 1.85}
    ch = IndexChooser(seed=4, epsilon=0.0)
    rng = np.random.default_rng(0)
    picks = []
    for k in range(40):
        n, q, side = 4_000_000, 400_000, -9.0 + 0.05 * rng.normal()
        c = ch.choose(n, q, side)
        ms = cost[c[1]] * (1 + 0.01 * rng.normal())
        ch.record(c, n, q, side, ms)
        picks.append(c)
    assert all(c[0] == QUAD for c in picks)
    assert picks[-10:] == [(QUAD, 256)] * 10
    # the gain over the method without the model (the fixed capacity 128)
    assert np.mean([cost[c[1]] for c in picks[-10:]]) <= 0.93 * cost[128]
    ch.close()


def test_chooser_learns_a_region_candidate():
    """With per-region candidates among the configurations, the chooser
    settles on the cheapest one of a known cost function."""
    torch_dev()
    from paper_1411_3212_gb300.costmodel import GRID, QUAD, REGIONS, IndexChooser
    cost = {(QUAD, 128): 1.9, (QUAD, 256): 1.8, (GRID, 8): 2.4, (REGIONS, 3, 8, 0.25): 1.6,
            (REGIONS, 3, 8, -0.25): 2.0, (REGIONS, 3, 7, 0.5): 1.75}
    ch = IndexChooser(candidates=list(cost), seed=2, epsilon=0.0)
    rng = np.random.default_rng(1)
    picks = []
    for k in range(48):
        side = -9.0 + 0.05 * rng.normal()
        c = ch.choose(4_000_000, 400_000, side)
        ch.record(c, 4_000_000, 400_000, side, cost[c] * (1 + 0.01 * rng.normal()))
        picks.append(c)
    assert picks[-10:] == [(REGIONS, 3, 8, 0.25)] * 10
    assert np.mean([cost[c] for c in picks[-10:]]) <= 0.85 * cost[(QUAD, 128)]   # gain over the fixed capacity
    ch.close()


def test_region_chooser_learns_per_region_optimum():
    """Synthetic per-region costs whose best capacity grows with the region's
    density: after exploration the node-level model gives most regions their
    own best capacity (neighbouring candidates cost within a few percent)."""
    torch_dev()
    from paper_1411_3212_gb300.costmodel import RegionChooser
    rb = 2
    R = 16
    rng = np.random.default_rng(3)
    objects = np.exp2(rng.uniform(8, 18, R)).round()
    queries = (objects / 10).round()
    caps = np.array([32, 64, 128, 256, 512, 1024], np.float64)
    best = np.clip(np.round(4 + (np.log2(objects) - 8) * 0.5), 5, 10)      # log2 of the best capacity

    def work_for(cap_r):
        # region cost 1 ms x (1 + 0.3 (log2 cap - best)^2) x objects / 2^16, as filter tests at 1 ms each
        cost = (1 + 0.3 * (np.log2(cap_r) - best) ** 2) * objects / 65536.0
        w = {k: np.zeros(R) for k in ("objects", "leaves", "queries", "side_log2_sum", "sub_intersecting",
                                      "sub_covering", "tests", "results_intersecting", "results_covering")}
        w["objects"] = objects.copy()
        w["queries"] = queries.copy()
        w["side_log2_sum"] = queries * -9.0
        w["tests"] = cost
        return w, {"filter": float(cost.sum())}

    ch = RegionChooser(region_bits=rb, caps=caps, explore_rounds=5, epsilon=0.0, retrain_every=10, first_epochs=600,
                       seed=5)
    w, ph = work_for(np.full(R, 128.0))
    ch.observe(w, ph)                                  # a first tick at the fallback capacity
    for k in range(60):
        c = ch.choose().astype(np.float64)
        w, ph = work_for(c)
        ch.observe(w, ph)
    got = np.log2(ch.choose().astype(np.float64))
    assert np.mean(np.abs(got - best) <= 1) >= 0.9, (got, best)
    assert np.mean(got == best) >= 0.6, (got, best)
    # the gain over one fixed capacity for every region (128, the method without the model)
    w_model, _ = work_for(np.exp2(got))
    w_fixed, _ = work_for(np.full(R, 128.0))
    assert w_model["tests"].sum() < 0.9 * w_fixed["tests"].sum()
    ch.close()
