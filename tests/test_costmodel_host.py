"""Host-side logic of the choosers and tuners (no GPU): the per-region
capacity rule and the non-negative least squares that fits unit costs of
the logged work to the logged phase times."""
import numpy as np
import pytest

from paper_1411_3212_gb300.costmodel import nonneg_lstsq, region_caps


def test_region_caps_rule():
    """Per-region capacities of the cost-model chooser: 2^(a + b log2 d_r)
    with d_r the region's density over the mean; empty regions take 2^a."""
    counts = np.array([300, 100, 0, 0])            # densities 3, 1, -, - (mean 1 per region)
    np.testing.assert_array_equal(region_caps(counts, 1, 7, 0.0), [128] * 4)
    np.testing.assert_array_equal(region_caps(counts, 1, 7, 1.0), [384, 128, 128, 128])
    np.testing.assert_array_equal(region_caps(counts, 1, 7, -1.0), [43, 128, 128, 128])
    np.testing.assert_array_equal(region_caps(counts, 1, 14, 1.0), [16384, 16384, 16384, 16384])
    np.testing.assert_array_equal(region_caps([0, 0, 0, 0], 1, 3, 0.5), [8] * 4)
    big = np.zeros(16, np.int64)
    big[5] = 10 ** 6
    big[6] = 1
    c = region_caps(big, 2, 4, -1.0)
    assert c[5] == 1 and c[6] == 16384 and c[0] == 16
    with pytest.raises(ValueError):
        region_caps(counts, 2, 7, 0.0)


def test_nonneg_lstsq_recovers_nonnegative_coefficients():
    rng = np.random.default_rng(1)
    A = rng.uniform(0, 1, (40, 5))
    x = np.array([2.0, 0.0, 0.5, 3.0, 0.0])
    np.testing.assert_allclose(nonneg_lstsq(A, A @ x), x, atol=1e-9)
    # a target that ordinary least squares fits with a negative weight
    b = A @ np.array([1.0, 0.0, 0.0, 0.0, 0.0]) - 0.3 * A[:, 1]
    sol = nonneg_lstsq(A, b)
    assert np.all(sol >= 0) and sol[1] == 0.0
    # the kept columns are the least-squares fit on those columns alone
    keep = sol > 0
    ls, *_ = np.linalg.lstsq(A[:, keep], b, rcond=None)
    np.testing.assert_allclose(sol[keep], ls, atol=1e-9)


class _Float64Model:
    """The float64 reference network (oracle/cost_mlp.py) in place of the
    device model, so that the choosers' logic runs without a GPU."""

    def __init__(self, params):
        from oracle import cost_mlp
        self.mlp = cost_mlp
        self.p = np.asarray(params, np.float64)
        self.m = self.v = None
        self.step = 0

    def predict(self, X):
        return self.mlp.forward(self.p, np.asarray(X, np.float64))[0]

    def train(self, X, y, epochs, lr):
        X = np.asarray(X, np.float64)
        y = np.asarray(y, np.float64)
        self.p, self.m, self.v, _ = self.mlp.adam(self.p, X, y, epochs=epochs, lr=lr, m=self.m, v=self.v,
                                                  step0=self.step)
        self.step += epochs
        return self.mlp.loss(self.p, X, y)

    def close(self):
        pass


@pytest.fixture
def cpu_model(monkeypatch):
    from paper_1411_3212_gb300 import mqr
    monkeypatch.setattr(mqr, "CostModel", _Float64Model)


def _work(R, objects, tests, **extra):
    w = {k: np.zeros(R) for k in ("objects", "leaves", "queries", "side_log2_sum", "sub_intersecting",
                                  "sub_covering", "tests", "results_intersecting", "results_covering")}
    w["objects"] = np.asarray(objects, np.float64)
    w["queries"] = w["objects"] / 10
    w["side_log2_sum"] = w["queries"] * -9.0
    w["tests"] = np.asarray(tests, np.float64)
    for k, v in extra.items():
        w[k] = np.asarray(v, np.float64)
    return w


def test_region_chooser_fits_unit_costs_exactly(cpu_model):
    """Phase times that are exact non-negative combinations of the logged
    work give back those unit costs, and the region costs they price."""
    from paper_1411_3212_gb300.costmodel import RegionChooser
    ch = RegionChooser(region_bits=1, caps=(64, 128), explore_rounds=2, retrain_every=1, epochs=5)
    rng = np.random.default_rng(4)
    for _ in range(6):
        ch.choose()
        w = _work(4, rng.integers(1000, 9000, 4), rng.uniform(1e5, 1e6, 4),
                  sub_intersecting=rng.uniform(100, 900, 4), results_covering=rng.uniform(1e4, 1e5, 4))
        ms = 2e-9 * w["tests"].sum() + 5e-7 * w["sub_intersecting"].sum() + 1e-9 * w["results_covering"].sum() + 0.1
        ch.observe(w, {"filter": ms})
    np.testing.assert_allclose(ch.unit_cost[[0, 1, 4]], [2e-9, 5e-7, 1e-9], rtol=1e-6)
    assert np.all(ch.unit_cost >= 0)
    np.testing.assert_allclose(ch.region_costs(w), 2e-9 * w["tests"] + 5e-7 * w["sub_intersecting"] +
                               1e-9 * w["results_covering"], rtol=1e-6)


def test_region_chooser_learns_per_region_optimum_on_cpu(cpu_model):
    """The node-level chooser with the float64 network: regions whose best
    capacity grows with their density get their own best capacity, a clear
    gain over one capacity for all; empty regions keep the fallback."""
    from paper_1411_3212_gb300.costmodel import RegionChooser
    R = 16
    rng = np.random.default_rng(3)
    objects = np.exp2(rng.uniform(8, 18, R)).round()
    objects[5] = 0                                            # an empty region
    caps = np.array([32, 64, 128, 256, 512, 1024], np.float64)
    best = np.clip(np.round(4 + (np.log2(np.maximum(objects, 1)) - 8) * 0.5), 5, 10)

    def tick(cap_r):
        cost = (1 + 0.3 * (np.log2(cap_r) - best) ** 2) * objects / 65536.0
        return _work(R, objects, cost), {"filter": float(cost.sum())}

    ch = RegionChooser(region_bits=2, caps=caps, explore_rounds=5, epsilon=0.0, retrain_every=10, first_epochs=600,
                       seed=5)
    ch.observe(*tick(np.full(R, 128.0)))
    for _ in range(60):
        ch.observe(*tick(ch.choose().astype(np.float64)))
    got = ch.choose().astype(np.float64)
    live = objects > 0
    assert got[5] == 128                                      # the fallback for the empty region
    assert np.mean(np.log2(got[live]) == best[live]) >= 0.6
    model_cost = tick(got)[1]["filter"]
    fixed_cost = tick(np.full(R, 128.0))[1]["filter"]
    assert model_cost < 0.9 * fixed_cost


def test_index_chooser_on_cpu(cpu_model):
    """The per-tick chooser with the float64 network: round-robin
    exploration, then the cheapest configuration of a known cost (a region
    rule here), a gain over the fixed capacity; applying a choice configures
    an index through its calls."""
    from paper_1411_3212_gb300.costmodel import GRID, QUAD, REGIONS, IndexChooser
    cost = {(QUAD, 128): 1.9, (QUAD, 256): 1.8, (GRID, 8): 2.4, (REGIONS, 3, 8, 0.25): 1.6}
    ch = IndexChooser(candidates=list(cost), seed=2, epsilon=0.0)
    rng = np.random.default_rng(1)
    picks = []
    for k in range(40):
        side = -9.0 + 0.05 * rng.normal()
        c = ch.choose(4_000_000, 400_000, side)
        ch.record(c, 4_000_000, 400_000, side, cost[c] * (1 + 0.01 * rng.normal()))
        picks.append(c)
    assert picks[:8] == list(cost) * 2                        # two exploration rounds
    assert picks[-10:] == [(REGIONS, 3, 8, 0.25)] * 10
    assert np.mean([cost[c] for c in picks[-10:]]) < 0.9 * cost[(QUAD, 128)]

    calls = []

    class FakeIndex:
        def set_index(self, kind, leaf_cap=0, grid_level=0):
            calls.append(("index", kind, leaf_cap, grid_level))

        def set_region_caps(self, bits, caps=None):
            calls.append(("regions", bits, None if caps is None else list(caps)))

        def region_counts(self, bits):
            return np.array([300] + [100] * (4 ** bits - 1))

    ch.apply(FakeIndex(), (GRID, 8))
    ch.apply(FakeIndex(), (REGIONS, 1, 7, 1.0))
    assert calls[0] == ("regions", 0, None) and calls[1] == ("index", GRID, 0, 8)
    assert calls[2] == ("index", QUAD, 128, 0)
    assert calls[3][0] == "regions" and calls[3][1] == 1 and calls[3][2] == [256, 85, 85, 85]


def test_launch_autotuner_coordinate_descent():
    """The launch-shape tuner takes, kernel by kernel, the option with the
    smallest time (others held), leaves the index at the best shapes, and
    refuses shapes that change the results."""
    from paper_1411_3212_gb300.autotune import tune_launch_config

    class FakeIndex:
        def __init__(self):
            self.cfg = {}
            self.applied = []

        def set_launch_config(self, **cfg):
            self.cfg = dict(cfg)
            self.applied.append(dict(cfg))

    target = {"candidate": 4, "compact": 16, "filter": 2, "emit": 8}

    def timer(idx, ticks, kind, reps):
        ms = 1.0 + sum(abs(np.log2(idx.cfg[k]) - np.log2(v)) for k, v in target.items())
        return ms, 12345

    idx = FakeIndex()
    best, table = tune_launch_config(idx, [None], options=(2, 4, 8, 16), timer=timer)
    assert best == target and idx.cfg == target and len(table) == 16
    bad = FakeIndex()
    with pytest.raises(RuntimeError):
        tune_launch_config(bad, [None], options=(2, 8), timer=lambda i, t, k, r: (1.0, i.cfg["candidate"]))


def test_argmin_chooser_picks_the_cheapest_measured_configuration():
    """The network-free baseline: the same two exploration rounds, then the
    configuration with the smallest mean measured time; with no record of a
    candidate it falls back."""
    from paper_1411_3212_gb300.costmodel import GRID, QUAD, ArgminChooser
    cost = {(QUAD, 128): 1.9, (QUAD, 256): 1.7, (GRID, 8): 2.4}
    ch = ArgminChooser(candidates=list(cost), seed=1, epsilon=0.0)
    rng = np.random.default_rng(3)
    picks = []
    for k in range(20):
        c = ch.choose()
        ch.record(c, 0, 0, 0.0, cost[c] * (1 + 0.01 * rng.normal()))
        picks.append(c)
    assert picks[:6] == list(cost) * 2
    assert picks[-10:] == [(QUAD, 256)] * 10
    # a drift that makes another configuration cheaper is seen only through what is re-timed
    fresh = ArgminChooser(candidates=list(cost), explore_rounds=0, epsilon=0.0, fallback=(GRID, 8))
    assert fresh.choose() == (GRID, 8)


def test_world_capacity_tuner_coordinate_descent():
    """Per-world capacities: every label takes the capacity of the smallest
    time with the others held; worlds get their label's capacity in their
    region (world w = region w at depth world_bits); the results stay fixed."""
    from paper_1411_3212_gb300.autotune import tune_world_caps
    optimum = {"small": 64, "big": 512}
    classes = ["small", "big", "small", "big", "big"]        # 5 worlds, world_bits 2 (16 regions)

    class FakeIndex:
        caps = None

        def set_region_caps(self, bits, caps):
            assert bits == 2 and len(caps) == 16
            self.caps = np.array(caps)

    def timer(idx, ticks, kind, reps):
        ms = 0.0
        for w, c in enumerate(classes):
            ms += abs(np.log2(idx.caps[w]) - np.log2(optimum[c]))
        return 1.0 + ms, 12345
    fi = FakeIndex()
    best, vec, table = tune_world_caps(fi, [], 2, classes, caps=(32, 64, 128, 256, 512), timer=timer)
    assert best == optimum
    assert list(vec[:5]) == [64, 512, 64, 512, 512] and list(vec[5:]) == [128] * 11
    assert list(fi.caps) == list(vec)
    assert len(table) == 10

    def bad_timer(idx, ticks, kind, reps):
        return 1.0, int(idx.caps[0])
    with pytest.raises(RuntimeError, match="changed the results"):
        tune_world_caps(FakeIndex(), [], 2, classes, timer=bad_timer)
