"""Choice of the index configuration by learned cost models: per tick
(IndexChooser) and per region of the quadtree (RegionChooser).

Every index configuration answers every tick exactly (the index only decides
how much work the filter does, never a result), so the configuration of the
next tick can be chosen for speed alone.  The paper reasons about that cost
analytically (the filtering complexity of Sec. 5.4; the estimated number of
intersecting subqueries of Sec. 6) and fixes the quadtree threshold per
experiment; here an MLP (5 -> 64 -> 64 -> 1, trained on the device by the
library's own kernels, `mqr_cost_*`) learns log(tick time) from the ticks
already run, and the chooser takes the configuration with the smallest
prediction -- after a round-robin exploration of the candidates, with a
small exploration rate afterwards, and the fixed configuration as fallback
while there is too little data.

Configurations: the quadtree with one leaf capacity (QUAD, cap), the uniform
grid (GRID, level), and the quadtree with per-region capacities (REGIONS,
region_bits, a, b): region r of density d_r (objects per unit area over the
mean, counted on the device from the previous tick) splits at
2^(a + b log2 d_r).  b = 0 is one capacity everywhere; b = 1 keeps leaves of
one size, like a grid.

Features of a (tick, configuration): log2 objects, log2 queries, the mean
log2 of the query sides, log2 of the objects per leaf the configuration aims
for at the mean density (leaf capacity, objects per grid cell, or 2^a), and
how that target scales with the local density (0 for one capacity, 1 for the
grid, b for per-region capacities).  Scheduling and marshalling only: the
ticks and the model's arithmetic run in the library's kernels.
"""
from __future__ import annotations

import math

import numpy as np

from . import mqr

QUAD, GRID, REGIONS = 0, 1, 2
MAX_REGION_CAP = 16384


def region_caps(counts, region_bits, a, b):
    """Per-region capacities 2^(a + b log2 d_r), d_r = the region's objects per
    unit area over the mean (empty regions: 2^a), rounded, within 1..16384."""
    c = np.asarray(counts, np.float64)
    if c.shape != (4 ** region_bits,):
        raise ValueError("counts must hold 4^region_bits entries")
    total = c.sum()
    d = c * (4 ** region_bits) / total if total > 0 else np.ones_like(c)
    ld = np.where(c > 0, np.log2(np.maximum(d, 1e-30)), 0.0)
    return np.clip(np.rint(np.exp2(a + b * ld)), 1, MAX_REGION_CAP).astype(np.uint32)


def he_uniform_params(seed: int) -> np.ndarray:
    """Initial parameters in the C ABI layout (W1, b1, W2, b2, W3, b3)."""
    rng = np.random.default_rng(seed)
    w1 = rng.uniform(-1, 1, (64, 5)) * math.sqrt(6.0 / 5)
    w2 = rng.uniform(-1, 1, (64, 64)) * math.sqrt(6.0 / 64)
    w3 = rng.uniform(-1, 1, 64) * math.sqrt(6.0 / 64)
    return np.concatenate([w1.ravel(), np.zeros(64), w2.ravel(), np.zeros(64), w3, [0.0]]).astype(np.float32)


class IndexChooser:
    def __init__(self, candidates=((QUAD, 64), (QUAD, 128), (QUAD, 256), (QUAD, 512)),
                 fallback=(QUAD, 128), explore_rounds=2, epsilon=0.1, retrain_every=4, epochs=400, lr=3e-3,
                 seed=0):
        self.cands = [tuple(c) for c in candidates]
        self.fallback = tuple(fallback)
        self.explore_rounds = explore_rounds
        self.epsilon = epsilon
        self.retrain_every = retrain_every
        self.epochs, self.lr = epochs, lr
        self.rng = np.random.default_rng(seed)
        self.model = mqr.CostModel(he_uniform_params(seed))
        self.X, self.y = [], []
        self.trained = False
        self.n_choices = 0

    @staticmethod
    def features(cand, n_objects, n_queries, mean_log2_side):
        kind = cand[0]
        if kind == QUAD:
            per_leaf, slope = cand[1], 0.0
        elif kind == GRID:
            per_leaf, slope = max(n_objects / float(4 ** cand[1]), 1e-3), 1.0
        else:
            per_leaf, slope = 2.0 ** cand[2], float(cand[3])
        return np.array([math.log2(max(n_objects, 1)) / 32.0, math.log2(max(n_queries, 1)) / 32.0,
                         mean_log2_side / 16.0, math.log2(per_leaf) / 16.0, slope], np.float32)

    def choose(self, n_objects, n_queries, mean_log2_side):
        k = self.n_choices
        self.n_choices += 1
        if k < self.explore_rounds * len(self.cands):                 # round-robin exploration
            return self.cands[k % len(self.cands)]
        if not self.trained:
            return self.fallback
        if self.rng.random() < self.epsilon:
            return self.cands[int(self.rng.integers(len(self.cands)))]
        X = np.stack([self.features(c, n_objects, n_queries, mean_log2_side) for c in self.cands])
        return self.cands[int(np.argmin(self.model.predict(X)))]

    def record(self, cand, n_objects, n_queries, mean_log2_side, ms):
        self.X.append(self.features(cand, n_objects, n_queries, mean_log2_side))
        self.y.append(math.log(max(ms, 1e-6)))
        if len(self.y) >= len(self.cands) and len(self.y) % self.retrain_every == 0:
            self.loss = self.model.train(np.stack(self.X), np.array(self.y, np.float32), self.epochs, self.lr)
            self.trained = True

    def apply(self, idx, cand):
        apply_config(idx, cand)

    def close(self):
        self.model.close()


class ArgminChooser:
    """The same choice without a network, as the learned chooser's baseline:
    the same round-robin exploration and exploration rate, then the candidate
    whose measured tick times (its last `window` records) have the smallest
    mean.  It knows only the configurations it has timed, on the conditions
    under which it timed them; the network also predicts from the tick's
    features."""

    def __init__(self, candidates=((QUAD, 64), (QUAD, 128), (QUAD, 256), (QUAD, 512)),
                 fallback=(QUAD, 128), explore_rounds=2, epsilon=0.1, window=8, seed=0):
        self.cands = [tuple(c) for c in candidates]
        self.fallback = tuple(fallback)
        self.explore_rounds = explore_rounds
        self.epsilon = epsilon
        self.window = window
        self.rng = np.random.default_rng(seed)
        self.times = {c: [] for c in self.cands}
        self.n_choices = 0

    def choose(self, n_objects=0, n_queries=0, mean_log2_side=0.0):
        k = self.n_choices
        self.n_choices += 1
        if k < self.explore_rounds * len(self.cands):                 # round-robin exploration
            return self.cands[k % len(self.cands)]
        if self.rng.random() < self.epsilon:
            return self.cands[int(self.rng.integers(len(self.cands)))]
        timed = [c for c in self.cands if self.times[c]]
        if not timed:
            return self.fallback
        return min(timed, key=lambda c: float(np.mean(self.times[c][-self.window:])))

    def record(self, cand, n_objects, n_queries, mean_log2_side, ms):
        self.times[tuple(cand)].append(float(ms))

    def apply(self, idx, cand):
        apply_config(idx, cand)

    def close(self):
        pass


def apply_config(idx, cand):
    """Configure the index for the next tick (between ticks: leaves are
    rebuilt every tick, results never change)."""
    kind = cand[0]
    if kind == REGIONS:
        _, rb, a, b = cand
        try:
            counts = idx.region_counts(rb)          # densities of the previous tick
        except mqr.MqrError:                        # no tick yet: one capacity
            counts = np.ones(4 ** rb, np.uint32)
        idx.set_index(QUAD, leaf_cap=int(min(2 ** a, MAX_REGION_CAP)))
        idx.set_region_caps(rb, region_caps(counts, rb, a, b))
        return
    idx.set_region_caps(0)
    if kind == QUAD:
        idx.set_index(QUAD, leaf_cap=cand[1])
    else:
        idx.set_index(GRID, grid_level=cand[1])


# Phases whose time depends on the split thresholds (the rest -- updates,
# keys, sort -- does not), and the kinds of per-region work they do.
THRESHOLD_PHASES = ("leaves", "query_blocks", "candidates", "group", "filter", "result_scan", "emit")
WORK_KINDS = ("tests", "sub_intersecting", "sub_covering", "results_intersecting", "results_covering", "leaves")


def nonneg_lstsq(A, b):
    """Least squares with non-negative coefficients: solve, drop the columns
    whose coefficient is negative, solve again (until none is)."""
    keep = np.ones(A.shape[1], bool)
    x = np.zeros(A.shape[1])
    while keep.any():
        sol, *_ = np.linalg.lstsq(A[:, keep], b, rcond=None)
        if np.all(sol >= 0):
            x[keep] = sol
            break
        idx = np.nonzero(keep)[0]
        keep[idx[sol < 0]] = False
    return x


class RegionChooser:
    """Per-region split thresholds chosen by an MLP over node features.

    After every tick the method logs, per region (the quadrants of depth
    region_bits), its objects, queries, query sides, leaves, subqueries,
    containment tests and results (`mqr_region_work`), and the tick's time per
    phase (the library's phase timing).  The time of the threshold-dependent
    phases is fitted, over the logged ticks, as a non-negative combination of
    the tick's work of each kind (WORK_KINDS) plus a constant; the fitted unit
    costs price each region's work, which gives a cost per region and tick.
    The MLP (the library's, trained on the device) maps a region's features
    -- log2 objects, log2 queries, mean log2 query side, log2 area, log2
    capacity, standardised over the samples -- to log(cost), standardised; the next tick gives each region the candidate
    capacity with the smallest prediction if that beats the best single
    capacity (smallest predicted total) by the margin, else the best single
    capacity.  Exploration: every candidate capacity for all regions at once,
    explore_rounds times (so that the unit costs are identifiable and every
    region is seen at every capacity), then a neighbouring capacity (half or
    double) for a fraction epsilon of the regions; the fallback capacity for empty regions.  Results
    never depend on the choice.
    """

    def __init__(self, region_bits=3, caps=(32, 64, 128, 256, 512, 1024), fallback=128, explore_rounds=2,
                 epsilon=0.02, margin=0.05, retrain_every=4, epochs=100, first_epochs=400, lr=3e-3,
                 timing_every=10, max_samples=4096, seed=0):
        self.rb = int(region_bits)
        self.R = 4 ** self.rb
        self.caps = np.array(caps, np.float64)
        self.fallback = int(fallback)
        self.explore_ticks = explore_rounds * len(self.caps)
        self.epsilon = epsilon
        self.margin = margin
        self.retrain_every = retrain_every
        self.epochs, self.first_epochs, self.lr = epochs, first_epochs, lr
        self.timing_every = timing_every
        self._timed = False
        self.max_samples = max_samples
        self.rng = np.random.default_rng(seed)
        self.model = mqr.CostModel(he_uniform_params(seed))
        self.X, self.W = [], []            # per-region samples: features, work by kind
        self.tick_work, self.tick_ms = [], []
        self.unit_cost = None
        self.trained = False
        self.ticks = 0
        self.last_work = None
        self.current = np.full(self.R, self.fallback, np.uint32)
        self._t0 = None

    def features(self, work, caps):
        """Node features of every region under the capacities caps[R]."""
        n = work["objects"]
        q = work["queries"]
        side = np.where(q > 0, work["side_log2_sum"] / np.maximum(q, 1), -16.0)
        area = np.full(self.R, -2.0 * self.rb)
        return np.stack([np.log2(1 + n) / 32.0, np.log2(1 + q) / 32.0, side / 16.0, area / 16.0,
                         np.log2(np.asarray(caps, np.float64)) / 16.0], 1).astype(np.float32)

    def region_costs(self, work):
        """Cost (ms) of every region's work at the fitted unit costs."""
        if self.unit_cost is None:
            return np.zeros(self.R)
        return np.stack([work[k] for k in WORK_KINDS], 1) @ self.unit_cost

    def choose(self):
        """Capacities for the next tick, from the regions of the last one."""
        k = self.ticks
        if self.last_work is None:
            caps = np.full(self.R, float(self.fallback))
        elif k < self.explore_ticks:
            caps = np.full(self.R, self.caps[k % len(self.caps)])
        elif not self.trained:
            caps = np.full(self.R, float(self.fallback))
        else:
            C = len(self.caps)
            X = np.concatenate([self.features(self.last_work, np.full(self.R, c)) for c in self.caps])
            pred = self.model.predict((X - self.x_mean) / self.x_std).reshape(C, self.R)
            pc = np.exp(pred * self.y_std + self.y_mean)              # predicted cost, ms
            live = self.last_work["objects"] > 0
            base = int(np.argmin(pc[:, live].sum(1)))                 # the best single capacity
            best = np.argmin(pc, axis=0)
            r = np.arange(self.R)
            own = pc[best, r] < (1.0 - self.margin) * pc[base, r]     # a region leaves it only for a clear gain
            j = np.where(own, best, base)
            flip = self.rng.random(self.R) < self.epsilon          # explore a neighbouring capacity
            j[flip] = np.clip(j[flip] + self.rng.choice([-1, 1], int(flip.sum())), 0, C - 1)
            caps = self.caps[j]
        if self.last_work is not None:
            caps = np.where(self.last_work["objects"] > 0, caps, self.fallback)
        self.current = np.asarray(caps, np.float64).clip(1, MAX_REGION_CAP).astype(np.uint32)
        return self.current

    def apply(self, idx):
        """Configure the next tick.  Phase timing (events between the phases,
        tens of microseconds a tick) runs on the exploration ticks and on
        every timing_every-th tick, which refit the unit costs."""
        timed = self.ticks < self.explore_ticks or self.ticks % self.timing_every == 0
        if timed != self._timed:
            idx.set_timing(timed)
            self._timed = timed
        idx.set_index(QUAD, leaf_cap=self.fallback)
        idx.set_region_caps(self.rb, self.choose())
        self._t0 = idx.timing()["ms"] if timed else None

    def record(self, idx, rects_dev):
        """Log the tick just run with apply()'s capacities."""
        phase_ms = None
        if self._t0 is not None:
            t1 = idx.timing()["ms"]
            phase_ms = {p: t1[p] - self._t0.get(p, 0.0) for p in t1}
        self.observe(idx.region_work(rects_dev, self.rb), phase_ms)

    def finish(self, idx):
        """Switch the phase timing off again."""
        if self._timed:
            idx.set_timing(False)
            self._timed = False

    def observe(self, work, phase_ms=None):
        """Add one tick (work as mqr_region_work returns it, and the phase
        times in ms if the tick was timed) run under the current capacities;
        refit and retrain."""
        if phase_ms is not None:
            self.tick_work.append([work[k].sum() for k in WORK_KINDS])
            self.tick_ms.append(sum(phase_ms.get(p, 0.0) for p in THRESHOLD_PHASES))
        live = work["objects"] > 0
        self.X.extend(self.features(work, self.current)[live])
        self.W.extend(np.stack([work[k] for k in WORK_KINDS], 1)[live])
        self.X, self.W = self.X[-self.max_samples:], self.W[-self.max_samples:]
        self.last_work = work
        self.ticks += 1
        if self.ticks >= self.explore_ticks and self.ticks % self.retrain_every == 0:
            A = np.concatenate([np.array(self.tick_work), np.ones((len(self.tick_ms), 1))], 1)
            scale = np.maximum(A.max(axis=0), 1e-30)
            sol = nonneg_lstsq(A / scale, np.array(self.tick_ms)) / scale
            self.unit_cost = sol[:-1]
            cost = np.array(self.W) @ self.unit_cost
            ok = cost > 0
            if ok.any():
                # standardised features and targets (the targets span several
                # orders of magnitude across regions)
                X = np.stack(self.X)[ok].astype(np.float64)
                y = np.log(cost[ok])
                self.x_mean, self.x_std = X.mean(0), X.std(0)
                self.x_std[self.x_std == 0] = 1.0
                self.y_mean, self.y_std = y.mean(), max(y.std(), 1e-12)
                self.loss = self.model.train(((X - self.x_mean) / self.x_std).astype(np.float32),
                                             ((y - self.y_mean) / self.y_std).astype(np.float32),
                                             self.epochs if self.trained else self.first_epochs, self.lr)
                self.trained = True

    def close(self):
        self.model.close()


def mean_log2_side(rects: np.ndarray) -> float:
    s = np.maximum(np.maximum(rects[:, 2] - rects[:, 0], rects[:, 3] - rects[:, 1]), 1e-9)
    return float(np.mean(np.log2(s)))
