"""Per-tick choice of the index configuration by a learned cost model.

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

    def close(self):
        self.model.close()


def mean_log2_side(rects: np.ndarray) -> float:
    s = np.maximum(np.maximum(rects[:, 2] - rects[:, 0], rects[:, 3] - rects[:, 1]), 1e-9)
    return float(np.mean(np.log2(s)))
