"""Seeded synthetic workloads for the repeated-range-query join.

This module only draws inputs: object positions, per-tick moves and query
rectangles.  It holds none of the join's arithmetic, so both the CUDA path and
the CPU oracle (which never import each other) can be fed from it.

The paper's own generator (a Brinkhoff-derived moving-object generator inside
a third-party benchmarking framework, Sec. 6) and its road-network dataset are
not available; these generators keep the structure of its workloads (Table 1):
uniform or Gaussian-hotspot object distributions, square queries centred on
the objects that issue them, bounded random-walk motion between ticks.  The
paper's region is a 22500u square with query sides of 200-800u; here the
region is the unit square and sides are given as fractions of it.

All draws use ``numpy.random.default_rng`` seeded through ``SeedSequence``;
values are produced in float64, clamped, then cast to float32.  Query corners
are computed in float32 as ``c - s/2`` and ``c + s/2`` (round to nearest), so a
query always contains the object that issued it (self-inclusion, Def. 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

TOP = np.float32(1.0) - np.float32(2.0 ** -24)   # largest float32 below 1


def _rngs(seed: int, k: int):
    return [np.random.default_rng(s) for s in np.random.SeedSequence(seed).spawn(k)]


def squares_around(centres: np.ndarray, sides) -> np.ndarray:
    """Closed squares (xa, ya, xb, yb) of the given sides centred on ``centres``."""
    c = np.asarray(centres, np.float32).reshape(-1, 2)
    h = (np.asarray(sides, np.float64) / 2.0).astype(np.float32)
    h = np.broadcast_to(h, (c.shape[0],))
    out = np.empty((c.shape[0], 4), np.float32)
    out[:, 0] = c[:, 0] - h
    out[:, 1] = c[:, 1] - h
    out[:, 2] = c[:, 0] + h
    out[:, 3] = c[:, 1] + h
    return out


def uniform_points(n: int, rng) -> np.ndarray:
    return np.clip(rng.random((n, 2)), 0.0, TOP).astype(np.float32)


@dataclass
class Tick:
    """One tick: the updates of the tick (ids, xy) and its queries."""
    ids: np.ndarray          # u32[n]
    xy: np.ndarray           # f32[n, 2]
    rects: np.ndarray        # f32[Q, 4]  (xa, ya, xb, yb)
    issuers: np.ndarray      # u32[Q]     object that issued each query
    arrivals: np.ndarray = None   # f64[Q]  served streams: arrival time inside the tick, s (ascending)


# ----------------------------------------------------------------------------
# 16K uniform objects, 1,024 side-0.01 queries, one tick.
# ----------------------------------------------------------------------------
def uniform_small(seed: int = 0, n: int = 16384, q: int = 1024, side: float = 0.01) -> Tick:
    r_init, r_q = _rngs(seed, 2)
    xy = uniform_points(n, r_init)
    iss = r_q.integers(0, n, size=q).astype(np.uint32)       # with replacement
    rects = squares_around(xy[iss], side)
    return Tick(np.arange(n, dtype=np.uint32), xy, rects, iss)


# ----------------------------------------------------------------------------
# Random-walk world: uniform start, Gaussian steps clamped to the unit square,
# a fixed fraction of objects issuing fixed-side queries each tick.
# ----------------------------------------------------------------------------
@dataclass
class UniformWalk:
    n: int = 1_000_000
    q: int = 100_000
    side: float = 0.002
    step: float = 0.0005
    seed: int = 0
    _xy: np.ndarray = field(init=False, repr=False)

    def __post_init__(self):
        self._r_init, self._r_move, self._r_q = _rngs(self.seed, 3)
        self._xy = uniform_points(self.n, self._r_init).astype(np.float64)
        self._t = 0

    def next_tick(self) -> Tick:
        if self._t > 0:
            self._xy = np.clip(self._xy + self._r_move.normal(0.0, self.step, (self.n, 2)), 0.0, float(TOP))
        self._t += 1
        xy = self._xy.astype(np.float32)
        iss = np.sort(self._r_q.choice(self.n, size=self.q, replace=False)).astype(np.uint32)
        rects = squares_around(xy[iss], self.side)
        return Tick(np.arange(self.n, dtype=np.uint32), xy, rects, iss)


# ----------------------------------------------------------------------------
# Skewed world: a mixture of Gaussian hotspots (centres uniform, sigma
# log-uniform) plus a uniform background; objects random-walk and hotspot
# members also follow their hotspot's drift (fixed heading per hotspot,
# reflected at the borders); queries of log-uniform side centred on objects
# sampled without replacement.
# ----------------------------------------------------------------------------
@dataclass
class HotspotWalk:
    n: int = 4_000_000
    q: int = 400_000
    hotspots: int = 64
    frac_hot: float = 0.9
    sigma_lo: float = 0.002
    sigma_hi: float = 0.02
    side_lo: float = 0.0005
    side_hi: float = 0.005
    step: float = 0.0005
    drift: float = 0.001
    seed: int = 0

    def __post_init__(self):
        r_init, self._r_move, self._r_q, r_hot = _rngs(self.seed, 4)
        H = self.hotspots
        self.centres = r_hot.random((H, 2))
        self.sigmas = np.exp(r_hot.uniform(np.log(self.sigma_lo), np.log(self.sigma_hi), H))
        ang = r_hot.uniform(0.0, 2.0 * np.pi, H)
        self.heading = np.stack([np.cos(ang), np.sin(ang)], 1)
        n_hot = int(round(self.n * self.frac_hot))
        member = np.full(self.n, -1, np.int64)
        member[:n_hot] = r_init.integers(0, H, size=n_hot)
        r_init.shuffle(member)
        self.member = member
        hot = member >= 0
        xy = np.empty((self.n, 2))
        xy[hot] = self.centres[member[hot]] + r_init.normal(0.0, 1.0, (int(hot.sum()), 2)) * self.sigmas[member[hot], None]
        xy[~hot] = r_init.random((int((~hot).sum()), 2))
        self._xy = np.clip(xy, 0.0, float(TOP))
        self._t = 0

    def _advance_hotspots(self):
        c = self.centres + self.heading * self.drift
        for d in range(2):
            lo = c[:, d] < 0.0
            hi = c[:, d] > 1.0
            c[lo, d] = -c[lo, d]
            c[hi, d] = 2.0 - c[hi, d]
            self.heading[lo | hi, d] *= -1.0
        delta = c - self.centres
        self.centres = c
        return delta

    def next_tick(self) -> Tick:
        if self._t > 0:
            delta = self._advance_hotspots()
            hot = self.member >= 0
            move = self._r_move.normal(0.0, self.step, (self.n, 2))
            move[hot] += delta[self.member[hot]]
            self._xy = np.clip(self._xy + move, 0.0, float(TOP))
        self._t += 1
        xy = self._xy.astype(np.float32)
        iss = np.sort(self._r_q.choice(self.n, size=self.q, replace=False)).astype(np.uint32)
        sides = np.exp(self._r_q.uniform(np.log(self.side_lo), np.log(self.side_hi), self.q))
        rects = squares_around(xy[iss], sides)
        return Tick(np.arange(self.n, dtype=np.uint32), xy, rects, iss)


# ----------------------------------------------------------------------------
# Alternating queries: the hotspot world, whose ticks alternate between two
# query regimes -- many small squares (even ticks) and few large ones (odd
# ticks).  The best index configuration differs between the regimes, so a
# chooser that ignores the tick's features can only find one compromise.
# Both regimes come from HotspotWalk generators of one seed, whose object
# positions are drawn from their own random streams and therefore agree.
# ----------------------------------------------------------------------------
class AlternatingQueries:
    def __init__(self, n: int = 4_000_000, q_small: int = 400_000, small_lo: float = 0.0002,
                 small_hi: float = 0.001, q_large: int = 4_000, large_lo: float = 0.005, large_hi: float = 0.02,
                 seed: int = 0):
        self.n = n
        self.regimes = [HotspotWalk(n=n, q=q_small, side_lo=small_lo, side_hi=small_hi, seed=seed),
                        HotspotWalk(n=n, q=q_large, side_lo=large_lo, side_hi=large_hi, seed=seed)]
        self._t = 0

    def next_tick(self) -> Tick:
        ticks = [g.next_tick() for g in self.regimes]     # both advance: the same positions
        t = ticks[self._t % 2]
        self._t += 1
        return t


# ----------------------------------------------------------------------------
# Mixed density: the left half of the square holds Gaussian hotspots (a
# fraction frac_dense of the objects) queried by many small squares, the right
# half a uniform sparse population queried by few large squares; objects
# random-walk inside their half.  A workload whose regions prefer different
# leaf capacities.
# ----------------------------------------------------------------------------
@dataclass
class MixedDensity:
    n: int = 4_000_000
    q_small: int = 300_000
    q_large: int = 10_000
    frac_dense: float = 0.75
    hotspots: int = 32
    sigma: float = 0.01
    small_lo: float = 0.0003
    small_hi: float = 0.001
    large_lo: float = 0.01
    large_hi: float = 0.04
    step: float = 0.0005
    seed: int = 0

    def __post_init__(self):
        r_init, self._r_move, self._r_q = _rngs(self.seed, 3)
        self.n_dense = int(round(self.n * self.frac_dense))
        cent = np.column_stack([r_init.uniform(0.05, 0.45, self.hotspots), r_init.uniform(0.05, 0.95, self.hotspots)])
        k = r_init.integers(0, self.hotspots, self.n_dense)
        dense = cent[k] + r_init.normal(0.0, self.sigma, (self.n_dense, 2))
        sparse = np.column_stack([r_init.uniform(0.5, 1.0, self.n - self.n_dense),
                                  r_init.uniform(0.0, 1.0, self.n - self.n_dense)])
        self._xy = self._clamp(np.concatenate([dense, sparse]))
        self._t = 0

    def _clamp(self, xy):
        xy[: self.n_dense, 0] = np.clip(xy[: self.n_dense, 0], 0.0, 0.4999)
        xy[self.n_dense:, 0] = np.clip(xy[self.n_dense:, 0], 0.5, float(TOP))
        xy[:, 1] = np.clip(xy[:, 1], 0.0, float(TOP))
        return xy

    @property
    def q(self):
        return self.q_small + self.q_large

    def next_tick(self) -> Tick:
        if self._t > 0:
            self._xy = self._clamp(self._xy + self._r_move.normal(0.0, self.step, (self.n, 2)))
        self._t += 1
        xy = self._xy.astype(np.float32)
        iss_s = self._r_q.choice(self.n_dense, size=self.q_small, replace=False)
        iss_l = self.n_dense + self._r_q.choice(self.n - self.n_dense, size=self.q_large, replace=False)
        iss = np.concatenate([np.sort(iss_s), np.sort(iss_l)]).astype(np.uint32)
        sides = np.concatenate([np.exp(self._r_q.uniform(np.log(self.small_lo), np.log(self.small_hi), self.q_small)),
                                np.exp(self._r_q.uniform(np.log(self.large_lo), np.log(self.large_hi), self.q_large))])
        rects = squares_around(xy[iss], sides)
        return Tick(np.arange(self.n, dtype=np.uint32), xy, rects, iss)


# ----------------------------------------------------------------------------
# Served stream: a denser hotspot world (95% of the objects in 16 hotspots of
# sigma 0.005) whose queries arrive as a Poisson process of the given rate;
# the queries arriving during a tick of duration dt form that tick's batch
# (Sec. 2.2), each with its arrival time inside the tick (for the latency of
# Def. 2-3).  Issuers are drawn with replacement (several queries of one
# object may share a tick).
# ----------------------------------------------------------------------------
@dataclass
class ServedWorld(HotspotWalk):
    n: int = 10_000_000
    hotspots: int = 16
    frac_hot: float = 0.95
    sigma_lo: float = 0.005
    sigma_hi: float = 0.005
    side_lo: float = 0.0005
    side_hi: float = 0.004
    rate: float = 5.0e6          # query arrivals per second
    dt: float = 0.010            # tick duration, s

    def next_tick(self) -> Tick:
        if self._t > 0:
            delta = self._advance_hotspots()
            hot = self.member >= 0
            move = self._r_move.normal(0.0, self.step, (self.n, 2))
            move[hot] += delta[self.member[hot]]
            self._xy = np.clip(self._xy + move, 0.0, float(TOP))
        self._t += 1
        xy = self._xy.astype(np.float32)
        q = int(self._r_q.poisson(self.rate * self.dt))
        arrivals = np.sort(self._r_q.random(q)) * self.dt
        iss = self._r_q.integers(0, self.n, size=q).astype(np.uint32)
        sides = np.exp(self._r_q.uniform(np.log(self.side_lo), np.log(self.side_hi), q))
        rects = squares_around(xy[iss], sides)
        return Tick(np.arange(self.n, dtype=np.uint32), xy, rects, iss, arrivals)


# ----------------------------------------------------------------------------
# Batched independent worlds: world sizes log-uniform in [n_lo, n_hi], half of
# the worlds uniform random walks, half hotspot walks (8 hotspots of sigma
# 0.01); each world issues n_w * q_frac fixed-side queries per tick.  A tick
# concatenates the worlds in order: object ids and queries are global, world
# w owning ids [obj_base[w], obj_base[w+1]) and queries [q_base[w],
# q_base[w+1]).
# ----------------------------------------------------------------------------
@dataclass
class BatchedTick:
    ids: np.ndarray
    xy: np.ndarray
    rects: np.ndarray
    obj_base: np.ndarray     # u32[W+1]
    q_base: np.ndarray       # u32[W+1]


class BatchedWorlds:
    def __init__(self, n_worlds: int = 256, n_lo: int = 1000, n_hi: int = 262_144, q_frac: float = 0.1,
                 side: float = 0.003, step: float = 0.0005, seed: int = 0):
        r_size, r_seed = _rngs(seed, 2)
        sizes = np.exp(r_size.uniform(np.log(n_lo), np.log(n_hi), n_worlds)).astype(np.int64)
        seeds = r_seed.integers(0, 2 ** 31, size=n_worlds)
        self.worlds = []
        for w in range(n_worlds):
            n = int(sizes[w])
            q = max(1, int(n * q_frac))
            if w % 2 == 0:
                self.worlds.append(UniformWalk(n=n, q=q, side=side, step=step, seed=int(seeds[w])))
            else:
                self.worlds.append(HotspotWalk(n=n, q=q, hotspots=8, sigma_lo=0.01, sigma_hi=0.01, side_lo=side,
                                               side_hi=side, step=step, seed=int(seeds[w])))
        self.obj_base = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint32)
        self.n = int(self.obj_base[-1])

    def next_tick(self) -> BatchedTick:
        ticks = [w.next_tick() for w in self.worlds]
        q_base = np.concatenate([[0], np.cumsum([t.rects.shape[0] for t in ticks])]).astype(np.uint32)
        return BatchedTick(np.arange(self.n, dtype=np.uint32), np.concatenate([t.xy for t in ticks]),
                           np.concatenate([t.rects for t in ticks]), self.obj_base.copy(), q_base)


def hotspot_small(seed: int = 0, n: int = 200_000, q: int = 20_000) -> HotspotWalk:
    """A reduced hotspot world with the same recipe (for parity tests)."""
    return HotspotWalk(n=n, q=q, seed=seed)
