"""Host logic of the served-stream scheduler (batching by arrival time,
admission of a prefix, queueing of the rest, latency accounting of Def. 2-3)
with a fake clock and a fake backend: no GPU."""
import numpy as np
import pytest

from paper_1411_3212_gb300.serve import TickServer


class FakeClock:
    def __init__(self):
        self.t = 100.0

    def __call__(self):
        return self.t

    def sleep(self, s):
        self.t += s


class FakeBackend:
    """Admits at most `cap` queries per batch; each answer takes `proc` s."""

    def __init__(self, clock, cap, proc):
        self.clock, self.cap, self.proc = clock, cap, proc
        self.calls, self.ticks = [], []

    def start(self, t0):
        self.t0 = t0

    def begin_tick(self, k):
        self.ticks.append(k)

    def answer(self, lo, hi):
        self.calls.append((lo, hi))
        adm = min(self.cap, hi - lo)
        self.clock.t += self.proc
        return adm, 2 * adm, self.clock.t - self.t0

    def finish(self, token):
        return token


def test_batches_follow_arrivals_and_ticks():
    clk = FakeClock()
    be = FakeBackend(clk, cap=100, proc=0.001)
    dt = 0.010
    arrivals = np.array([0.001, 0.004, 0.0099, 0.010, 0.015, 0.031, 0.039])
    rep = TickServer(be, dt, clock=clk, sleep=clk.sleep).run(arrivals, n_ticks=4)
    # tick k answers the queries that arrived in [0, (k+1) dt): [0,3), [3,5), none, [5,7)
    assert be.calls == [(0, 3), (3, 5), (5, 7)]
    assert rep["answered"] == 7 and rep["deferred_batches"] == 0
    # a batch starts at the end of its tick and takes 1 ms: t_f = (k+1) dt + 1 ms
    tf = np.array([0.011] * 3 + [0.021] * 2 + [0.041] * 2)
    np.testing.assert_allclose(rep["query_latency_ms"]["max"], 1e3 * np.max(tf - arrivals), rtol=1e-9)
    per = [t for t in rep["per_tick"] if t["queries"]]
    np.testing.assert_allclose([t["tick_latency"] for t in per], [0.011 - 0.001, 0.021 - 0.010, 0.041 - 0.031])
    assert rep["beta_queries_per_s"] == pytest.approx(7 / 0.003)


def test_admission_defers_the_rest_to_later_ticks():
    clk = FakeClock()
    be = FakeBackend(clk, cap=2, proc=0.0005)
    arrivals = np.linspace(0.0, 0.0095, 5)                 # 5 queries in tick 0
    rep = TickServer(be, 0.010, clock=clk, sleep=clk.sleep).run(arrivals, n_ticks=1, drain_ticks=5)
    assert be.calls == [(0, 5), (2, 5), (4, 5)]              # prefixes of 2, then the queue
    assert rep["answered"] == 5 and rep["deferred_batches"] == 2
    lat = rep["query_latency_ms"]
    assert lat["max"] > 20.0                                 # the last query waited two more ticks
    # queueing + processing = latency for every query (Def. 2)
    assert rep["queueing_ms_p50"] <= lat["p50"]


def test_overrun_ticks_start_late_and_queue_grows():
    clk = FakeClock()
    be = FakeBackend(clk, cap=1000, proc=0.025)              # processing longer than dt
    arrivals = np.arange(40) * 0.001
    rep = TickServer(be, 0.010, clock=clk, sleep=clk.sleep).run(arrivals, n_ticks=4)
    starts = [t["processing"] for t in rep["per_tick"] if t["queries"]]
    assert all(p == pytest.approx(0.025) for p in starts)
    # Lemma 1 violated: tick latency exceeds dt + processing for the late ticks
    lats = [t["tick_latency"] for t in rep["per_tick"] if t["queries"]]
    assert lats[-1] > 0.010 + 0.025


def test_query_too_large_alone_is_rejected_not_stalling():
    clk = FakeClock()

    class Picky(FakeBackend):
        def answer(self, lo, hi):
            self.calls.append((lo, hi))
            adm = 0 if lo == 1 else min(self.cap, hi - lo)     # query 1 never fits
            if lo == 0:
                adm = 1
            self.clock.t += self.proc
            return adm, adm, self.clock.t - self.t0

    be = Picky(clk, cap=10, proc=0.001)
    rep = TickServer(be, 0.010, clock=clk, sleep=clk.sleep).run(np.array([0.001, 0.002, 0.003]), n_ticks=1,
                                                                 drain_ticks=5)
    assert rep["rejected"] == [1]
    assert rep["answered"] == 2
    assert be.calls == [(0, 3), (1, 3), (2, 3)]


def test_max_batch_bounds_the_offered_queue():
    clk = FakeClock()
    be = FakeBackend(clk, cap=100, proc=0.001)
    arrivals = np.arange(10) * 0.0009                       # 10 queries in tick 0
    rep = TickServer(be, 0.010, clock=clk, sleep=clk.sleep, max_batch=4).run(arrivals, n_ticks=1, drain_ticks=5)
    assert be.calls == [(0, 4), (4, 8), (8, 10)]
    assert rep["answered"] == 10 and rep["queued_at_end"] == 0

