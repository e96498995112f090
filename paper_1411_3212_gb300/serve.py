"""Served stream: queries that arrive continuously, answered in ticks of fixed
duration (Sec. 2.2 batch processing; Sec. 2.4 latency, Def. 2-3, Lemmas 1-2).

The queries that arrive during tick k are answered in one batch at the start
of tick k + 1.  Each batch goes through the C ABI's admission entry point
(`mqr_tick_admit`): the exact counts of the two-pass scheme bound the batch's
output before anything is written, and a batch whose output would exceed the
per-tick output memory is answered for its longest fitting prefix; the rest
stays queued for the next tick (a query whose output alone exceeds the
memory is rejected, so the queue cannot stall).  The GPU backend
double-buffers the output and copies each tick's (covering-compressed)
result to pinned host memory on a second stream, so the copy of tick k
overlaps the work of tick k + 1.

Latency accounting (Def. 2): a query issued at t, whose batch starts at t'
and whose result is complete at t_f, has latency t_f - t = queueing (t' - t)
+ processing (t_f - t').  Tick latency (Def. 3) is the maximum over the
tick's queries.  beta is the number of answered queries per second of
processing (Lemma 2: the latency budget lambda holds when
beta >= Q_max / (lambda - dt)).

This module is scheduling only: every step of the join runs in the CUDA
kernels behind the C ABI.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np


@dataclass
class TickRecord:
    k: int               # tick index
    lo: int              # first query of the batch (global arrival order)
    hi: int              # one past the last query that had arrived
    admitted: int        # queries answered (a prefix of [lo, hi))
    out_count: int       # output elements written
    t_start: float       # batch start, s since the stream began
    done: object         # backend token resolved to t_f after the run


class TickServer:
    """Real-time tick scheduler over a backend with three calls:
    begin_tick(k) applies the tick's position updates, answer(lo, hi) answers
    the queries lo..hi-1 (in arrival order) and returns (admitted, out_count,
    token), finish(token) returns the completion time t_f of that answer in
    seconds since start(t0) was called."""

    def __init__(self, backend, dt: float, clock=time.perf_counter, sleep=time.sleep, max_batch=None):
        self.backend = backend
        self.dt = float(dt)
        self.clock = clock
        self.sleep = sleep
        self.max_batch = max_batch      # queries offered per tick (None: the whole queue)

    def run(self, arrivals: np.ndarray, n_ticks: int, drain_ticks: int = 0) -> dict:
        """arrivals: ascending arrival times (s since the stream began) of all
        queries, in the order the backend knows them.  Runs n_ticks ticks of
        arrivals plus up to drain_ticks ticks that only answer queued queries."""
        arrivals = np.asarray(arrivals, np.float64)
        nq = arrivals.shape[0]
        records, rejected = [], []
        first = 0
        t0 = self.clock()
        self.backend.start(t0)
        for k in range(n_ticks + drain_ticks):
            if k >= n_ticks and first >= nq:
                break
            t_tick = (k + 1) * self.dt
            wait = t0 + t_tick - self.clock()
            if wait > 0:
                self.sleep(wait)
            hi = int(np.searchsorted(arrivals, t_tick, side="left")) if k < n_ticks else nq
            if self.max_batch is not None:
                hi = min(hi, first + int(self.max_batch))   # bounds the counting work of a backlog
            self.backend.begin_tick(k)
            t_start = self.clock() - t0
            if hi > first:
                admitted, cnt, token = self.backend.answer(first, hi)
            else:
                admitted, cnt, token = 0, 0, None
            records.append(TickRecord(k, first, hi, admitted, cnt, t_start, token))
            first += admitted
            if hi > first and admitted == 0:
                rejected.append(first)          # its output alone exceeds the tick's memory
                first += 1
        return self._report(arrivals, records, first - len(rejected), rejected)

    def _report(self, arrivals, records, answered, rejected) -> dict:
        lat = np.full(arrivals.shape[0], np.nan)
        queue = np.full(arrivals.shape[0], np.nan)
        tick_lat, proc, per_tick = [], [], []
        for r in records:
            if r.admitted == 0:
                per_tick.append(dict(k=r.k, queries=0, deferred=r.hi - r.lo))
                continue
            t_f = self.backend.finish(r.done)
            a = arrivals[r.lo:r.lo + r.admitted]
            lat[r.lo:r.lo + r.admitted] = t_f - a
            queue[r.lo:r.lo + r.admitted] = r.t_start - a
            tick_lat.append(float(t_f - a.min()))                 # Def. 3
            proc.append(float(t_f - r.t_start))
            per_tick.append(dict(k=r.k, queries=r.admitted, deferred=r.hi - r.lo - r.admitted,
                                 out_elems=r.out_count, tick_latency=tick_lat[-1], processing=proc[-1]))
        done = ~np.isnan(lat)
        pct = lambda x, p: float(np.percentile(x, p)) if len(x) else None
        return {
            "queries": int(arrivals.shape[0]), "answered": int(answered), "rejected": rejected,
            "ticks": len(records), "dt_ms": 1000.0 * self.dt,
            "deferred_batches": int(sum(1 for r in records if r.admitted < r.hi - r.lo)),
            "queued_at_end": int(arrivals.shape[0] - answered - len(rejected)),
            "tick_latency_ms": {"p50": 1e3 * pct(tick_lat, 50), "p99": 1e3 * pct(tick_lat, 99),
                                "max": 1e3 * max(tick_lat)} if tick_lat else None,
            "query_latency_ms": {"p50": 1e3 * pct(lat[done], 50), "p99": 1e3 * pct(lat[done], 99),
                                 "max": 1e3 * float(lat[done].max())} if done.any() else None,
            "queueing_ms_p50": 1e3 * pct(queue[done], 50) if done.any() else None,
            "processing_ms": {"p50": 1e3 * pct(proc, 50), "p99": 1e3 * pct(proc, 99)} if proc else None,
            "beta_queries_per_s": float(answered / sum(proc)) if proc and sum(proc) > 0 else None,
            "per_tick": per_tick,
        }


class GpuBackend:
    """The served stream on one GPU through the C ABI.  updates: list of
    (ids_dev, xy_dev) position sets, tick k applies set k mod len; rects_dev:
    float32[Q_total, 4] device, all queries in arrival order; budget_bytes:
    output memory per tick (each of two buffers).  copy_out: copy every
    tick's output to pinned host memory on a second stream; t_f is then the
    end of that copy, else the end of the tick's kernels.  overlap=False is
    the plain form: each tick's copy is waited for before the next tick starts
    (no overlap of a tick's copy with the next tick's work)."""

    def __init__(self, idx, updates, rects_dev, kind="runs", budget_bytes=1 << 30, copy_out=True, overlap=True):
        import torch
        from . import mqr
        self.torch, self.mqr = torch, mqr
        self.idx, self.updates, self.rects = idx, updates, rects_dev
        self.kind = mqr.KINDS[kind]
        self.elem = 4 if self.kind == mqr.MQR_OUT_CSR else 8
        self.budget = int(budget_bytes) // 16 * 16
        dev = rects_dev.device
        self.out = [torch.empty(self.budget // 4, dtype=torch.int32, device=dev) for _ in range(2)]
        self.copy_out = copy_out
        self.host = [torch.empty(self.budget // 4, dtype=torch.int32).pin_memory() for _ in range(2)] \
            if copy_out else None
        self.copy_stream = torch.cuda.Stream(device=dev)
        self.buf_free = [None, None]
        self.n_answers = 0
        self.ref = None
        self.overlap = overlap

    def start(self, t0):
        torch = self.torch
        torch.cuda.synchronize()
        self.ref = torch.cuda.Event(enable_timing=True)
        self.ref.record(self.copy_stream)
        self.ref.synchronize()
        self.t_ref = time.perf_counter() - t0          # ref's time on the stream clock

    def begin_tick(self, k):
        ids, xy = self.updates[k % len(self.updates)]
        self.idx.apply_updates(ids, xy)

    def answer(self, lo, hi):
        torch, mqr = self.torch, self.mqr
        b = self.n_answers & 1
        self.n_answers += 1
        if self.buf_free[b] is not None:
            self.buf_free[b].synchronize()               # the copy that last read this buffer is done
        admitted, cnt = mqr.mqr_tick_admit(self.idx.ctx, self.rects[lo:hi], hi - lo, self.kind, self.out[b],
                                           self.budget)
        ev = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(self.copy_stream):
            if self.copy_out and cnt:
                n = cnt * self.elem // 4
                self.host[b][:n].copy_(self.out[b][:n], non_blocking=True)
            ev.record(self.copy_stream)
        self.buf_free[b] = ev
        if not self.overlap:
            ev.synchronize()                             # plain: the copy ends before anything else starts
        return admitted, cnt, ev

    def finish(self, ev):
        ev.synchronize()
        return self.t_ref + self.ref.elapsed_time(ev) / 1000.0


class SlotBackend(GpuBackend):
    """Continuous batching on join slots (mqr_slot_*): every tick takes one
    snapshot of the object state (mqr_snapshot) after the tick's updates, and
    the offered queries are split into n_slots consecutive parts answered by
    the slots concurrently, each on its own stream, so that the parts' kernels
    overlap on the device; each part is admitted against its slot's share of
    the output memory (budget_bytes / n_slots) and copied to pinned host
    memory as soon as its slot ends, while the other slots still run.  The
    batch's answered queries are the longest prefix of fully answered parts
    plus the admitted prefix of the first cut part (a part after a cut one is
    answered again in a later tick, and its answer here is not reported)."""

    def __init__(self, idx, updates, rects_dev, kind="runs", budget_bytes=1 << 30, copy_out=True, n_slots=2):
        import torch
        from . import mqr
        self.torch, self.mqr = torch, mqr
        self.idx, self.updates, self.rects = idx, updates, rects_dev
        self.kind = mqr.KINDS[kind]
        self.elem = 4 if self.kind == mqr.MQR_OUT_CSR else 8
        self.n_slots = int(n_slots)
        self.budget = int(budget_bytes) // self.n_slots // 16 * 16          # per slot
        dev = rects_dev.device
        self.slots = [idx.slot() for _ in range(self.n_slots)]
        self.out = [torch.empty(self.budget // 4, dtype=torch.int32, device=dev) for _ in range(self.n_slots)]
        self.copy_out = copy_out
        self.host = [torch.empty(self.budget // 4, dtype=torch.int32).pin_memory() for _ in range(self.n_slots)] \
            if copy_out else None
        self.copy_stream = torch.cuda.Stream(device=dev)
        self.buf_free = [None] * self.n_slots
        self.last_parts = []        # (lo, admitted, out_count, slot) of the last answer, for checks
        self.ref = None

    def begin_tick(self, k):
        ids, xy = self.updates[k % len(self.updates)]
        self.idx.apply_updates(ids, xy)
        self.idx.snapshot()

    def answer(self, lo, hi):
        torch, mqr = self.torch, self.mqr
        n = hi - lo
        cuts = [lo + (n * i) // self.n_slots for i in range(self.n_slots + 1)]
        begun = []
        for i in range(self.n_slots):
            a, b = cuts[i], cuts[i + 1]
            if b <= a:
                continue
            if self.buf_free[i] is not None:
                self.buf_free[i].synchronize()           # the copy that last read this slot's output is done
            self.slots[i].begin(self.rects[a:b], self.kind, self.out[i], self.budget)
            begun.append((i, a, b))
        admitted, out_count, last_ev, cut = 0, 0, None, False
        self.last_parts = []
        for i, a, b in begun:
            adm, cnt = self.slots[i].end()               # every begun join is ended
            if cut:
                continue                                  # after a cut part: answered again later
            ev = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(self.copy_stream):
                if self.copy_out and cnt:
                    m = cnt * self.elem // 4
                    self.host[i][:m].copy_(self.out[i][:m], non_blocking=True)
                ev.record(self.copy_stream)
            self.buf_free[i] = ev
            self.last_parts.append((a, adm, cnt, i))
            admitted += adm
            out_count += cnt
            cut = adm < b - a
            last_ev = ev
        return admitted, out_count, last_ev

    def close(self):
        for sl in self.slots:
            sl.close()


class PlainBackend(GpuBackend):
    """The plain fixed-capacity GPU quadtree: every tick answers the whole
    offered batch with one blocking mqr_tick (device output buffer grown when
    a batch needs more), then copies the result to pinned host memory and
    waits for it before the next tick; no admission, no overlap."""

    def __init__(self, idx, updates, rects_dev, kind="runs", copy_out=True):
        import torch
        from . import mqr
        self.torch, self.mqr = torch, mqr
        self.idx, self.updates, self.rects = idx, updates, rects_dev
        self.kind = mqr.KINDS[kind]
        self.elem = 4 if self.kind == mqr.MQR_OUT_CSR else 8
        dev = rects_dev.device
        self.out = torch.empty(1 << 20, dtype=torch.int32, device=dev)
        self.copy_out = copy_out
        self.host = torch.empty(1 << 20, dtype=torch.int32).pin_memory() if copy_out else None
        self.copy_stream = torch.cuda.current_stream(dev)
        self.ref = None

    def answer(self, lo, hi):
        torch, mqr = self.torch, self.mqr
        st, cnt = mqr.mqr_tick(self.idx.ctx, self.rects[lo:hi], hi - lo, self.kind, self.out, self.out.numel() * 4)
        if st == mqr.MQR_ERR_CAPACITY:
            self.out = torch.empty(int(cnt * self.elem * 1.25) // 4 + 1024, dtype=torch.int32,
                                   device=self.rects.device)
            st, cnt = mqr.mqr_tick(self.idx.ctx, self.rects[lo:hi], hi - lo, self.kind, self.out,
                                   self.out.numel() * 4)
        mqr._check(st)
        m = cnt * self.elem // 4
        if self.copy_out and m:
            if self.host.numel() < m:
                self.host = torch.empty(int(m * 1.25) + 1024, dtype=torch.int32).pin_memory()
            self.host[:m].copy_(self.out[:m], non_blocking=True)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(self.copy_stream)
        ev.synchronize()
        return hi - lo, cnt, ev
