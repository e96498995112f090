"""Autotuning of the leaf capacity and of the work-item kernels' launch shapes.

The quadtree's split threshold (th_quad, Alg. 1; the paper fixes it per
experiment) trades fewer, larger leaves (more containment tests, Eq. of the
filtering complexity) against more subqueries and candidates.  Every
capacity gives the same results (the index never changes an answer), so the
choice only moves time: this tunes it on the caller's own ticks by timing a
few ticks per candidate capacity with CUDA events and keeping the fastest.
Scheduling only: the ticks themselves run in the kernels behind the C ABI.
"""
from __future__ import annotations


def tune_leaf_cap(make_index, ticks, caps=(32, 64, 128, 256, 512), kind="pairs", reps=2):
    """make_index(cap) -> mqr.Index; ticks: list of (ids_dev, xy_dev,
    rects_dev) in the caller's order.  Each capacity answers every tick once
    untimed, then `reps` more times timed.  Returns (best_cap, table) with
    table[cap] = {"ms_per_tick", "results"}; results must agree across caps."""
    import torch
    table = {}
    for cap in caps:
        idx = make_index(cap)
        try:
            for ids, xy, rects in ticks:                   # warm-up: buffer growth
                idx.apply_updates(ids, xy)
                idx.tick(rects, kind=kind)
            torch.cuda.synchronize()
            start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            results = 0
            start.record()
            for _ in range(reps):
                for ids, xy, rects in ticks:
                    idx.apply_updates(ids, xy)
                    idx.tick(rects, kind=kind)
                    results += idx.stats()["n_results"]
            end.record()
            end.synchronize()
            table[cap] = {"ms_per_tick": start.elapsed_time(end) / (reps * len(ticks)),
                          "results": results // reps}
        finally:
            idx.close()
    best = min(table, key=lambda c: table[c]["ms_per_tick"])
    return best, table


def _time_ticks(idx, ticks, kind, reps):
    import torch
    for ids, xy, rects in ticks:                       # warm-up: buffer growth, graph capture
        idx.apply_updates(ids, xy)
        idx.tick(rects, kind=kind)
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = 0
    start.record()
    for _ in range(reps):
        for ids, xy, rects in ticks:
            idx.apply_updates(ids, xy)
            idx.tick(rects, kind=kind)
            results += idx.stats()["n_results"]
    end.record()
    end.synchronize()
    return start.elapsed_time(end) / (reps * len(ticks)), results // reps


def tune_launch_config(idx, ticks, options=(2, 4, 8, 16), kind="pairs", reps=2, timer=None):
    """Blocks per SM of the candidate pass, the leaf-list pass, the filter and
    the emit (mqr_set_launch_config), by coordinate descent: each kernel in turn
    takes the option with the smallest tick time, the others held.  Block
    sizes are fixed per kernel (register budgets); only the grids move, and
    results must not.  timer(idx, ticks, kind, reps) -> (ms per tick,
    results) defaults to CUDA-event timing of the ticks.  Returns (best dict,
    table of (config, ms, results))."""
    from .mqr import LAUNCH_KERNELS
    timer = timer or _time_ticks
    best = {k: 8 for k in LAUNCH_KERNELS}
    table = []
    ms0, res0 = None, None
    for k in LAUNCH_KERNELS:
        timings = {}
        for v in options:
            cfg = dict(best, **{k: v})
            idx.set_launch_config(**cfg)
            ms, res = timer(idx, ticks, kind, reps)
            if res0 is None:
                res0 = res
            if res != res0:
                raise RuntimeError("launch shapes changed the results")
            timings[v] = ms
            table.append((cfg, ms, res))
        best[k] = min(timings, key=timings.get)
    idx.set_launch_config(**best)
    return best, table


def tune_world_caps(idx, ticks, world_bits, classes, caps=(32, 64, 128, 256, 512), kind="pairs", reps=2,
                    timer=None, start=128, sweeps=1):
    """Per-world leaf capacities of batched worlds.  World w's quadtree is
    the node of depth world_bits whose Morton prefix is w (mqr_set_worlds),
    so the per-region capacities of mqr_set_region_caps at region_bits =
    world_bits give every world its own th_quad.  classes[w] labels world w
    (worlds of one label share a capacity); coordinate descent over the
    labels: each label in turn takes the capacity in `caps` with the smallest
    tick time, the others held (`sweeps` passes).  Results must not change.
    timer(idx, ticks, kind, reps) -> (ms per tick, results) as for
    tune_launch_config.  Returns (best capacity per label, the capacity of
    every region, table of (assignment, ms, results))."""
    import numpy as np
    timer = timer or _time_ticks
    classes = list(classes)
    labels = sorted(set(classes))
    n_regions = 4 ** world_bits
    if len(classes) > n_regions:
        raise ValueError("more worlds than regions of depth world_bits")

    def region_vector(assign):
        v = np.full(n_regions, start, np.uint32)
        for w, c in enumerate(classes):
            v[w] = assign[c]
        return v

    best = {c: start for c in labels}
    table, res0 = [], None
    for _ in range(sweeps):
        for c in labels:
            timings = {}
            for cap in caps:
                assign = dict(best, **{c: cap})
                idx.set_region_caps(world_bits, region_vector(assign))
                ms, res = timer(idx, ticks, kind, reps)
                if res0 is None:
                    res0 = res
                if res != res0:
                    raise RuntimeError("per-world capacities changed the results")
                timings[cap] = ms
                table.append((assign, ms, res))
            best[c] = min(timings, key=timings.get)
    vec = region_vector(best)
    idx.set_region_caps(world_bits, vec)
    return best, vec, table
