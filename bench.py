"""Benchmark: repeated range queries over moving objects on GB300.

One step = one tick of the whole hot path: the tick's position updates of
every object (mqr_apply_updates) followed by the spatial join of the tick's
queries through the PR-quadtree (mqr_tick), pair-list output; the tick's
kernels are replayed as one captured CUDA graph (mqr_set_graph; --no-graph:
plain launches), with CUDA events around the dominant phase as event nodes
of the graph.

Default workload (N=1): 4,000,000 objects, 90% in 64 Gaussian hotspots (sigma
log-uniform 0.002-0.02) and 10% uniform, random walk sigma 0.0005 with
hotspot drift 0.001/tick, 400,000 square queries per tick of side
log-uniform 0.0005-0.005 centred on objects, leaf_cap 128, pairs output.

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle
instead (bounded samples of the same workload).  Multi-GPU (torchrun): every
rank runs an independent replica world (weak scaling, no collective on the
data path); a barrier brackets the timed region and the max over ranks is
reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "emit_kernel_traffic.txt")
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0

WORKLOADS = {
    "hotspot4m": dict(kind="hotspot", n=4_000_000, q=400_000, cap=128,
                      desc="hotspot-4M: 4,000,000 objects (90% in 64 Gaussian hotspots, sigma log-uniform "
                           "0.002-0.02; 10% uniform), random walk sigma 0.0005, hotspot drift 0.001/tick, "
                           "400,000 square queries/tick of side log-uniform 0.0005-0.005 centred on objects, "
                           "leaf_cap 128 (fixed), pair-list output"),
    "hotspot2m": dict(kind="hotspot", n=2_000_000, q=200_000, cap=128,
                      desc="hotspot-2M: the hotspot-4M recipe at 2,000,000 objects and 200,000 queries/tick "
                           "(profiling size)"),
    "hotspot1m": dict(kind="hotspot", n=1_000_000, q=100_000, cap=128,
                      desc="hotspot-1M: the hotspot-4M recipe at 1,000,000 objects and 100,000 queries/tick "
                           "(profiling size)"),
    "uniform1m": dict(kind="uniform", n=1_000_000, q=100_000, cap=128,
                      desc="uniform-1M: 1,000,000 uniform objects, random walk sigma 0.0005, 100,000 queries/tick "
                           "of side 0.002 centred on objects, leaf_cap 128, pair-list output"),
    "mixed4m": dict(kind="mixed", n=4_000_000, q=310_000, cap=128,
                    desc="mixed-4M: 4,000,000 objects, 75% in 32 Gaussian hotspots (sigma 0.01) in the left "
                         "half queried by 300,000 squares of side log-uniform 0.0003-0.001, 25% uniform in the "
                         "right half queried by 10,000 squares of side log-uniform 0.01-0.04; random walk "
                         "sigma 0.0005 inside each half; leaf_cap 128, pair-list output"),
    "alternating4m": dict(kind="alternating", n=4_000_000, q=400_000, cap=128,
                          desc="alternating-4M: the hotspot-4M objects; even ticks 400,000 squares of side "
                               "log-uniform 0.0002-0.001, odd ticks 4,000 squares of side log-uniform 0.005-0.02 "
                               "(two query regimes that prefer different index configurations); leaf_cap 128, "
                               "pair-list output"),
    "uniform16k": dict(kind="small", n=16384, q=1024, cap=64,
                       desc="uniform-16K: 16,384 uniform objects, 1,024 queries of side 0.01, leaf_cap 64"),
    "batched256": dict(kind="batched", n=0, q=0, cap=128,
                       desc="batched-256: 256 independent worlds in one index, sizes log-uniform 1,000-262,144 "
                            "objects (12.3M in all), half uniform and half 8-hotspot (sigma 0.01) random walks, "
                            "each issuing sizes/10 queries of side 0.003 per tick (1.23M in all), leaf_cap 128, "
                            "pair-list output"),
}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ----------------------------------------------------------------------------
# workload
# ----------------------------------------------------------------------------
def make_world(name, seed):
    from paper_1411_3212_gb300 import workloads
    w = WORKLOADS[name]
    if w["kind"] == "hotspot":
        return workloads.HotspotWalk(n=w["n"], q=w["q"], seed=seed)
    if w["kind"] == "uniform":
        return workloads.UniformWalk(n=w["n"], q=w["q"], seed=seed)
    if w["kind"] == "batched":
        return workloads.BatchedWorlds(n_worlds=256, seed=seed)
    if w["kind"] == "mixed":
        return workloads.MixedDensity(n=w["n"], seed=seed)
    if w["kind"] == "alternating":
        return workloads.AlternatingQueries(n=w["n"], seed=seed)

    class Small:
        def __init__(self):
            self.t = 0

        def next_tick(self):
            self.t += 1
            return workloads.uniform_small(seed=seed + self.t)
    return Small()


def gen_ticks(name, seed, count):
    world = make_world(name, seed)
    return [world.next_tick() for _ in range(count)]


def replica_ticks(name, rank, count):
    """The ticks of rank `rank`'s replica world: every rank answers an
    independent world of the same recipe (its own seed), so the job's
    throughput is the sum over ranks and no data crosses ranks."""
    return gen_ticks(name, 1000 * rank, count)


# ----------------------------------------------------------------------------
# algorithmic bytes per phase (the data the method must move)
# ----------------------------------------------------------------------------
def phase_bytes(s, n_updates, nmax, n_out=None, fp=None, elem=8):
    """Algorithmic bytes of each phase of one tick: what the method must move
    at least once (inputs read, outputs written), from the tick's counters
    (mqr_get_stats), its output size n_out (elements of elem bytes) and its
    leaf footprint fp (mqr_result_footprint).  Re-reads that hit or miss L2 are not counted."""
    N, Q = s["n_objects"], s["n_queries"]
    R, W = s["n_results"], s["n_bitmap_words"]
    S, SI = s["n_sub_intersecting"] + s["n_covering_runs"], s["n_sub_intersecting"]
    out_elems = R if n_out is None else n_out
    fp = fp or {}
    tested = fp.get("tested_leaf_objects", s["n_filter_loads"])
    productive = fp.get("result_leaf_objects", 0)
    return {
        "updates": 20 * n_updates,                       # read id+xy, write xy
        "keys": 16 * nmax,                               # read xy, write key
        "sort": 3 * 16 * nmax + 32 * nmax,               # 3 x (read+write 8B), last: read 8B + gather 8B + write 16B
        "leaves": 4 * N + 12 * s["n_leaves"],
        "query_blocks": 32 * Q + 24 * s["n_pairs"],     # rects in; cells, offsets, pair records out
        "candidates": 8 * s["n_candidates"] + 16 * S,   # leaf intervals in; subquery records out
        "group": 16 * s["n_leaves"] + 4 * S + 8 * SI,
        # each tested leaf's positions once, rect + query index and count per
        # intersecting subquery, the bitmap words written
        "filter": 8 * tested + 24 * SI + 4 * W,
        "result_scan": 16 * S,                           # count + leaf word in, 8-byte offset out
        # output written, bitmap words read, record metadata (query, leaf,
        # length, 8-byte offset), the ids of every leaf with results once
        "emit": elem * out_elems + 4 * W + 20 * S + 4 * productive,
    }


PHASE_FORMULA = {
    "emit": "out_elem_bytes*out_elems + 4*bitmap_words + 20*records + 4*result_leaf_objects",
    "filter": "8*objects of the tested leaves + 24*intersecting subqueries + 4*bitmap_words",
    "sort": "80*max_objects (3 passes x 16 B + last pass 32 B per key)",
}


def guarded(name, fn, *a, **kw):
    """Run an optional leg of the bench; its failure is reported in the line."""
    try:
        return fn(*a, **kw)
    except Exception as e:                  # noqa: BLE001 - recorded, not swallowed
        log("%s leg failed: %r" % (name, e))
        return {"error": "%s: %s" % (type(e).__name__, e)}


KERNEL_SOURCES = {"emit_kernel": "k_join.cu"}


def source_hash(kernel="emit_kernel"):
    """Hash of a kernel's source file and the shared header (the host code
    and the other kernels' files do not change what the kernel moves)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1411_3212_gb300", "csrc")
    for f in (KERNEL_SOURCES[kernel], "mqr_internal.cuh"):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def read_peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def read_traffic(kernel, results_per_launch):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary (a
    smaller case of the same workload recipe), scaled by the results the
    timed launches processed, if the CUDA sources have not changed since it
    was taken (else None)."""
    try:
        kv = {}
        with open(TRAFFIC_FILE) as f:
            for line in f:
                line = line.strip()
                if line and not line.startswith("#") and "=" in line:
                    k, v = line.split("=", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel") == kernel and kernel in KERNEL_SOURCES and kv.get("source_hash") == source_hash(kernel):
            return float(kv["dram_bytes_per_launch"]) * results_per_launch / float(kv["results"])
    except Exception:
        pass
    return None


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "25"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------
# distributed helpers (replicas only)
# ----------------------------------------------------------------------------
def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = os.environ.get("MQR_DIST_BACKEND") or ("nccl" if torch.cuda.is_available() else "gloo")
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        return dist, rank, world, local
    return None, rank, world, local


def barrier(dist, dev):
    import torch
    if dist is not None:
        dist.barrier()
    if dev is not None:
        torch.cuda.synchronize()


def reduce_max(dist, x, dev):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=dev if dev is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, on a bounded sample
# ----------------------------------------------------------------------------
def oracle_join_timed(st, rects, sample_q, seed, cell=0.002):
    """One oracle step: a full uniform-grid build over every present object
    plus the join of a random sample of sample_q of the tick's queries (all of
    them if sample_q >= their number).  Returns (queries answered, seconds
    spent) -- measured, nothing extrapolated."""
    import oracle
    q = rects.shape[0]
    if sample_q >= q:
        pick = rects
    else:
        rng = np.random.default_rng(seed)
        pick = rects[np.sort(rng.choice(q, size=sample_q, replace=False))]
    t0 = time.perf_counter()
    oracle.join_grid(st, pick, cell_side=cell)
    return pick.shape[0], time.perf_counter() - t0


def cpu_baseline(ticks, name, nmax, sample_q):
    import oracle
    st = oracle.State(nmax)
    for t in ticks:
        st.apply_updates(t.ids, t.xy)
    t = ticks[-1]
    nq, secs = oracle_join_timed(st, t.rects, sample_q, seed=1234)
    return {"value": nq / secs, "unit": "queries/s", "cores": 1, "kind": "oracle",
            "sample": "one tick of %s (the last generated): single-threaded C uniform-grid join (cell 0.002), a "
                      "full grid build over all %d objects plus %d of the tick's %d queries%s, timed as a whole: "
                      "%.1f s of CPU work" % (name, nmax, nq, t.rects.shape[0],
                                               "" if nq == t.rects.shape[0] else " (random sample)", secs)}


def run_reference(args, name):
    """--impl reference: the CPU oracle on bounded samples of the workload.
    Each step applies the tick's updates to the oracle state, then builds the
    uniform grid over every object and joins a random --ref-sample of the
    tick's queries; value = queries answered / time spent, both measured."""
    import oracle
    dist, rank, world, local = dist_setup(args.gpus)
    if rank != 0:
        return
    w = WORKLOADS[name]
    uniq = min(args.steps, args.unique_ticks)
    t_gen = time.perf_counter()
    ticks = gen_ticks(name, 0, args.warmup + uniq)
    log("reference: generated %d ticks in %.1f s" % (len(ticks), time.perf_counter() - t_gen))
    st = oracle.State(w["n"])
    sample_q = args.ref_sample
    for i in range(args.warmup):
        st.apply_updates(ticks[i].ids, ticks[i].xy)
        oracle_join_timed(st, ticks[i].rects, sample_q, seed=i)
    answered, times = 0, []
    t_wall = time.perf_counter()
    for k in range(args.steps):
        i = args.warmup + (k % uniq)
        t0 = time.perf_counter()
        st.apply_updates(ticks[i].ids, ticks[i].xy)
        nq, _ = oracle_join_timed(st, ticks[i].rects, sample_q, seed=1000 + k)
        times.append(time.perf_counter() - t0)
        answered += nq
    wall = time.perf_counter() - t_wall
    value = answered / sum(times)
    ms = 1000.0 * sum(times) / len(times)
    sample = ("per step: the tick's updates of all %d objects applied to the oracle state, a full uniform-grid "
              "build (cell 0.002) and the single-threaded C join of a random %d of the tick's %d queries; each "
              "step timed as a whole (nothing extrapolated)" % (w["n"], min(sample_q, w["q"]), w["q"]))
    line = {"impl": "reference", "metric": "queries/s at 4M skewed objects" if name == "hotspot4m" else "queries/s",
            "value": value, "unit": "queries/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w["desc"], "objects": w["n"], "queries_per_tick": w["q"],
                       "queries_per_step": min(sample_q, w["q"]),
                       "leaf_cap": w["cap"], "parallelism": "replicas"},
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def run_gpu(args, name):
    import torch
    from paper_1411_3212_gb300 import mqr

    dist, rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    w = WORKLOADS[name]
    nmax, Q = w["n"], w["q"]

    t_gen = time.perf_counter()
    uniq = min(args.steps, args.unique_ticks)          # timed steps cycle over these ticks
    ticks = replica_ticks(name, rank, args.warmup + uniq)
    log("rank %d: generated %d ticks in %.1f s" % (rank, len(ticks), time.perf_counter() - t_gen))

    batched = w["kind"] == "batched"
    if batched:                                          # sizes come from the generated worlds
        nmax, Q = int(ticks[0].ids.shape[0]), int(ticks[0].rects.shape[0])
    ids_d = torch.from_numpy(ticks[0].ids.view(np.int32)).to(dev)
    xy_d = [torch.from_numpy(t.xy).to(dev) for t in ticks]
    rect_d = [torch.from_numpy(t.rects).to(dev) for t in ticks]
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.int32, device=dev)

    cap = args.leaf_cap or w["cap"]
    covering = not args.no_covering
    if args.index == "ug":                               # uniform grid of 2^grid_level cells per axis
        idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=1, max_objects=nmax, index_kind=1,
                        grid_level=args.grid_level, covering=covering)
    else:
        idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=cap, max_objects=nmax, covering=covering)
    if batched:
        idx.set_worlds(ticks[0].obj_base)
        idx.set_query_worlds(ticks[0].q_base)
    if args.graph:
        idx.set_graph(True)
    kind = mqr.KINDS[args.kind]
    elem = 8 if kind in (mqr.MQR_OUT_PAIRS, mqr.MQR_OUT_PAIRS_SORTED, mqr.MQR_OUT_RUNS, mqr.MQR_OUT_PAIRS_ATOMIC) else 4
    out = torch.empty(1, dtype=torch.int32, device=dev)
    offs = torch.empty(Q + 1, dtype=torch.int64, device=dev) if args.offsets else None

    def step(i):
        nonlocal out
        idx.apply_updates(ids_d, xy_d[i])
        st, cnt = mqr.mqr_tick(idx.ctx, rect_d[i], Q, kind, out, out.numel() * 4, offs)
        if st == mqr.MQR_ERR_CAPACITY:                  # only during warm-up
            out = torch.empty(int(cnt * elem * 1.3) // 4 + 1024, dtype=torch.int32, device=dev)
            st, cnt = mqr.mqr_tick(idx.ctx, rect_d[i], Q, kind, out, out.numel() * 4, offs)
        mqr._check(st)
        return cnt

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()

    # Per-phase breakdown from untimed calibration ticks with events around
    # every phase; the timed region then records events around the dominant
    # phase only (each event record costs stream time; launches are still
    # counted for every phase).  Phase events would stop the graph replay.
    calib_bytes, dom = {}, "emit"
    idx.set_timing(True)
    with_fp = kind != mqr.MQR_OUT_PAIRS_ATOMIC

    def tick_bytes(cnt):
        fp = idx.footprint() if with_fp else None
        return phase_bytes(idx.stats(), nmax, nmax, cnt, fp, elem), fp

    for k in range(max(args.calib_ticks, 1)):
        flush.zero_()
        cnt = step(args.warmup + (k % uniq))
        for ph, b in tick_bytes(cnt)[0].items():
            calib_bytes[ph] = calib_bytes.get(ph, 0) + b
    calib = idx.timing()
    cand = {p: calib["ms"][p] for p in calib_bytes if calib["launches"].get(p, 0) > 0}
    if cand:
        dom = max(cand, key=cand.get)
    idx.set_timing(True, phases=[dom])
    if args.graph:
        # capture the tick's graph (with the dominant phase's event nodes)
        # before the timed region, then restart the accumulators
        for k in range(2):
            step(args.warmup + (k % uniq))
        idx.set_timing(True, phases=[dom])
    clocks = Clocks(local if world > 1 else 0)
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    bytes_acc = {}
    fp_acc = {}
    results = 0
    # the clock sampler starts under the same tick load about 0.25 s before
    # the timed region (a timed region of 20 ticks lasts ~40 ms, one or two
    # samples); those ticks are untimed and their accumulators are reset
    clocks.start()
    t_pre = time.perf_counter()
    k = 0
    while time.perf_counter() - t_pre < args.clock_lead_s:
        flush.zero_()
        step(args.warmup + (k % uniq))
        k += 1
    idx.set_timing(True, phases=[dom])
    barrier(dist, dev)
    t_wall = time.perf_counter()
    for k in range(args.steps):
        i = args.warmup + (k % uniq)
        flush.zero_()                                   # L2 flush between timed steps
        evs[k][0].record(stream)
        cnt = step(i)
        evs[k][1].record(stream)
        results += idx.stats()["n_results"]
        # the tick's counters and leaf footprint (two small kernels, after the
        # step's end event: outside the timed step)
        tb, fp = tick_bytes(cnt)
        for ph, b in tb.items():
            bytes_acc[ph] = bytes_acc.get(ph, 0) + b
        for key, v in (fp or {}).items():
            fp_acc[key] = fp_acc.get(key, 0) + v
        st_k = idx.stats()
        for key, v in (("out_elems", cnt), ("bitmap_words", st_k["n_bitmap_words"]),
                       ("records", st_k["n_sub_intersecting"] + st_k["n_covering_runs"]),
                       ("results", st_k["n_results"])):
            fp_acc[key] = fp_acc.get(key, 0) + v
    barrier(dist, dev)
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    timing = idx.timing()
    stats = idx.stats()
    idx.set_timing(False)

    total_ms = reduce_max(dist, sum(step_ms), dev)
    mean_ms = total_ms / args.steps
    value = world * Q * args.steps / (total_ms / 1000.0)

    # roofline of the dominant kernel phase, timed live in the timed region
    launches = max(timing["launches"][dom], 1)
    per_launch_ms = timing["ms"][dom] / launches
    per_launch_bytes = bytes_acc[dom] / launches
    peak, peak_kind = read_peaks()
    achieved = per_launch_bytes / (per_launch_ms / 1000.0) / 1e9 if per_launch_ms > 0 else 0.0
    kernel_names = {"emit": "emit_kernel", "filter": "filter_kernel",
                    "sort": "tile_hist_kernel+digit_scan_kernel+onesweep_kernel",
                    "query_blocks": "zmap_kernel+query_blocks_kernel", "candidates": "cand_write_kernel",
                    "group": "leaf_scan_kernel+leaf_lists_kernel",
                    "leaves": "leaves_kernel", "keys": "morton_kernel", "updates": "stamp_kernel+write_winner_kernel",
                    "result_scan": "result_scan_kernel"}
    kname = kernel_names.get(dom, dom)
    traffic = read_traffic(kname, results / max(args.steps, 1))
    traffic_gbs = traffic / (per_launch_ms / 1000.0) / 1e9 if traffic and per_launch_ms > 0 else None
    roofline = {"bound": "hbm", "kernel": kname, "phase": dom,
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": achieved / NOMINAL_HBM_GBS,
                "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind if peak_kind == "measured" else "fallback 6.8 TB/s",
                "traffic": traffic,
                "traffic_from": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one emit launch at hotspot-2M "
                                "(profiles/emit_kernel_traffic.txt), scaled by the timed launches' results"
                                if traffic else None,
                "frac_dram": traffic_gbs / peak if traffic_gbs else None,
                "algorithmic_bytes_per_launch": per_launch_bytes, "launch_ms": per_launch_ms,
                "launches": launches,
                "bytes_formula": PHASE_FORMULA.get(dom),
                # the byte formula's terms averaged over the timed launches:
                # elem * out_elems + 4 * bitmap_words + 20 * records + 4 * result_leaf_objects
                "terms_per_launch": {k: v / launches for k, v in fp_acc.items()} if dom == "emit" else None,
                "out_elem_bytes": elem}
    join = ["filter", "emit"]
    join_ms = sum(calib["ms"][p] for p in join)
    join_bytes = sum(calib_bytes.get(p, 0) for p in join)
    join_gbs = join_bytes / (join_ms / 1000.0) / 1e9 if join_ms > 0 else 0.0
    phases = {p: {"ms_per_tick": calib["ms"][p] / max(calib["ticks"], 1),
                  "launches_per_tick": calib["launches"][p] / max(calib["ticks"], 1),
                  "GB/s": (calib_bytes[p] / (calib["ms"][p] / 1000.0) / 1e9)
                  if p in calib_bytes and calib["ms"][p] > 0 else None}
              for p in mqr.PHASES if calib["launches"][p] > 0}
    gpu_launches = int(sum(timing["launches"].values()))

    # end to end through the host-buffer entry points; the optional legs
    # record their failure in the line instead of losing it
    e2e = e2e_runs = e2e_csr = None
    if not args.no_e2e:
        e2e = guarded("e2e", run_e2e, args, idx, ticks, kind, elem, Q, dev)
        if kind == mqr.MQR_OUT_PAIRS:
            # the same ticks and answers as per-query id lists (CSR: 4-byte ids
            # and Q + 1 offsets), and with covering runs reported compressed
            # (RUNS kind)
            e2e_csr = guarded("e2e_csr", run_e2e, args, idx, ticks, mqr.MQR_OUT_CSR, 4, Q, dev)
            e2e_runs = guarded("e2e_covering_compressed", run_e2e, args, idx, ticks, mqr.MQR_OUT_RUNS, 8, Q, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not batched:
        cpu = guarded("cpu_baseline", cpu_baseline, ticks, name, nmax, args.cpu_sample)

    idx.close()
    if rank != 0:
        return
    srt = sorted(step_ms)
    line = {
        "metric": "queries/s at 4M skewed objects" if name == "hotspot4m" else "queries/s",
        "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["desc"], "objects": nmax, "queries_per_tick": Q,
                   "index": "quadtree" if args.index == "quad" else "uniform grid level %d" % args.grid_level,
                   "leaf_cap": cap,
                   "covering": "on" if covering else "off (every subquery tested)",
                   "output": args.kind, "parallelism": "replicas" if world > 1 else "single-gpu",
                   "l2": "flushed (%d MB write) between timed steps" % args.flush_mb,
                   "launch": "one captured CUDA graph per tick (replayed)" if args.graph else "plain kernel launches",
                   "ticks": "%d distinct generated ticks, cycled over the %d timed steps" % (uniq, args.steps)},
        "tick_latency_ms": {"p50": srt[len(srt) // 2], "p99": srt[min(len(srt) - 1, int(0.99 * len(srt)))],
                            "max": srt[-1]},
        "join_kernels": {"phases": join, "GB/s": join_gbs, "frac_of_peak": join_gbs / peak},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "e2e_csr": e2e_csr,
        "e2e_covering_compressed": e2e_runs,
        "gpu_launches": gpu_launches,
        "launches_between_steps": "per step, after its end event: the L2 flush and the two footprint-statistics "
                                  "kernels of mqr_result_footprint (not in gpu_launches or the step times)",
        "clocks": clk,
        "clocks_window": "nvidia-smi sampled every 25 ms from %.2f s of untimed ticks before the timed region to its "
                         "end" % args.clock_lead_s,
        "phases": phases,
        "phases_from": "%d untimed calibration ticks with events around every phase (the timed region records "
                       "events around the %s phase only)" % (max(args.calib_ticks, 1), dom),
        "stats": stats,
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)


def run_gpu_slots(args, name):
    """--slots S: every step applies the tick's updates, takes one snapshot of
    the state (mqr_snapshot) and answers the tick's queries split into S
    consecutive parts on S join slots concurrently (mqr_slot_begin / _end),
    each slot on its own stream; the step's CUDA events are recorded on the
    context's stream, the end event after the stream has waited for every
    slot.  Same workload, ticks and L2 flush as the plain bench."""
    import torch
    from paper_1411_3212_gb300 import mqr
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = WORKLOADS[name]
    nmax, Q = w["n"], w["q"]
    uniq = min(args.steps, args.unique_ticks)
    ticks = gen_ticks(name, 0, args.warmup + uniq)
    ids_d = torch.from_numpy(ticks[0].ids.view(np.int32)).to(dev)
    xy_d = [torch.from_numpy(t.xy).to(dev) for t in ticks]
    rect_d = [torch.from_numpy(t.rects).to(dev) for t in ticks]
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.int32, device=dev)
    S = args.slots
    cut = [(Q * j) // S for j in range(S + 1)]
    parts = [[r[cut[j]:cut[j + 1]] for j in range(S)] for r in rect_d]
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=args.leaf_cap or w["cap"], max_objects=nmax)
    stream = torch.cuda.current_stream()
    slots = [idx.slot() for _ in range(S)]
    kind = mqr.KINDS[args.kind]
    elem = 4 if kind == mqr.MQR_OUT_CSR else 8
    outs = [torch.empty(1 << 20, dtype=torch.int32, device=dev) for _ in range(S)]

    def begin(i):
        idx.apply_updates(ids_d, xy_d[i])
        idx.snapshot()
        for j in range(S):
            slots[j].begin(parts[i][j], kind, outs[j], outs[j].numel() * 4)
        for sl in slots:
            stream.wait_stream(sl.stream)

    def end(i):
        """-> results of the step; a part cut by a too-small buffer grows it
        and is answered again (on the same snapshot)."""
        res = 0
        for j in range(S):
            adm, cnt = slots[j].end()
            while adm < parts[i][j].shape[0]:
                outs[j] = torch.empty(max(2 * outs[j].numel(), 1 << 20), dtype=torch.int32, device=dev)
                slots[j].begin(parts[i][j], kind, outs[j], outs[j].numel() * 4)
                adm, cnt = slots[j].end()
            res += slots[j].stats()["n_results"]
        return res

    for i in range(args.warmup):
        begin(i)
        end(i)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(0)
    clocks.start()
    torch.cuda.synchronize()
    results = 0
    for k in range(args.steps):
        i = args.warmup + (k % uniq)
        flush.zero_()
        evs[k][0].record(stream)
        begin(i)
        evs[k][1].record(stream)
        results += end(i)
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    for sl in slots:
        sl.close()
    idx.close()
    srt = sorted(step_ms)
    total = sum(step_ms)
    print(json.dumps({"metric": "queries/s", "value": Q * args.steps / (total / 1000.0), "unit": "queries/s",
                      "ms_per_step": total / args.steps, "steps": args.steps, "warmup": args.warmup,
                      "tick_latency_ms": {"p50": srt[len(srt) // 2], "p99": srt[min(len(srt) - 1, int(0.99 * len(srt)))]},
                      "config": {"workload": w["desc"], "slots": S, "output": args.kind,
                                 "l2": "flushed (%d MB write) between timed steps" % args.flush_mb},
                      "results_per_step": results / args.steps, "clocks": clk}), flush=True)


def run_e2e(args, idx, ticks, kind, elem, Q, dev):
    """End to end through the host-buffer entry points: every step copies the
    tick's updates and queries in from pinned host memory and its output back
    (mqr_apply_updates_host + mqr_tick_host_async; each tick's copy overlaps
    the next tick, mqr_host_wait closes the timed region).  The replayed ticks
    are the timed region's.  The pinned output buffers are sized beforehand
    from the exact output size of every replayed tick (an untimed counting
    tick each); a tick that still does not fit grows them and is answered
    again.  For the covering-compressed kind the step also copies the tick's
    sorted ids (what a consumer needs to expand the runs); for CSR, the
    per-query offsets."""
    import torch
    from paper_1411_3212_gb300 import mqr
    n = ticks[0].ids.shape[0]
    steps = args.steps
    order = [args.warmup + (k % min(args.steps, args.unique_ticks)) for k in range(steps)]
    order = [i if i < len(ticks) else i % len(ticks) for i in order]
    sid_h = torch.empty(n, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
    ids_h = torch.from_numpy(ticks[0].ids.view(np.int32)).pin_memory().numpy().view(np.uint32)
    xy_h = {i: torch.from_numpy(ticks[i].xy).pin_memory().numpy() for i in set(order)}
    rect_h = {i: torch.from_numpy(ticks[i].rects).pin_memory().numpy() for i in set(order)}
    ids_d = torch.from_numpy(ticks[0].ids.view(np.int32)).to(dev)
    csr = kind == mqr.MQR_OUT_CSR
    offs_d = torch.empty(Q + 1, dtype=torch.int64, device=dev) if csr else None
    # exact output size of every replayed tick (a zero-capacity tick reports it)
    need, i_max = -1, order[0]
    for i in sorted(set(order)):
        idx.apply_updates(ids_d, torch.from_numpy(ticks[i].xy).to(dev))
        st, cnt = mqr.mqr_tick(idx.ctx, torch.from_numpy(ticks[i].rects).to(dev), Q, kind, None, 0, offs_d)
        if st not in (mqr.MQR_OK, mqr.MQR_ERR_CAPACITY):
            mqr._check(st)
        if cnt > need:
            need, i_max = cnt, i
    cap_elems = int(need * 1.02) + 4096

    def alloc(elems):
        return [torch.empty(elems * elem // 4, dtype=torch.int32).pin_memory().numpy() for _ in range(2)]

    out_hs = alloc(cap_elems)
    off_hs = [torch.empty(Q + 1, dtype=torch.int64).pin_memory().numpy() if csr else None for _ in range(2)]
    # warm both device staging buffers of the asynchronous path on the
    # largest replayed tick, so that no timed tick grows them
    for oh, ofh in zip(out_hs, off_hs):
        mqr.mqr_apply_updates_host(idx.ctx, ids_h, xy_h[i_max])
        mqr._check(mqr.mqr_tick_host_async(idx.ctx, rect_h[i_max], Q, kind, oh, oh.nbytes, ofh)[0])
    mqr.mqr_host_wait(idx.ctx)
    d2h, regrown, t_calls = [], 0, []
    runs = kind == mqr.MQR_OUT_RUNS
    t_all = time.perf_counter()
    for k, i in enumerate(order):
        t_calls.append(time.perf_counter())
        mqr.mqr_apply_updates_host(idx.ctx, ids_h, xy_h[i])
        oh, ofh = out_hs[k & 1], off_hs[k & 1]
        st, cnt = mqr.mqr_tick_host_async(idx.ctx, rect_h[i], Q, kind, oh, oh.nbytes, ofh, check=False)
        if st == mqr.MQR_ERR_CAPACITY:      # not expected: every replayed tick was counted above
            mqr.mqr_host_wait(idx.ctx)
            cap_elems = int(cnt * 1.1) + 4096
            out_hs = alloc(cap_elems)
            oh = out_hs[k & 1]
            regrown += 1
            st, cnt = mqr.mqr_tick_host_async(idx.ctx, rect_h[i], Q, kind, oh, oh.nbytes, ofh, check=False)
        mqr._check(st)
        ns = mqr.mqr_get_sorted_async(idx.ctx, sid_h) if runs else 0
        d2h.append(cnt * elem + ns * 4 + (8 * (Q + 1) if csr else 0))
    mqr.mqr_host_wait(idx.ctx)
    total = time.perf_counter() - t_all
    t_calls.append(t_all + total)
    gaps = [1000.0 * (b - a) for a, b in zip(t_calls[:-1], t_calls[1:])]
    return {"value": Q * steps / total, "unit": "queries/s",
            "h2d_bytes_per_step": int(n * 12 + Q * 16), "d2h_bytes_per_step": int(sum(d2h) / steps),
            "ms_per_step": 1000.0 * total / steps, "steps": steps, "buffer_regrowths": regrown,
            "d2h_GB_per_s": sum(d2h) / total / 1e9,
            "host_ms_per_step": {"min": min(gaps), "median": statistics.median(gaps), "max": max(gaps)},
            "api": "mqr_apply_updates_host + mqr_tick_host_async%s, mqr_host_wait at the end (pinned host "
                   "buffers; each tick's copy overlaps the next tick)" %
                   (" + mqr_get_sorted_async" if runs else " with the per-query offsets" if csr else "")}


def run_served(args):
    """--served: the served stream (10M objects, 95% in 16 hotspots of sigma
    0.005; Poisson query arrivals at --rate per second, batched into ticks of
    --dt-ms; covering-compressed output with admission by --budget-mb of
    output memory per tick, copied to pinned host memory on a second stream).
    Prints one JSON line with Def. 3 tick latency and Def. 2 query latency
    percentiles and beta (answered queries per second of processing)."""
    import torch
    from paper_1411_3212_gb300 import mqr, workloads
    from paper_1411_3212_gb300.serve import GpuBackend, PlainBackend, SlotBackend, TickServer
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    dt = args.dt_ms / 1000.0
    n_pos = 10                                          # distinct position sets, cycled over the ticks
    t_gen = time.perf_counter()
    world = workloads.ServedWorld(n=args.served_objects, rate=args.rate, dt=dt, seed=0)
    ticks = [world.next_tick() for _ in range(n_pos)]
    rng = np.random.default_rng(12345)                  # arrivals of the ticks after the first n_pos
    arr, rects = [], []
    for k in range(args.served_ticks):
        if k < n_pos:
            a, r = ticks[k].arrivals, ticks[k].rects
        else:
            xy = ticks[k % n_pos].xy
            q = int(rng.poisson(args.rate * dt))
            a = np.sort(rng.random(q)) * dt
            iss = rng.integers(0, world.n, size=q)
            r = workloads.squares_around(xy[iss], np.exp(rng.uniform(np.log(world.side_lo),
                                                                      np.log(world.side_hi), q)))
        arr.append(k * dt + a)
        rects.append(r)
    arrivals = np.concatenate(arr)
    rects = np.concatenate(rects)
    log("served: %d queries over %d ticks generated in %.1f s" % (rects.shape[0], args.served_ticks,
                                                                  time.perf_counter() - t_gen))
    ids_d = torch.from_numpy(ticks[0].ids.view(np.int32)).to(dev)
    updates = [(ids_d, torch.from_numpy(t.xy).to(dev)) for t in ticks]
    rects_d = torch.from_numpy(rects).to(dev)
    max_batch = int(args.max_batch_factor * args.rate * dt) if args.max_batch_factor > 0 else None
    budget = args.budget_mb << 20

    def serve(make_backend):
        """One served run on the arrivals above: 3 warm-up ticks, then the
        stream; a fresh context per run."""
        idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=128, max_objects=world.n)
        be = make_backend(idx)
        TickServer(be, dt, max_batch=max_batch).run(arrivals[arrivals < 3 * dt], n_ticks=3)   # warm-up
        clocks = Clocks(0)
        clocks.start()
        rep = TickServer(be, dt, max_batch=max_batch).run(arrivals, n_ticks=args.served_ticks,
                                                          drain_ticks=args.served_ticks)
        rep["clocks"] = clocks.stop()
        per = rep.pop("per_tick")
        rep["max_out_elems_per_tick"] = max((t.get("out_elems", 0) for t in per), default=0)
        if hasattr(be, "close"):
            be.close()
        idx.close()
        return rep

    copy_out = not args.no_copy_out
    modes = [m for m in args.served_modes.split(",") if m]
    reps = {}
    for m in modes:
        if m == "slots":
            reps[m] = serve(lambda idx: SlotBackend(idx, updates, rects_d, kind="runs", budget_bytes=budget,
                                                    copy_out=copy_out, n_slots=args.served_slots))
        elif m == "admit":
            reps[m] = serve(lambda idx: GpuBackend(idx, updates, rects_d, kind="runs", budget_bytes=budget,
                                                   copy_out=copy_out, overlap=not args.served_plain))
        elif m == "plain":
            reps[m] = serve(lambda idx: PlainBackend(idx, updates, rects_d, kind="runs", copy_out=copy_out))
        else:
            raise SystemExit("unknown served mode %r" % m)
        log("served %s: %s" % (m, json.dumps({k: reps[m][k] for k in ("tick_latency_ms", "beta_queries_per_s")})))
    head = reps[modes[0]]
    desc = {"slots": "continuous batching on %d join slots against one snapshot per tick (mqr_snapshot, "
                     "mqr_slot_begin / mqr_slot_end), each slot admitted against %d MB / %d of output"
                     % (args.served_slots, args.budget_mb, args.served_slots),
            "admit": "one admitted batch per tick (mqr_tick_admit, %d MB of output), copies overlapping the next "
                     "tick" % args.budget_mb,
            "plain": "the plain fixed-capacity quadtree: one blocking mqr_tick per tick on the whole batch, the "
                     "copy waited for"}
    line = {"metric": "served queries/s (beta, Lemma 2)", "value": head["beta_queries_per_s"],
            "unit": "queries/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "served-10M: %d objects (95%% in 16 Gaussian hotspots, sigma 0.005; 5%% "
                                   "uniform), Poisson arrivals %.3g queries/s, square sides log-uniform "
                                   "0.0005-0.004, ticks of %.1f ms, leaf_cap 128, covering-compressed output, %s"
                                   % (world.n, args.rate, args.dt_ms,
                                      "output kept on the device" if args.no_copy_out
                                      else "output copied to pinned host memory"),
                       "ticks": args.served_ticks, "max_batch": max_batch, "mode": modes[0],
                       "modes": {m: desc[m] for m in modes}},
            "served": head, "by_mode": reps}
    print(json.dumps(line), flush=True)


def run_autotune(args):
    """--autotune: the leaf capacity (64..512), then the work-item kernels'
    blocks per SM (2..16, coordinate descent) at that capacity, tuned by
    timing on the workload's ticks; the tuned tick time against the
    configured one (leaf_cap of the workload, 8 blocks per SM), L2 flushed
    before every timed tick."""
    import torch
    from paper_1411_3212_gb300 import mqr
    from paper_1411_3212_gb300.autotune import tune_launch_config, tune_leaf_cap
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    name = args.workload
    w = WORKLOADS[name]
    nmax = w["n"]
    ticks = gen_ticks(name, 0, 6)
    batched = w["kind"] == "batched"
    if batched:                                          # sizes come from the generated worlds
        nmax = int(ticks[0].ids.shape[0])
    dticks = [(torch.from_numpy(t.ids.view(np.int32)).to(dev), torch.from_numpy(t.xy).to(dev),
               torch.from_numpy(t.rects).to(dev)) for t in ticks[1:]]

    def mk(cap):
        index = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=cap, max_objects=nmax)
        if batched:                                      # the worlds keep their sizes across ticks
            index.set_worlds(ticks[0].obj_base)
            index.set_query_worlds(ticks[0].q_base)
        return index
    best_cap, cap_table = tune_leaf_cap(mk, dticks, caps=(64, 128, 256, 512), reps=1)
    idx = mk(best_cap)
    best_launch, launch_table = tune_launch_config(idx, dticks, options=(2, 4, 8, 16), reps=1)
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.int32, device=dev)

    def timed(index):
        ts = []
        for k in range(args.steps):
            ids, xy, rects = dticks[k % len(dticks)]
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            index.apply_updates(ids, xy)
            index.tick(rects, kind="pairs")
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.mean(ts))
    tuned_ms = timed(idx)
    world = None
    if batched:
        # per-world capacities: worlds labelled by kind (even: uniform, odd: 8 hotspots) and size
        from paper_1411_3212_gb300.autotune import tune_world_caps
        sizes = np.diff(ticks[0].obj_base.astype(np.int64))
        labels = ["%s-%s" % ("uniform" if wi % 2 == 0 else "hotspot",
                             "small" if n < 8192 else ("mid" if n < 65536 else "large"))
                  for wi, n in enumerate(sizes)]
        wbits = 0
        while 4 ** wbits < len(sizes):
            wbits += 1
        best_w, _, wtable = tune_world_caps(idx, dticks, wbits, labels, caps=(32, 64, 128, 256, 512), reps=1)
        world_ms = timed(idx)
        idx.set_region_caps(0)
        world = {"labels": "kind (uniform / 8-hotspot) x size (< 8,192, < 65,536, more objects)",
                 "capacity_per_label": best_w, "ms": world_ms, "evaluations": len(wtable),
                 "worlds_per_label": {l: labels.count(l) for l in sorted(set(labels))}}
    idx.close()
    base = mk(w["cap"])
    for ids, xy, rects in dticks:
        base.apply_updates(ids, xy)
        base.tick(rects, kind="pairs")
    base_ms = timed(base)
    base.close()
    line = {"metric": "ms per tick, autotuned leaf capacity and launch shapes vs configured", "unit": "ms",
            "config": {"workload": w["desc"], "steps": args.steps,
                       "l2": "flushed (%d MB write) before every timed tick" % args.flush_mb},
            "configured_ms": base_ms, "tuned_ms": tuned_ms, "leaf_cap": best_cap, "blocks_per_sm": best_launch,
            "per_world_caps": world,
            "leaf_cap_table": {str(c): v["ms_per_tick"] for c, v in cap_table.items()},
            "launch_table": [{"config": c, "ms": ms} for c, ms, _ in launch_table]}
    print(json.dumps(line), flush=True)


def run_per_world(args):
    """--per-world: the batched-worlds workload answered the plain way, one
    context per world and one tick per world in turn, for comparison with the
    single batched index (`--workload batched256`)."""
    import torch
    from paper_1411_3212_gb300 import mqr
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = WORKLOADS["batched256"]
    uniq = min(args.steps, args.unique_ticks)
    ticks = gen_ticks("batched256", 0, args.warmup + uniq)
    ob, qb = ticks[0].obj_base.astype(np.int64), ticks[0].q_base.astype(np.int64)
    W = ob.shape[0] - 1
    xy_d = [torch.from_numpy(t.xy).to(dev) for t in ticks]
    rect_d = [torch.from_numpy(t.rects).to(dev) for t in ticks]
    ids_w = [torch.arange(ob[k + 1] - ob[k], dtype=torch.int32, device=dev) for k in range(W)]
    idxs = [mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=w["cap"], max_objects=int(ob[k + 1] - ob[k]))
            for k in range(W)]
    outs = [torch.empty(1, dtype=torch.int32, device=dev) for _ in range(W)]

    def step(i):
        res = 0
        for k in range(W):
            idx = idxs[k]
            idx.apply_updates(ids_w[k], xy_d[i][ob[k]:ob[k + 1]])
            q = int(qb[k + 1] - qb[k])
            st, cnt = mqr.mqr_tick(idx.ctx, rect_d[i][qb[k]:qb[k + 1]], q, mqr.MQR_OUT_PAIRS, outs[k],
                                   outs[k].numel() * 4)
            if st == mqr.MQR_ERR_CAPACITY:
                outs[k] = torch.empty(int(cnt * 2 * 1.3) + 1024, dtype=torch.int32, device=dev)
                st, cnt = mqr.mqr_tick(idx.ctx, rect_d[i][qb[k]:qb[k + 1]], q, mqr.MQR_OUT_PAIRS, outs[k],
                                       outs[k].numel() * 4)
            mqr._check(st)
            res += cnt
        return res

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    results = 0
    for k in range(args.steps):
        results += step(args.warmup + (k % uniq))
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b) / args.steps
    for idx in idxs:
        idx.close()
    Q = int(qb[-1])
    print(json.dumps({"metric": "queries/s", "value": Q / (ms / 1000.0), "unit": "queries/s", "ms_per_step": ms,
                      "steps": args.steps, "warmup": args.warmup,
                      "config": {"workload": w["desc"] + "; answered per world, one context and one tick each",
                                 "worlds": W, "objects": int(ob[-1]), "queries_per_tick": Q},
                      "results_per_tick": results / args.steps}), flush=True)


def run_costmodel(args):
    """--costmodel: the index configuration chosen per tick by the learned
    cost model (leaf capacities 64..512, the uniform grid at levels 8 and 9,
    density rules for per-region capacities), and per-region capacities chosen
    by the node-level model, against the fixed workload configuration, on the
    same ticks."""
    import torch
    from paper_1411_3212_gb300 import mqr
    from paper_1411_3212_gb300.costmodel import (GRID, QUAD, REGIONS, WORK_KINDS, ArgminChooser, IndexChooser,
                                                 RegionChooser, mean_log2_side)
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    name = args.workload
    w = WORKLOADS[name]
    nmax, Q = w["n"], w["q"]
    uniq = min(args.steps, args.unique_ticks)
    ticks = gen_ticks(name, 0, args.warmup + uniq)
    ids_d = torch.from_numpy(ticks[0].ids.view(np.int32)).to(dev)
    xy_d = [torch.from_numpy(t.xy).to(dev) for t in ticks]
    rect_d = [torch.from_numpy(t.rects).to(dev) for t in ticks]
    sides = [mean_log2_side(t.rects) for t in ticks]
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=w["cap"], max_objects=nmax)
    out = torch.empty(1, dtype=torch.int32, device=dev)

    qs = [int(r.shape[0]) for r in rect_d]           # queries of each tick (the alternating workload varies them)

    def tick(i):
        nonlocal out
        idx.apply_updates(ids_d, xy_d[i])
        st, cnt = mqr.mqr_tick(idx.ctx, rect_d[i], qs[i], mqr.MQR_OUT_PAIRS, out, out.numel() * 4)
        if st == mqr.MQR_ERR_CAPACITY:
            out = torch.empty(int(cnt * 2 * 1.3) + 1024, dtype=torch.int32, device=dev)
            st, cnt = mqr.mqr_tick(idx.ctx, rect_d[i], qs[i], mqr.MQR_OUT_PAIRS, out, out.numel() * 4)
        mqr._check(st)

    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.int32, device=dev)

    def timed(i):
        flush.zero_()                 # every arm starts its tick from a flushed L2
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        tick(i)
        b.record()
        b.synchronize()
        return a.elapsed_time(b)

    for i in range(args.warmup):
        tick(i)
    fixed = [timed(args.warmup + (k % uniq)) for k in range(args.steps)]
    cands = [(QUAD, 64), (QUAD, 128), (QUAD, 256), (QUAD, 512), (GRID, 8), (GRID, 9),
             (REGIONS, 3, 8, -0.25), (REGIONS, 3, 8, 0.25), (REGIONS, 3, 7, 0.5)]
    ch = IndexChooser(candidates=cands, fallback=(QUAD, w["cap"]), seed=0)
    chosen, times = [], []
    for k in range(args.steps):
        i = args.warmup + (k % uniq)
        c = ch.choose(nmax, qs[i], sides[i])
        ch.apply(idx, c)
        ms = timed(i)
        ch.record(c, nmax, qs[i], sides[i], ms)
        chosen.append(c)
        times.append(ms)
    # the same candidates chosen by the argmin of their measured times (no network)
    ach = ArgminChooser(candidates=cands, fallback=(QUAD, w["cap"]), seed=0)
    achosen, atimes = [], []
    for k in range(args.steps):
        i = args.warmup + (k % uniq)
        c = ach.choose(nmax, qs[i], sides[i])
        ach.apply(idx, c)
        ms = timed(i)
        ach.record(c, nmax, qs[i], sides[i], ms)
        achosen.append(c)
        atimes.append(ms)
    # node level: per-region capacities from the MLP over region features
    rch = RegionChooser(region_bits=args.region_bits, fallback=w["cap"], seed=0)
    rtimes = []
    for k in range(args.steps):
        i = args.warmup + (k % uniq)
        rch.apply(idx)
        rtimes.append(timed(i))
        rch.record(idx, rect_d[i])
    final_caps = rch.current.copy()
    rch.finish(idx)
    idx.set_region_caps(0)
    idx.close()
    ch.close()
    rch.close()
    tail = max(1, args.steps // 2)

    def label(c):
        if c[0] == QUAD:
            return "leaf_cap %d" % c[1]
        if c[0] == GRID:
            return "grid level %d" % c[1]
        return "regions %d: cap 2^(%g %+g log2 density)" % (c[1], c[2], c[3])
    counts, acounts = {}, {}
    for c in chosen[-tail:]:
        counts[label(c)] = counts.get(label(c), 0) + 1
    for c in achosen[-tail:]:
        acounts[label(c)] = acounts.get(label(c), 0) + 1
    explored = {}
    for c, ms in zip(chosen[:2 * len(cands)], times[:2 * len(cands)]):   # the round-robin exploration
        explored.setdefault(label(c), []).append(ms)
    line = {"metric": "ms per tick, learned per-tick index choice vs fixed", "unit": "ms",
            "config": {"workload": w["desc"], "candidates": [list(c) for c in cands], "steps": args.steps,
                       "l2": "flushed (%d MB write) before every timed tick" % args.flush_mb},
            "fixed_ms_mean": float(np.mean(fixed[-tail:])), "chosen_ms_mean": float(np.mean(times[-tail:])),
            "explore_ms_mean": float(np.mean(times[:2 * len(cands)])), "chosen_last_half": counts,
            "explored_ms": {k: float(np.mean(v)) for k, v in explored.items()},
            "model_loss": getattr(ch, "loss", None),
            "argmin": {"what": "the same candidates, exploration and exploration rate; the candidate with the smallest "
                               "mean measured time (no network)",
                       "ms_mean": float(np.mean(atimes[-tail:])), "chosen_last_half": acounts},
            "regions": {"region_bits": args.region_bits, "ms_mean": float(np.mean(rtimes[-tail:])),
                        "explore_ms_mean": float(np.mean(rtimes[:rch.explore_ticks])),
                        "capacities_last_tick": {str(int(c)): int((final_caps == c).sum())
                                                 for c in np.unique(final_caps)},
                        "model_loss": getattr(rch, "loss", None), "samples": len(rch.X),
                        "unit_cost_ms": None if rch.unit_cost is None else
                        {k: float(v) for k, v in zip(WORK_KINDS, rch.unit_cost)}}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--unique-ticks", type=int, default=20, help="distinct ticks the timed steps cycle over")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="hotspot4m", choices=sorted(WORKLOADS))
    ap.add_argument("--kind", default="pairs", choices=["pairs", "csr", "count", "runs", "pairs_atomic"])
    ap.add_argument("--offsets", action="store_true", help="also write per-query offsets")
    ap.add_argument("--flush-mb", type=int, default=256)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=400000)
    ap.add_argument("--ref-sample", type=int, default=100000,
                    help="--impl reference: queries joined per step (of the tick's queries)")
    ap.add_argument("--leaf-cap", type=int, default=0, help="override the workload's leaf capacity")
    ap.add_argument("--index", default="quad", choices=["quad", "ug"], help="quadtree or uniform grid")
    ap.add_argument("--no-graph", action="store_true",
                    help="plain kernel launches instead of replaying each tick as one captured CUDA graph")
    ap.add_argument("--graph", action="store_true", help="(the default) replay the tick as a captured CUDA graph")
    ap.add_argument("--grid-level", type=int, default=8, help="uniform grid: 2^level cells per axis")
    ap.add_argument("--served", action="store_true", help="run the served stream instead")
    ap.add_argument("--costmodel", action="store_true", help="learned per-tick index choice vs fixed")
    ap.add_argument("--region-bits", type=int, default=3, help="--costmodel: depth of the node-level regions")
    ap.add_argument("--autotune", action="store_true",
                    help="tune the leaf capacity and the work-item kernels' launch shapes on the workload")
    ap.add_argument("--clock-lead-s", type=float, default=0.25,
                    help="seconds of untimed ticks under the clock sampler before the timed region")
    ap.add_argument("--calib-ticks", type=int, default=5,
                    help="untimed ticks with events around every phase (the per-phase breakdown)")
    ap.add_argument("--no-covering", action="store_true",
                    help="ablation: no covering subqueries (every subquery goes through the containment tests)")
    ap.add_argument("--per-world", action="store_true", help="batched-256 worlds answered one context each")
    ap.add_argument("--slots", type=int, default=0,
                    help="answer each tick's queries split over this many concurrent join slots")
    ap.add_argument("--rate", type=float, default=5.0e6, help="served: query arrivals per second")
    ap.add_argument("--dt-ms", type=float, default=10.0, help="served: tick duration")
    ap.add_argument("--served-ticks", type=int, default=100)
    ap.add_argument("--served-objects", type=int, default=10_000_000)
    ap.add_argument("--budget-mb", type=int, default=1024, help="served: output memory per tick")
    ap.add_argument("--served-modes", default="slots,admit,plain",
                    help="served: backends run on the same arrivals (slots, admit, plain); the first is the headline")
    ap.add_argument("--served-slots", type=int, default=2, help="served: join slots of the slots mode")
    ap.add_argument("--served-plain", action="store_true",
                    help="served: the plain form, no overlap of a tick's copy with the next tick")
    ap.add_argument("--max-batch-factor", type=float, default=1.5,
                    help="served: queries offered per tick, x the mean arrivals per tick (0: whole queue)")
    ap.add_argument("--no-copy-out", action="store_true", help="served: keep each tick's output on the device")
    args = ap.parse_args()
    args.graph = not args.no_graph
    if args.warmup < 3:
        log("warm-up raised to 3 steps")
        args.warmup = 3
    if args.served:
        run_served(args)
    elif args.costmodel:
        run_costmodel(args)
    elif args.autotune:
        run_autotune(args)
    elif args.per_world:
        run_per_world(args)
    elif args.slots > 0:
        run_gpu_slots(args, args.workload)
    elif args.impl == "reference":
        run_reference(args, args.workload)
    else:
        run_gpu(args, args.workload)


if __name__ == "__main__":
    main()
