"""Thin ctypes binding of libmqr (include/mqr.h): same names, argument
marshalling only.  Every step of the join runs in the CUDA library; this
module never computes results itself.  If libmqr.so is missing the functions
raise -- there is no fallback.

Device arguments accept torch CUDA tensors (their data_ptr is passed) or raw
integer device pointers.  Host-buffer entry points accept numpy arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmqr.so")

MQR_OK, MQR_ERR_INVALID_ARG, MQR_ERR_OOM, MQR_ERR_CAPACITY, MQR_ERR_CUDA, MQR_ERR_TIMEOUT, MQR_ERR_INTERNAL = range(7)
(MQR_OUT_PAIRS, MQR_OUT_PAIRS_SORTED, MQR_OUT_CSR, MQR_OUT_CSR_SORTED, MQR_OUT_BITMAP, MQR_OUT_COUNT, MQR_OUT_RUNS,
 MQR_OUT_PAIRS_ATOMIC) = range(8)
MQR_INDEX_QUADTREE, MQR_INDEX_UNIFORM_GRID = 0, 1

KINDS = {"pairs": MQR_OUT_PAIRS, "pairs_sorted": MQR_OUT_PAIRS_SORTED, "csr": MQR_OUT_CSR,
         "csr_sorted": MQR_OUT_CSR_SORTED, "bitmap": MQR_OUT_BITMAP, "count": MQR_OUT_COUNT,
         "runs": MQR_OUT_RUNS, "pairs_atomic": MQR_OUT_PAIRS_ATOMIC}

# Every symbol include/mqr.h declares.
EXPORTS = ["mqr_config_default", "mqr_create", "mqr_create_ex", "mqr_apply_updates",
           "mqr_apply_updates_host", "mqr_tick", "mqr_tick_host", "mqr_tick_host_async", "mqr_host_wait",
           "mqr_get_sorted_async",
           "mqr_tick_admit", "mqr_snapshot", "mqr_slot_create", "mqr_slot_destroy", "mqr_slot_begin",
           "mqr_slot_end", "mqr_slot_get_stats", "mqr_set_graph", "mqr_set_worlds",
           "mqr_set_query_worlds", "mqr_set_index", "mqr_set_region_caps", "mqr_set_launch_config", "mqr_region_counts", "mqr_region_work", "mqr_cost_param_count", "mqr_cost_create",
           "mqr_cost_set_params", "mqr_cost_get_params", "mqr_cost_train", "mqr_cost_gradient", "mqr_cost_predict",
           "mqr_cost_destroy", "mqr_get_stats",
           "mqr_get_leaves",
           "mqr_get_sorted", "mqr_result_footprint", "mqr_export_state", "mqr_import_state",
           "mqr_debug_fail_allocation", "mqr_debug_stall_scan",
           "mqr_set_timing", "mqr_set_timing_phases", "mqr_get_timing",
           "mqr_sort_objects_noalloc",
           "mqr_last_error", "mqr_destroy"]

MQR_NOALLOC_MAX_OBJECTS = 262144

PHASES = ["updates", "keys", "sort", "leaves", "query_blocks", "group", "candidates", "filter",
          "result_scan", "emit", "offsets", "output_sort"]


class MqrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("mqr status %d: %s" % (status, msg))
        self.status = status


class mqr_rect(ctypes.Structure):
    _fields_ = [("xmin", ctypes.c_float), ("ymin", ctypes.c_float),
                ("xmax", ctypes.c_float), ("ymax", ctypes.c_float)]


class mqr_config(ctypes.Structure):
    _fields_ = [("max_objects", ctypes.c_uint32), ("leaf_cap", ctypes.c_uint32),
                ("index_kind", ctypes.c_int32), ("grid_level", ctypes.c_uint32),
                ("covering", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class mqr_launch_config(ctypes.Structure):
    _fields_ = [("candidate_blocks_per_sm", ctypes.c_uint32), ("compact_blocks_per_sm", ctypes.c_uint32),
                ("filter_blocks_per_sm", ctypes.c_uint32), ("emit_blocks_per_sm", ctypes.c_uint32)]


class mqr_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "n_objects", "n_queries", "n_leaves", "max_level", "n_sub_intersecting", "n_sub_covering",
        "n_covering_runs", "n_tests", "n_filter_items", "n_bitmap_words", "n_results",
        "n_results_covering", "n_retries", "n_filter_loads", "n_pairs", "n_candidates")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class mqr_timing(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 12), ("launches", ctypes.c_uint64 * 12), ("ticks", ctypes.c_uint64)]

    def as_dict(self):
        return {"ms": {PHASES[i]: float(self.ms[i]) for i in range(12)},
                "launches": {PHASES[i]: int(self.launches[i]) for i in range(12)},
                "ticks": int(self.ticks)}


_lib = None


def load(path: str = LIB_PATH):
    """Load libmqr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libmqr.so is not built (call __graft_entry__.build()); "
                           "there is no CPU fallback")
    lib = ctypes.CDLL(path)
    P, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    pctx = ctypes.POINTER(P)
    sig = {
        "mqr_config_default": ([ctypes.POINTER(mqr_config)], i32),
        "mqr_create": ([mqr_rect, u32, u32, pctx], i32),
        "mqr_create_ex": ([mqr_rect, ctypes.POINTER(mqr_config), P, pctx], i32),
        "mqr_apply_updates": ([P, P, P, u32], i32),
        "mqr_apply_updates_host": ([P, P, P, u32], i32),
        "mqr_tick": ([P, P, u32, i32, P, u64, ctypes.POINTER(u64), P], i32),
        "mqr_tick_host": ([P, P, u32, i32, P, u64, ctypes.POINTER(u64), P], i32),
        "mqr_tick_host_async": ([P, P, u32, i32, P, u64, ctypes.POINTER(u64), P], i32),
        "mqr_host_wait": ([P], i32),
        "mqr_get_sorted_async": ([P, P, u64, ctypes.POINTER(u64)], i32),
        "mqr_tick_admit": ([P, P, u32, i32, P, u64, ctypes.POINTER(u32), ctypes.POINTER(u64), P], i32),
        "mqr_snapshot": ([P], i32),
        "mqr_slot_create": ([P, P, pctx], i32),
        "mqr_slot_destroy": ([P], None),
        "mqr_slot_begin": ([P, P, u32, i32, P, u64, P], i32),
        "mqr_slot_end": ([P, ctypes.POINTER(u32), ctypes.POINTER(u64)], i32),
        "mqr_slot_get_stats": ([P, ctypes.POINTER(mqr_stats)], i32),
        "mqr_set_graph": ([P, i32], i32),
        "mqr_set_worlds": ([P, u32, P], i32),
        "mqr_set_query_worlds": ([P, P], i32),
        "mqr_set_index": ([P, i32, u32, u32], i32),
        "mqr_set_region_caps": ([P, u32, P], i32),
        "mqr_set_launch_config": ([P, ctypes.POINTER(mqr_launch_config)], i32),
        "mqr_region_counts": ([P, u32, P], i32),
        "mqr_region_work": ([P, P, u32, u32, P], i32),
        "mqr_cost_param_count": ([], u32),
        "mqr_cost_create": ([pctx], i32),
        "mqr_cost_set_params": ([P, P, u32], i32),
        "mqr_cost_get_params": ([P, P, u32], i32),
        "mqr_cost_train": ([P, P, P, u32, u32, ctypes.c_float, ctypes.POINTER(ctypes.c_float)], i32),
        "mqr_cost_gradient": ([P, P, P, u32, P, ctypes.POINTER(ctypes.c_float)], i32),
        "mqr_cost_predict": ([P, P, u32, P], i32),
        "mqr_cost_destroy": ([P], None),
        "mqr_get_stats": ([P, ctypes.POINTER(mqr_stats)], i32),
        "mqr_get_leaves": ([P, P, u64, ctypes.POINTER(u64)], i32),
        "mqr_get_sorted": ([P, P, P, u64, ctypes.POINTER(u64)], i32),
        "mqr_set_timing": ([P, i32], i32),
        "mqr_set_timing_phases": ([P, u32], i32),
        "mqr_export_state": ([P, P, P, u32], i32),
        "mqr_import_state": ([P, P, P, u32], i32),
        "mqr_debug_fail_allocation": ([i32], i32),
        "mqr_debug_stall_scan": ([i32], i32),
        "mqr_result_footprint": ([P, P], i32),
        "mqr_get_timing": ([P, ctypes.POINTER(mqr_timing)], i32),
        "mqr_sort_objects_noalloc": ([mqr_rect, P, u32, P, P, P], i32),
        "mqr_last_error": ([], ctypes.c_char_p),
        "mqr_destroy": ([P], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return x.data_ptr()
    raise TypeError("expected a torch CUDA tensor or an int device pointer")


def _hptr(a):
    if a is None:
        return None
    if not isinstance(a, np.ndarray) or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a C-contiguous numpy array")
    return a.ctypes.data


def _check(status):
    if status != MQR_OK:
        raise MqrError(status, load().mqr_last_error().decode())
    return status


# -- same names as the C ABI -------------------------------------------------
def mqr_config_default():
    cfg = mqr_config()
    _check(load().mqr_config_default(ctypes.byref(cfg)))
    return cfg


def mqr_create(bounds, leaf_cap, max_objects):
    ctx = ctypes.c_void_p()
    _check(load().mqr_create(mqr_rect(*bounds), leaf_cap, max_objects, ctypes.byref(ctx)))
    return ctx


def mqr_create_ex(bounds, cfg: mqr_config, cuda_stream=None):
    ctx = ctypes.c_void_p()
    _check(load().mqr_create_ex(mqr_rect(*bounds), ctypes.byref(cfg), cuda_stream, ctypes.byref(ctx)))
    return ctx


def mqr_apply_updates(ctx, ids_dev, xy_dev, n=None):
    n = int(ids_dev.shape[0]) if n is None else n
    _check(load().mqr_apply_updates(ctx, _ptr(ids_dev), _ptr(xy_dev), n))


def mqr_apply_updates_host(ctx, ids_host, xy_host):
    n = int(ids_host.shape[0])
    _check(load().mqr_apply_updates_host(ctx, _hptr(ids_host), _hptr(xy_host), n))


def mqr_tick(ctx, rects_dev, Q, kind, out_dev, out_capacity_bytes, offsets_dev=None, check=True):
    """Returns (status, out_count)."""
    cnt = ctypes.c_uint64(0)
    st = load().mqr_tick(ctx, _ptr(rects_dev), Q, kind, _ptr(out_dev), out_capacity_bytes,
                         ctypes.byref(cnt), _ptr(offsets_dev))
    if check and st not in (MQR_OK, MQR_ERR_CAPACITY):
        _check(st)
    return st, int(cnt.value)


def mqr_tick_host(ctx, rects_host, Q, kind, out_host, out_capacity_bytes, offsets_host=None, check=True):
    cnt = ctypes.c_uint64(0)
    st = load().mqr_tick_host(ctx, _hptr(rects_host), Q, kind, _hptr(out_host), out_capacity_bytes,
                              ctypes.byref(cnt), _hptr(offsets_host))
    if check and st not in (MQR_OK, MQR_ERR_CAPACITY):
        _check(st)
    return st, int(cnt.value)


def mqr_tick_admit(ctx, rects_dev, Q, kind, out_dev, out_capacity_bytes, offsets_dev=None):
    """Returns (admitted, out_count)."""
    adm = ctypes.c_uint32(0)
    cnt = ctypes.c_uint64(0)
    _check(load().mqr_tick_admit(ctx, _ptr(rects_dev), Q, kind, _ptr(out_dev), out_capacity_bytes,
                                 ctypes.byref(adm), ctypes.byref(cnt), _ptr(offsets_dev)))
    return int(adm.value), int(cnt.value)


def mqr_snapshot(ctx):
    _check(load().mqr_snapshot(ctx))


def mqr_slot_create(ctx, cuda_stream=None):
    out = ctypes.c_void_p()
    _check(load().mqr_slot_create(ctx, cuda_stream, ctypes.byref(out)))
    return out.value


def mqr_slot_destroy(slot):
    if slot:
        load().mqr_slot_destroy(slot)


def mqr_slot_begin(slot, rects_dev, Q, kind, out_dev, out_capacity_bytes, offsets_dev=None):
    _check(load().mqr_slot_begin(slot, _ptr(rects_dev), Q, kind, _ptr(out_dev), out_capacity_bytes,
                                 _ptr(offsets_dev)))


def mqr_slot_end(slot):
    """Returns (admitted, out_count)."""
    a = ctypes.c_uint32(0)
    n = ctypes.c_uint64(0)
    _check(load().mqr_slot_end(slot, ctypes.byref(a), ctypes.byref(n)))
    return int(a.value), int(n.value)


def mqr_slot_get_stats(slot):
    s = mqr_stats()
    _check(load().mqr_slot_get_stats(slot, ctypes.byref(s)))
    return s.as_dict()


class Slot:
    """A join slot of an Index (mqr_slot_*): answers batches against the
    index's last snapshot on its own CUDA stream (a torch stream: `stream`,
    created if not given)."""

    def __init__(self, index, stream=None):
        import torch
        self.index = index
        self.stream = stream if stream is not None else torch.cuda.Stream(device=torch.cuda.current_device())
        self.slot = mqr_slot_create(index.ctx, ctypes.c_void_p(self.stream.cuda_stream))

    def begin(self, rects, kind, out, capacity_bytes, offsets=None):
        mqr_slot_begin(self.slot, rects, int(rects.shape[0]), KINDS[kind] if isinstance(kind, str) else kind,
                       out, capacity_bytes, offsets)

    def end(self):
        return mqr_slot_end(self.slot)

    def stats(self):
        return mqr_slot_get_stats(self.slot)

    def close(self):
        if self.slot:
            mqr_slot_destroy(self.slot)
            self.slot = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mqr_set_graph(ctx, enable):
    _check(load().mqr_set_graph(ctx, 1 if enable else 0))


def mqr_set_index(ctx, index_kind, leaf_cap=0, grid_level=0):
    _check(load().mqr_set_index(ctx, int(index_kind), int(leaf_cap), int(grid_level)))


def mqr_set_region_caps(ctx, region_bits, caps=None):
    """caps: 4^region_bits split thresholds in Morton order of the regions."""
    if region_bits:
        arr = np.ascontiguousarray(caps, dtype=np.uint32)
        if arr.shape != (4 ** int(region_bits),):
            raise ValueError("caps must hold 4^region_bits thresholds")
        _check(load().mqr_set_region_caps(ctx, int(region_bits), arr.ctypes.data_as(ctypes.c_void_p)))
    else:
        _check(load().mqr_set_region_caps(ctx, 0, None))


LAUNCH_KERNELS = ("candidate", "compact", "filter", "emit")


def mqr_set_launch_config(ctx, candidate=0, compact=0, filter=0, emit=0):
    """Blocks per SM of the work-item kernels (0: the default)."""
    cfg = mqr_launch_config(int(candidate), int(compact), int(filter), int(emit))
    _check(load().mqr_set_launch_config(ctx, ctypes.byref(cfg)))


def mqr_region_counts(ctx, region_bits):
    out = np.zeros(4 ** int(region_bits), np.uint32)
    _check(load().mqr_region_counts(ctx, int(region_bits), out.ctypes.data_as(ctypes.c_void_p)))
    return out


REGION_STATS = ("objects", "leaves", "queries", "side_log2_sum", "sub_intersecting", "sub_covering", "tests",
                "results_intersecting", "results_covering")


def mqr_region_work(ctx, rects_dev, Q, region_bits):
    """Per-region work of the last tick: dict statistic -> float64[4^region_bits]."""
    out = np.zeros((len(REGION_STATS), 4 ** int(region_bits)), np.float64)
    _check(load().mqr_region_work(ctx, _ptr(rects_dev), int(Q), int(region_bits),
                                  out.ctypes.data_as(ctypes.c_void_p)))
    return dict(zip(REGION_STATS, out))


class CostModel:
    """The learned tick-cost model (MLP 5 -> 64 -> 64 -> 1 trained on the
    device); marshalling only."""

    def __init__(self, params=None):
        lib = load()
        self.P = int(lib.mqr_cost_param_count())
        h = ctypes.c_void_p()
        _check(lib.mqr_cost_create(ctypes.byref(h)))
        self.h = h
        if params is not None:
            self.set_params(params)

    def set_params(self, params):
        a = np.ascontiguousarray(params, dtype=np.float32)
        _check(load().mqr_cost_set_params(self.h, a.ctypes.data, int(a.shape[0])))

    def params(self):
        a = np.zeros(self.P, np.float32)
        _check(load().mqr_cost_get_params(self.h, a.ctypes.data, self.P))
        return a

    def train(self, X, y, epochs=1, lr=1e-3):
        X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, 5)
        y = np.ascontiguousarray(y, dtype=np.float32).reshape(-1)
        loss = ctypes.c_float(0.0)
        _check(load().mqr_cost_train(self.h, X.ctypes.data, y.ctypes.data, int(X.shape[0]), int(epochs),
                                     float(lr), ctypes.byref(loss)))
        return float(loss.value)

    def gradient(self, X, y):
        X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, 5)
        y = np.ascontiguousarray(y, dtype=np.float32).reshape(-1)
        g = np.zeros(self.P, np.float32)
        loss = ctypes.c_float(0.0)
        _check(load().mqr_cost_gradient(self.h, X.ctypes.data, y.ctypes.data, int(X.shape[0]), g.ctypes.data,
                                        ctypes.byref(loss)))
        return g, float(loss.value)

    def predict(self, X):
        X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, 5)
        out = np.zeros(X.shape[0], np.float32)
        _check(load().mqr_cost_predict(self.h, X.ctypes.data, int(X.shape[0]), out.ctypes.data))
        return out

    def close(self):
        if self.h:
            load().mqr_cost_destroy(self.h)
            self.h = None


def mqr_set_worlds(ctx, obj_base):
    b = np.ascontiguousarray(obj_base, dtype=np.uint32)
    _check(load().mqr_set_worlds(ctx, int(b.shape[0]) - 1, b.ctypes.data))


def mqr_set_query_worlds(ctx, q_base):
    b = np.ascontiguousarray(q_base, dtype=np.uint32)
    _check(load().mqr_set_query_worlds(ctx, b.ctypes.data))


def mqr_tick_host_async(ctx, rects_host, Q, kind, out_host, out_capacity_bytes, offsets_host=None, check=True):
    cnt = ctypes.c_uint64(0)
    st = load().mqr_tick_host_async(ctx, _hptr(rects_host), Q, kind, _hptr(out_host), out_capacity_bytes,
                                    ctypes.byref(cnt), _hptr(offsets_host))
    if check and st not in (MQR_OK, MQR_ERR_CAPACITY):
        _check(st)
    return st, int(cnt.value)


def mqr_host_wait(ctx):
    _check(load().mqr_host_wait(ctx))


def mqr_get_sorted_async(ctx, ids_host):
    n = ctypes.c_uint64(0)
    _check(load().mqr_get_sorted_async(ctx, _hptr(ids_host), int(ids_host.shape[0]), ctypes.byref(n)))
    return int(n.value)


def mqr_get_stats(ctx):
    s = mqr_stats()
    _check(load().mqr_get_stats(ctx, ctypes.byref(s)))
    return s.as_dict()


def mqr_get_leaves(ctx):
    n = ctypes.c_uint64(0)
    st = load().mqr_get_leaves(ctx, None, 0, ctypes.byref(n))
    if st not in (MQR_OK, MQR_ERR_CAPACITY):
        _check(st)
    out = np.zeros((int(n.value), 4), np.uint32)
    if n.value:
        _check(load().mqr_get_leaves(ctx, out.ctypes.data, out.shape[0], ctypes.byref(n)))
    return out


def mqr_get_sorted(ctx):
    n = ctypes.c_uint64(0)
    st = load().mqr_get_sorted(ctx, None, None, 0, ctypes.byref(n))
    if st not in (MQR_OK, MQR_ERR_CAPACITY):
        _check(st)
    keys = np.zeros(int(n.value), np.uint32)
    ids = np.zeros(int(n.value), np.uint32)
    if n.value:
        _check(load().mqr_get_sorted(ctx, keys.ctypes.data, ids.ctypes.data, keys.shape[0], ctypes.byref(n)))
    return keys, ids


def mqr_set_timing(ctx, enable):
    _check(load().mqr_set_timing(ctx, 1 if enable else 0))


def mqr_export_state(ctx, max_objects):
    """-> (xy float32[max_objects, 2], present uint8[max_objects])."""
    xy = np.zeros((max_objects, 2), np.float32)
    present = np.zeros(max_objects, np.uint8)
    _check(load().mqr_export_state(ctx, xy.ctypes.data_as(ctypes.c_void_p), present.ctypes.data_as(ctypes.c_void_p),
                                   max_objects))
    return xy, present


def mqr_import_state(ctx, xy, present):
    xy = np.ascontiguousarray(xy, np.float32)
    present = np.ascontiguousarray(present, np.uint8)
    if xy.shape != (present.shape[0], 2):
        raise ValueError("xy must be [n, 2] with n = len(present)")
    _check(load().mqr_import_state(ctx, xy.ctypes.data_as(ctypes.c_void_p), present.ctypes.data_as(ctypes.c_void_p),
                                   present.shape[0]))


def mqr_debug_fail_allocation(after):
    _check(load().mqr_debug_fail_allocation(int(after)))


def mqr_debug_stall_scan(enable=True):
    _check(load().mqr_debug_stall_scan(1 if enable else 0))


def mqr_result_footprint(ctx):
    """-> dict of the last tick's leaf footprint: leaves with results and
    their objects, tested leaves and their objects."""
    out = np.zeros(4, np.uint64)
    _check(load().mqr_result_footprint(ctx, out.ctypes.data))
    return {"result_leaves": int(out[0]), "result_leaf_objects": int(out[1]),
            "tested_leaves": int(out[2]), "tested_leaf_objects": int(out[3])}


def mqr_set_timing_phases(ctx, phases):
    """Time only the named phases (launch counts for all); empty: off."""
    mask = 0
    for p in phases:
        mask |= 1 << PHASES.index(p)
    _check(load().mqr_set_timing_phases(ctx, mask))


def mqr_get_timing(ctx):
    t = mqr_timing()
    _check(load().mqr_get_timing(ctx, ctypes.byref(t)))
    return t.as_dict()


def mqr_sort_objects_noalloc(bounds, xy_dev, n, keys_out_dev, ids_out_dev, cuda_stream=None):
    _check(load().mqr_sort_objects_noalloc(mqr_rect(*bounds), _ptr(xy_dev), n, _ptr(keys_out_dev),
                                           _ptr(ids_out_dev), cuda_stream))


def mqr_last_error():
    return load().mqr_last_error().decode()


def mqr_destroy(ctx):
    if ctx:
        load().mqr_destroy(ctx)


# -- convenience wrapper ------------------------------------------------------
class Index:
    """Owns one mqr context; torch tensors in, torch tensors out."""

    def __init__(self, bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=128, max_objects=1 << 20,
                 index_kind=MQR_INDEX_QUADTREE, grid_level=8, covering=True, stream=None):
        import torch
        self._torch = torch
        cfg = mqr_config_default()
        cfg.max_objects = max_objects
        cfg.leaf_cap = min(int(leaf_cap), 0xFFFFFFFF)
        cfg.index_kind = index_kind
        cfg.grid_level = grid_level
        cfg.covering = 1 if covering else 0
        self.max_objects = max_objects
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = mqr_create_ex(bounds, cfg, ctypes.c_void_p(self.stream.cuda_stream))
        self._out = None

    def close(self):
        if self.ctx:
            mqr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply_updates(self, ids, xy):
        mqr_apply_updates(self.ctx, ids, xy, int(ids.shape[0]))

    def tick(self, rects, kind="pairs"):
        """Answer the queries; returns (result, offsets) as CUDA tensors.
        pairs/pairs_sorted -> int32[R, 2] (qidx, id); csr/csr_sorted -> int32[R];
        bitmap -> int32[Q, ceil(max_objects/32)]; count -> None; runs ->
        int32[E, 2] covering-compressed elements (MQR_OUT_RUNS).  Values
        are uint32 reinterpreted as int32."""
        torch = self._torch
        k = KINDS[kind]
        Q = int(rects.shape[0])
        offs = torch.empty(Q + 1, dtype=torch.int64, device=rects.device) if k != MQR_OUT_PAIRS_ATOMIC else None
        if k == MQR_OUT_BITMAP:
            W = (self.max_objects + 31) // 32
            out = torch.empty((Q, W), dtype=torch.int32, device=rects.device)
            mqr_tick(self.ctx, rects, Q, k, out, out.numel() * 4, offs)
            return out, offs
        if k == MQR_OUT_COUNT:
            mqr_tick(self.ctx, rects, Q, k, None, 0, offs)
            return None, offs
        elem = 8 if k in (MQR_OUT_PAIRS, MQR_OUT_PAIRS_SORTED, MQR_OUT_RUNS, MQR_OUT_PAIRS_ATOMIC) else 4
        if self._out is None:
            self._out = torch.empty(max(1 << 16, 8 * Q) * 2, dtype=torch.int32, device=rects.device)
        st, cnt = mqr_tick(self.ctx, rects, Q, k, self._out, self._out.numel() * 4, offs)
        if st == MQR_ERR_CAPACITY:
            self._out = torch.empty(max(cnt * elem // 4 + 1024, 1), dtype=torch.int32, device=rects.device)
            st, cnt = mqr_tick(self.ctx, rects, Q, k, self._out, self._out.numel() * 4, offs)
            _check(st)
        res = self._out[: cnt * elem // 4]
        return (res.view(cnt, 2) if elem == 8 else res), offs

    def set_index(self, index_kind=0, leaf_cap=0, grid_level=0):
        mqr_set_index(self.ctx, index_kind, leaf_cap, grid_level)

    def set_region_caps(self, region_bits, caps=None):
        mqr_set_region_caps(self.ctx, region_bits, caps)

    def export_state(self):
        return mqr_export_state(self.ctx, self.max_objects)

    def import_state(self, xy, present):
        mqr_import_state(self.ctx, xy, present)

    def set_launch_config(self, **blocks_per_sm):
        mqr_set_launch_config(self.ctx, **blocks_per_sm)

    def region_counts(self, region_bits):
        return mqr_region_counts(self.ctx, region_bits)

    def region_work(self, rects, region_bits):
        return mqr_region_work(self.ctx, rects, rects.shape[0], region_bits)

    def set_graph(self, enable=True):
        mqr_set_graph(self.ctx, enable)

    def set_worlds(self, obj_base):
        mqr_set_worlds(self.ctx, obj_base)

    def set_query_worlds(self, q_base):
        mqr_set_query_worlds(self.ctx, q_base)

    def snapshot(self):
        mqr_snapshot(self.ctx)

    def slot(self, stream=None):
        return Slot(self, stream)

    def footprint(self):
        return mqr_result_footprint(self.ctx)

    def stats(self):
        return mqr_get_stats(self.ctx)

    def set_timing(self, enable=True, phases=None):
        """Per-phase timing: all phases, or only the named ones (launches are
        counted for all)."""
        if enable and phases is not None:
            mqr_set_timing_phases(self.ctx, phases)
        else:
            mqr_set_timing(self.ctx, enable)

    def timing(self):
        return mqr_get_timing(self.ctx)

    def leaves(self):
        return mqr_get_leaves(self.ctx)

    def sorted_objects(self):
        return mqr_get_sorted(self.ctx)
