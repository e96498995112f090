"""CPU oracle for the per-tick repeated-range-query join (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` legs import this package.  The CUDA
product path (``paper_1411_3212_gb300``) never imports it, and the two share
no code: this module wraps ``mqr_oracle.c`` (plain single-threaded C) with
ctypes and numpy.

Functions (each citing the paper passage its C routine follows):
  apply_updates  -- Sec. 2.2 batch processing, last update of a tick wins.
  join_grid      -- Def. 1 result sets through a uniform grid (exact).
  join_brute     -- Def. 1 by testing every (query, object) pair.
  count_grid     -- per-query result counts (Def. 1), optionally with an
                    order-independent 64-bit checksum of each result set.
  bitmap         -- query x object bitmap of a result (bitmap layout of the
                    filtering phase, Sec. 5.4, taken over the whole Q x N).
  cell / scale / morton / keys -- Morton codes at l_max = 15 (Alg. 1).
  quadtree       -- Alg. 1 PR-quadtree leaves, level by level (one split
                    threshold, or one per region of a chosen level).
  subqueries     -- Def. "Mapping functions" g(q), intersecting/covering.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mqr_oracle.c")
_LIB = os.path.join(_HERE, "libmqr_oracle.%s.so" % platform.machine())
_FLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]

_lib = None


def build(force: bool = False) -> str:
    """Compile ``mqr_oracle.c`` into ``libmqr_oracle.<machine>.so`` next to it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", *_FLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Leaf(ctypes.Structure):
    _fields_ = [("level", ctypes.c_uint32), ("z", ctypes.c_uint32),
                ("begin", ctypes.c_uint32), ("end", ctypes.c_uint32)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    u32, u64, i64, f32, f64 = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64,
                               ctypes.c_float, ctypes.c_double)
    lib.orc_apply_updates.argtypes = [P, P, u32, P, P, u32]
    lib.orc_apply_updates.restype = ctypes.c_int
    lib.orc_join_brute.argtypes = [P, P, u32, P, u32, P, ctypes.POINTER(P)]
    lib.orc_join_brute.restype = i64
    lib.orc_join_grid.argtypes = [P, P, u32, P, u32, f64, f64, f64, f64, f64, P, ctypes.POINTER(P)]
    lib.orc_join_grid.restype = i64
    lib.orc_count_grid.argtypes = [P, P, u32, P, u32, f64, f64, f64, f64, f64, P, P]
    lib.orc_count_grid.restype = i64
    lib.orc_bitmap.argtypes = [P, P, u32, u32, P]
    lib.orc_bitmap.restype = None
    lib.orc_cell.argtypes = [f32, f32, f32]
    lib.orc_cell.restype = u32
    lib.orc_scale.argtypes = [f32, f32]
    lib.orc_scale.restype = f32
    lib.orc_morton.argtypes = [u32, u32]
    lib.orc_morton.restype = u32
    lib.orc_keys.argtypes = [P, P, u32, f32, f32, f32, f32, P]
    lib.orc_keys.restype = None
    lib.orc_quadtree.argtypes = [P, u32, u32, u32, P, u64]
    lib.orc_quadtree.restype = i64
    lib.orc_quadtree_regions.argtypes = [P, u32, u32, P, u32, P, u64]
    lib.orc_quadtree_regions.restype = i64
    lib.orc_subqueries.argtypes = [P, u64, ctypes.c_int, P, f32, f32, f32, f32, P, P, u64]
    lib.orc_subqueries.restype = i64
    lib.orc_free.argtypes = [P]
    lib.orc_free.restype = None
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


def _f32(a, shape_tail):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a.reshape((-1,) + shape_tail) if a.size else np.zeros((0,) + shape_tail, np.float32)


class State:
    """Last-known positions of objects ``0 .. nmax-1`` (absent until updated)."""

    def __init__(self, nmax: int):
        self.nmax = int(nmax)
        self.pos = np.zeros((self.nmax, 2), np.float32)
        self.present = np.zeros(self.nmax, np.uint8)

    def apply_updates(self, ids, xy) -> None:
        """Sec. 2.2: apply a tick's updates in order; the last one of an id wins."""
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        xy = _f32(xy, (2,))
        assert xy.shape[0] == ids.shape[0]
        rc = _load().orc_apply_updates(_ptr(self.pos), _ptr(self.present), self.nmax,
                                       _ptr(ids), _ptr(xy), ids.shape[0])
        if rc != 0:
            raise ValueError("object id out of range")


def _csr_from_c(lib, Q, offsets, ptr, total):
    if total < 0:
        raise MemoryError("oracle allocation failed")
    ids = np.zeros(int(total), np.uint32)
    if total:
        ctypes.memmove(ids.ctypes.data, ptr.value, int(total) * 4)
    lib.orc_free(ptr)
    return offsets, ids


def join_brute(state: State, rects):
    """Def. 1 by brute force -> (offsets u64[Q+1], ids u32[R]) ascending per query."""
    lib = _load()
    rects = _f32(rects, (4,))
    Q = rects.shape[0]
    off = np.zeros(Q + 1, np.uint64)
    p = ctypes.c_void_p()
    total = lib.orc_join_brute(_ptr(state.pos), _ptr(state.present), state.nmax,
                               _ptr(rects), Q, _ptr(off), ctypes.byref(p))
    return _csr_from_c(lib, Q, off, p, total)


def join_grid(state: State, rects, bounds=(0.0, 0.0, 1.0, 1.0), cell_side=0.01):
    """Def. 1 through a uniform grid -> (offsets u64[Q+1], ids u32[R]) ascending per query."""
    lib = _load()
    rects = _f32(rects, (4,))
    Q = rects.shape[0]
    off = np.zeros(Q + 1, np.uint64)
    p = ctypes.c_void_p()
    x0, y0, x1, y1 = (float(b) for b in bounds)
    total = lib.orc_join_grid(_ptr(state.pos), _ptr(state.present), state.nmax, _ptr(rects), Q,
                              x0, y0, x1, y1, float(cell_side), _ptr(off), ctypes.byref(p))
    return _csr_from_c(lib, Q, off, p, total)


def count_grid(state: State, rects, bounds=(0.0, 0.0, 1.0, 1.0), cell_side=0.01, with_hash=False):
    """Per-query result counts (Def. 1) -> u64[Q]; with_hash: (counts,
    hashes), hashes[q] = sum modulo 2^64 of splitmix64's output function of
    (q << 32 | id) over the ids of query q's result set."""
    lib = _load()
    rects = _f32(rects, (4,))
    Q = rects.shape[0]
    cnt = np.zeros(Q, np.uint64)
    hs = np.zeros(Q, np.uint64) if with_hash else None
    x0, y0, x1, y1 = (float(b) for b in bounds)
    r = lib.orc_count_grid(_ptr(state.pos), _ptr(state.present), state.nmax, _ptr(rects), Q,
                           x0, y0, x1, y1, float(cell_side), _ptr(cnt), _ptr(hs) if with_hash else None)
    if r < 0:
        raise MemoryError("oracle allocation failed")
    return (cnt, hs) if with_hash else cnt


def bitmap(offsets, ids, nmax: int):
    """Q x ceil(nmax/32) u32 words: bit (id mod 32) of word id/32 in row q."""
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    Q = offsets.shape[0] - 1
    W = (int(nmax) + 31) // 32
    words = np.zeros((Q, W), np.uint32)
    if Q and W:
        _load().orc_bitmap(_ptr(offsets), _ptr(ids), Q, int(nmax), _ptr(words))
    return words


def scale(lo: float, hi: float) -> float:
    return float(_load().orc_scale(lo, hi))


def cell(v: float, lo: float, sc: float) -> int:
    return int(_load().orc_cell(v, lo, sc))


def morton(i: int, j: int) -> int:
    return int(_load().orc_morton(i, j))


def keys(state: State, bounds=(0.0, 0.0, 1.0, 1.0)):
    """Morton key (l_max = 15) of every slot; 0xFFFFFFFF for absent slots."""
    out = np.zeros(state.nmax, np.uint32)
    x0, y0, x1, y1 = (float(b) for b in bounds)
    _load().orc_keys(_ptr(state.pos), _ptr(state.present), state.nmax, x0, y0, x1, y1, _ptr(out))
    return out


def quadtree(sorted_keys, th_quad: int, lmax: int = 15, region_bits: int = 0, region_caps=None):
    """Alg. 1 leaves -> structured array (level, z, begin, end) in Morton order.

    region_bits > 0: the split threshold of a quadrant at level >= region_bits
    is region_caps[its ancestor at level region_bits] (4^region_bits entries,
    Morton order) and th_quad is unused; non-empty quadrants above that level
    are split."""
    k = np.ascontiguousarray(sorted_keys, dtype=np.uint32)
    n = k.shape[0]
    cap = 4 * max(n, 1) * (lmax + 1) + 4 ** region_bits + 4
    out = (Leaf * cap)()
    if region_bits:
        caps = np.ascontiguousarray(region_caps, dtype=np.uint32)
        if caps.shape != (4 ** region_bits,):
            raise ValueError("region_caps must hold 4^region_bits thresholds")
        r = _load().orc_quadtree_regions(_ptr(k), n, region_bits, _ptr(caps), lmax,
                                         ctypes.cast(out, ctypes.c_void_p), cap)
    else:
        r = _load().orc_quadtree(_ptr(k), n, int(min(th_quad, 0xFFFFFFFF)), lmax,
                                 ctypes.cast(out, ctypes.c_void_p), cap)
    if r < 0:
        raise RuntimeError("oracle quadtree failed")
    dt = np.dtype([("level", np.uint32), ("z", np.uint32), ("begin", np.uint32), ("end", np.uint32)])
    return np.frombuffer(bytes(out)[: int(r) * 16], dtype=dt).copy()


def subqueries(leaves, rect, bounds=(0.0, 0.0, 1.0, 1.0), skip_empty=True):
    """g(q): (leaf indices u32[k], covering flags u8[k]) in leaf order."""
    lv = np.ascontiguousarray(leaves)
    r = _f32(rect, (4,)).reshape(4)
    cap = max(len(lv), 1)
    out_leaf = np.zeros(cap, np.uint32)
    out_cov = np.zeros(cap, np.uint8)
    x0, y0, x1, y1 = (float(b) for b in bounds)
    k = _load().orc_subqueries(_ptr(lv.view(np.uint8)) if len(lv) else ctypes.c_void_p(0), len(lv),
                               1 if skip_empty else 0, _ptr(r), x0, y0, x1, y1,
                               _ptr(out_leaf), _ptr(out_cov), cap)
    if k < 0:
        raise RuntimeError("oracle subqueries failed")
    return out_leaf[:k].copy(), out_cov[:k].copy()


def csr_lists(offsets, ids):
    """Split a CSR result into a list of per-query id arrays."""
    return [ids[int(offsets[q]):int(offsets[q + 1])] for q in range(len(offsets) - 1)]


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
