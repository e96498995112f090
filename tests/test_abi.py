"""The C-ABI library builds, loads and exports every function include/mqr.h
declares; argument validation that needs no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "mqr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mqr_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1411_3212_gb300 import build
    build.build()
    from paper_1411_3212_gb300 import mqr
    return mqr.load()


def test_header_declares_expected_api():
    fns = header_functions()
    for f in ["mqr_create", "mqr_apply_updates", "mqr_tick", "mqr_destroy", "mqr_last_error"]:
        assert f in fns


def test_library_exports_every_declared_symbol(lib):
    from paper_1411_3212_gb300 import mqr
    fns = header_functions()
    assert sorted(mqr.EXPORTS) == fns
    for f in fns:
        assert hasattr(lib, f), f


def test_config_default_and_invalid_args(lib):
    from paper_1411_3212_gb300 import mqr
    cfg = mqr.mqr_config_default()
    assert cfg.leaf_cap == 128 and cfg.max_objects == 1 << 20 and cfg.covering == 1
    ctx = ctypes.c_void_p()
    # argument checks happen before any CUDA call
    bad = mqr.mqr_rect(0.0, 0.0, 0.0, 1.0)
    assert lib.mqr_create(bad, 64, 100, ctypes.byref(ctx)) == mqr.MQR_ERR_INVALID_ARG
    assert "bounds" in mqr.mqr_last_error()
    ok = mqr.mqr_rect(0.0, 0.0, 1.0, 1.0)
    assert lib.mqr_create(ok, 0, 100, ctypes.byref(ctx)) == mqr.MQR_ERR_INVALID_ARG
    assert lib.mqr_create(ok, 64, 100, None) == mqr.MQR_ERR_INVALID_ARG
    cfg.index_kind = 1
    cfg.grid_level = 0
    assert lib.mqr_create_ex(ok, ctypes.byref(cfg), None, ctypes.byref(ctx)) == mqr.MQR_ERR_INVALID_ARG
    cnt = ctypes.c_uint64()
    assert lib.mqr_tick(None, None, 0, 0, None, 0, ctypes.byref(cnt), None) == mqr.MQR_ERR_INVALID_ARG
    assert lib.mqr_apply_updates(None, None, None, 1) == mqr.MQR_ERR_INVALID_ARG
    st = mqr.mqr_stats()
    assert lib.mqr_get_stats(None, ctypes.byref(st)) == mqr.MQR_ERR_INVALID_ARG
    lib.mqr_destroy(None)


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1411_3212_gb300 import mqr
    saved = mqr._lib
    try:
        mqr._lib = None
        with pytest.raises(RuntimeError, match="not built"):
            mqr.load(str(tmp_path / "missing.so"))
    finally:
        mqr._lib = saved


def test_new_entry_points_reject_bad_arguments_without_a_gpu(lib):
    """NULL contexts and out-of-range arguments of the region, launch-shape,
    checkpoint and timing calls are refused before any CUDA call; the
    binding checks array shapes before calling the library."""
    import numpy as np
    from paper_1411_3212_gb300 import mqr
    E = mqr.MQR_ERR_INVALID_ARG
    caps = (ctypes.c_uint32 * 4)(1, 2, 3, 4)
    assert lib.mqr_set_region_caps(None, 1, caps) == E
    assert lib.mqr_region_counts(None, 1, caps) == E
    out = (ctypes.c_double * 36)()
    assert lib.mqr_region_work(None, None, 0, 1, out) == E
    lc = mqr.mqr_launch_config(8, 8, 8, 8)
    assert lib.mqr_set_launch_config(None, ctypes.byref(lc)) == E
    assert lib.mqr_export_state(None, None, None, 0) == E
    assert lib.mqr_import_state(None, None, None, 0) == E
    assert lib.mqr_set_timing_phases(None, 1) == E
    assert lib.mqr_debug_fail_allocation(-1) == mqr.MQR_OK
    with pytest.raises(ValueError):
        mqr.mqr_set_region_caps(None, 2, np.ones(4, np.uint32))      # 4^2 thresholds expected
    with pytest.raises(ValueError):
        mqr.mqr_import_state(None, np.zeros((10, 2), np.float32), np.zeros(9, np.uint8))
    with pytest.raises(mqr.MqrError):
        mqr.mqr_set_launch_config(None, filter=8)


def test_noalloc_rejects_misaligned_pointers_before_any_cuda_call(lib):
    """The allocation-free sort reads float2 positions and writes uint32
    keys and ids: pointers that are not 8- / 4-byte aligned are refused with
    INVALID_ARG before anything is launched (these fake addresses are never
    dereferenced)."""
    from paper_1411_3212_gb300 import mqr
    b = mqr.mqr_rect(0.0, 0.0, 1.0, 1.0)
    assert lib.mqr_sort_objects_noalloc(b, 0x10004, 10, 0x20000, 0x30000, None) == mqr.MQR_ERR_INVALID_ARG
    assert "aligned" in mqr.mqr_last_error()
    assert lib.mqr_sort_objects_noalloc(b, 0x10000, 10, 0x20002, 0x30000, None) == mqr.MQR_ERR_INVALID_ARG
    assert lib.mqr_sort_objects_noalloc(b, 0x10000, 10, 0x20000, 0x30001, None) == mqr.MQR_ERR_INVALID_ARG
    assert lib.mqr_sort_objects_noalloc(b, 0x10000, mqr.MQR_NOALLOC_MAX_OBJECTS + 1, 0x20000, 0x30000,
                                        None) == mqr.MQR_ERR_INVALID_ARG
    assert lib.mqr_debug_stall_scan(0) == mqr.MQR_OK
    fp = (ctypes.c_uint64 * 4)()
    assert lib.mqr_result_footprint(None, fp) == mqr.MQR_ERR_INVALID_ARG
