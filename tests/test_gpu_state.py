"""Checkpoint / restart of the object state and failure handling by an
injected allocation failure (on the host: the allocation call reports out of
memory; no GPU fault is involved)."""
import numpy as np
import pytest

import oracle
from paper_1411_3212_gb300 import workloads
from tests.gpu_util import assert_same_csr, gpu_csr_sorted, oracle_state, to_dev, torch_dev

pytestmark = pytest.mark.gpu


def test_export_import_restarts_exactly():
    """A context restored from another's checkpoint answers every following
    tick exactly as the original (and as the oracle), including objects that
    were never updated and updates applied after the restore."""
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    n = 40_000
    w = workloads.HotspotWalk(n=n, q=1500, hotspots=5, side_lo=0.001, side_hi=0.03, seed=31)
    a = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=64, max_objects=n + 17)   # 17 slots never updated
    st = oracle.State(n + 17)
    for _ in range(3):
        t = w.next_tick()
        a.apply_updates(to_dev(t.ids, dev), to_dev(t.xy, dev))
        st.apply_updates(t.ids, t.xy)
        gpu_csr_sorted(a, t.rects, dev)
    xy, present = a.export_state()
    assert present.sum() == n and not present[n:].any()
    np.testing.assert_array_equal(xy[:n], t.xy)
    with pytest.raises(mqr.MqrError):
        mqr.mqr_export_state(a.ctx, n)                               # buffers smaller than max_objects
    b = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=64, max_objects=n + 17)
    b.import_state(xy, present)
    with pytest.raises(mqr.MqrError):
        b.import_state(xy[:n], present[:n])                          # not max_objects entries
    rects = t.rects
    want = oracle.join_grid(st, rects, cell_side=0.005)
    assert_same_csr(gpu_csr_sorted(b, rects, dev), want, "restored")
    assert_same_csr(gpu_csr_sorted(a, rects, dev), want, "original")
    # a later tick's updates win over the restored state, on both
    t = w.next_tick()
    half = t.ids[: n // 2]
    for idx in (a, b):
        idx.apply_updates(to_dev(half, dev), to_dev(t.xy[: n // 2], dev))
    st.apply_updates(half, t.xy[: n // 2])
    want = oracle.join_grid(st, t.rects, cell_side=0.005)
    assert_same_csr(gpu_csr_sorted(a, t.rects, dev), want, "original after updates")
    assert_same_csr(gpu_csr_sorted(b, t.rects, dev), want, "restored after updates")
    a.close()
    b.close()


@pytest.fixture
def disarm_hook():
    yield
    from paper_1411_3212_gb300 import mqr
    mqr.mqr_debug_fail_allocation(-1)              # never leave the hook armed for other tests


def test_injected_allocation_failure_is_reported_and_recoverable(disarm_hook):
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    n = 20_000
    rng = np.random.default_rng(2)
    xy = rng.random((n, 2)).astype(np.float32)
    ids = np.arange(n, dtype=np.uint32)
    # creation: the first device allocation fails -> OOM, nothing leaks, the next creation works
    mqr.mqr_debug_fail_allocation(0)
    with pytest.raises(mqr.MqrError) as exc:
        mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=32, max_objects=n)
    assert exc.value.status == mqr.MQR_ERR_OOM
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=32, max_objects=n)
    idx.apply_updates(to_dev(ids, dev), to_dev(xy, dev))
    small = workloads.squares_around(rng.random((100, 2)).astype(np.float32), 0.01)
    st = oracle_state(n, [(ids, xy)])
    assert_same_csr(gpu_csr_sorted(idx, small, dev), oracle.join_grid(st, small, cell_side=0.01), "first")
    # a tick whose buffers must grow: the growth fails -> OOM; the context stays usable
    big = workloads.squares_around(rng.random((30_000, 2)).astype(np.float32), 0.05)
    mqr.mqr_debug_fail_allocation(0)
    with pytest.raises(mqr.MqrError) as exc:
        idx.tick(to_dev(big, dev), kind="csr_sorted")
    assert exc.value.status == mqr.MQR_ERR_OOM
    mqr.mqr_debug_fail_allocation(-1)
    assert_same_csr(gpu_csr_sorted(idx, big, dev), oracle.join_grid(st, big, cell_side=0.02), "after OOM")
    assert_same_csr(gpu_csr_sorted(idx, small, dev), oracle.join_grid(st, small, cell_side=0.01), "small again")
    idx.close()
