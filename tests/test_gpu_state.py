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


@pytest.fixture
def disarm_stall():
    yield
    from paper_1411_3212_gb300 import mqr
    mqr.mqr_debug_stall_scan(False)                # never leave the hook armed for other tests


def test_bounded_wait_times_out_and_the_context_recovers(disarm_stall):
    """The result-count scan's look-back waits are bounded: with the test hook
    armed, the scan's first tile withholds its status and the other tiles'
    waits give up after 1 ms; the tick reports MQR_ERR_TIMEOUT and writes no
    output, and the following ticks are exact (the hook disarms itself)."""
    import time
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    n, Q = 40_000, 8_000
    rng = np.random.default_rng(17)
    xy = rng.random((n, 2)).astype(np.float32)
    ids = np.arange(n, dtype=np.uint32)
    rects = workloads.squares_around(xy[rng.integers(0, n, Q)], 0.02)
    st = oracle_state(n, [(ids, xy)])
    want = oracle.join_grid(st, rects, cell_side=0.02)
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=32, max_objects=n)
    idx.apply_updates(to_dev(ids, dev), to_dev(xy, dev))
    assert_same_csr(gpu_csr_sorted(idx, rects, dev), want, "before")
    s = idx.stats()
    assert s["n_sub_intersecting"] + s["n_covering_runs"] > 4 * 2048      # several scan tiles wait
    rects_d = to_dev(rects, dev)
    out = torch.full((2 * int(want[0][-1]) + 2048,), -1, dtype=torch.int32, device=dev)
    mqr.mqr_debug_stall_scan(True)
    t0 = time.perf_counter()
    status, _ = mqr.mqr_tick(idx.ctx, rects_d, Q, mqr.MQR_OUT_PAIRS, out, out.numel() * 4, check=False)
    dt = time.perf_counter() - t0
    assert status == mqr.MQR_ERR_TIMEOUT, mqr.mqr_last_error()
    assert "deadline" in mqr.mqr_last_error()
    assert dt < 1.0                                 # the 1 ms test limit, not the 2 s one
    assert bool((out == -1).all().item())           # the emit wrote nothing after the timeout
    # the hook disarmed itself and the context answers exactly again
    assert_same_csr(gpu_csr_sorted(idx, rects, dev), want, "after the timeout")
    status, cnt = mqr.mqr_tick(idx.ctx, rects_d, Q, mqr.MQR_OUT_PAIRS, out, out.numel() * 4)
    assert status == mqr.MQR_OK and cnt == int(want[0][-1])
    idx.close()
