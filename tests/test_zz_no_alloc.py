"""mqr_sort_objects_noalloc, the allocation-free Morton sort, against the
regular pipeline's sorted objects (mqr_get_sorted) and against the oracle
(its Morton keys at l_max = 15 and a stable sort of them, Alg. 1).

The entry point serves callers that cannot allocate device memory: embedders
that own all device memory (a fixed budget or their own pool) and
latency-critical loops that cannot afford the device-wide synchronisation a
cudaMalloc or cudaFree may cause.  Its scratch is one fixed static device
array, shared by every call: calls in a row with different sizes check that
it is cleared between calls, at sizes from 0 up to the limit
MQR_NOALLOC_MAX_OBJECTS.  This file is collected last on purpose."""
import numpy as np
import pytest

import oracle
from paper_1411_3212_gb300 import workloads
from tests.gpu_util import to_dev, torch_dev

pytestmark = pytest.mark.gpu


def reference_sorted(mqr, xy, dev):
    n = xy.shape[0]
    idx = mqr.Index(bounds=(0.0, 0.0, 1.0, 1.0), leaf_cap=64, max_objects=n)
    idx.apply_updates(to_dev(np.arange(n, dtype=np.uint32), dev), to_dev(xy, dev))
    idx.tick(to_dev(np.zeros((0, 4), np.float32), dev), kind="count")
    keys, ids = idx.sorted_objects()
    idx.close()
    return keys, ids


def oracle_sorted(xy):
    n = xy.shape[0]
    st = oracle.State(n)
    st.apply_updates(np.arange(n, dtype=np.uint32), xy)
    k = oracle.keys(st)
    order = np.argsort(k, kind="stable")
    return k[order], order.astype(np.uint32)


def test_noalloc_sort_matches_pipeline_and_oracle_in_a_row():
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    mqr.load()
    nmax = mqr.MQR_NOALLOC_MAX_OBJECTS
    rng = np.random.default_rng(3)
    cases = [workloads.HotspotWalk(n=200_000, q=1, hotspots=8, seed=11).next_tick().xy,
             workloads.uniform_points(70_001, rng),
             workloads.HotspotWalk(n=nmax, q=1, hotspots=4, seed=12).next_tick().xy,   # exactly the limit
             workloads.uniform_points(5, rng)]
    cases[1][:500] = cases[1][0]                                  # ties
    cases[2][-3000:] = cases[2][7]                                # ties at the limit
    for xy in cases:
        n = xy.shape[0]
        keys = torch.empty(n, dtype=torch.int32, device=dev)
        ids = torch.empty(n, dtype=torch.int32, device=dev)
        mqr.mqr_sort_objects_noalloc((0.0, 0.0, 1.0, 1.0), to_dev(xy, dev), n, keys, ids)
        got_k, got_i = keys.cpu().numpy().view(np.uint32), ids.cpu().numpy().view(np.uint32)
        want_k, want_i = oracle_sorted(xy)
        np.testing.assert_array_equal(got_k, want_k)
        np.testing.assert_array_equal(got_i, want_i)
        pipe_k, pipe_i = reference_sorted(mqr, xy, dev)
        np.testing.assert_array_equal(got_k, pipe_k)
        np.testing.assert_array_equal(got_i, pipe_i)
    # n = 0: nothing to do, the outputs are untouched
    out = torch.full((4,), 7, dtype=torch.int32, device=dev)
    mqr.mqr_sort_objects_noalloc((0.0, 0.0, 1.0, 1.0), to_dev(np.zeros((0, 2), np.float32), dev), 0, out, out)
    assert out.cpu().tolist() == [7, 7, 7, 7]


def test_noalloc_rejects_oversize():
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    n = mqr.MQR_NOALLOC_MAX_OBJECTS + 1
    xy = torch.zeros((n, 2), dtype=torch.float32, device=dev)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    with pytest.raises(mqr.MqrError, match="MQR_NOALLOC_MAX_OBJECTS"):
        mqr.mqr_sort_objects_noalloc((0.0, 0.0, 1.0, 1.0), xy, n, out, out)
