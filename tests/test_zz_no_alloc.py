"""mqr_sort_objects_noalloc, the allocation-free Morton sort, against the
sorted objects the regular pipeline reports (mqr_get_sorted).

It exists for callers that cannot allocate device memory (embedders that own
all device memory, or latency-critical loops that cannot afford cudaMalloc's
synchronisation).  Two calls in a row, with different sizes, check that the
shared static scratch is cleared between calls.  This file is collected last
on purpose."""
import numpy as np
import pytest

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


def test_noalloc_sort_matches_pipeline_sort_twice():
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    mqr.load()
    cases = [workloads.HotspotWalk(n=200_000, q=1, hotspots=8, seed=11).next_tick().xy,
             workloads.uniform_points(70_001, np.random.default_rng(3))]
    cases[1][:500] = cases[1][0]                                  # ties
    for xy in cases:
        n = xy.shape[0]
        keys = torch.empty(n, dtype=torch.int32, device=dev)
        ids = torch.empty(n, dtype=torch.int32, device=dev)
        mqr.mqr_sort_objects_noalloc((0.0, 0.0, 1.0, 1.0), to_dev(xy, dev), n, keys, ids)
        want_k, want_i = reference_sorted(mqr, xy, dev)
        np.testing.assert_array_equal(keys.cpu().numpy().view(np.uint32), want_k)
        np.testing.assert_array_equal(ids.cpu().numpy().view(np.uint32), want_i)


def test_noalloc_rejects_oversize():
    torch, dev = torch_dev()
    from paper_1411_3212_gb300 import mqr
    n = mqr.MQR_NOALLOC_MAX_OBJECTS + 1
    xy = torch.zeros((n, 2), dtype=torch.float32, device=dev)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    with pytest.raises(mqr.MqrError, match="MQR_NOALLOC_MAX_OBJECTS"):
        mqr.mqr_sort_objects_noalloc((0.0, 0.0, 1.0, 1.0), xy, n, out, out)
