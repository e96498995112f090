"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
the oracle on the same seeded inputs, and compare."""
import numpy as np

import oracle


def torch_dev():
    import torch
    return torch, torch.device("cuda:0")


def to_dev(a, dev):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).to(dev)


def gpu_csr_sorted(idx, rects, dev):
    res, offs = idx.tick(to_dev(rects, dev), kind="csr_sorted")
    return offs.cpu().numpy().view(np.uint64), res.cpu().numpy().view(np.uint32).copy()


def gpu_pairs_as_csr(idx, rects, dev):
    """PAIRS output (unsorted inside a query) -> sorted CSR on the host."""
    res, offs = idx.tick(to_dev(rects, dev), kind="pairs")
    p = res.cpu().numpy().view(np.uint32)
    off = offs.cpu().numpy().view(np.uint64)
    Q = rects.shape[0]
    # grouped by query in ascending qidx
    assert np.all(np.diff(p[:, 0].astype(np.int64)) >= 0)
    assert off[-1] == p.shape[0]
    counts = np.bincount(p[:, 0], minlength=Q) if p.shape[0] else np.zeros(Q, np.int64)
    assert np.array_equal(np.diff(off.astype(np.int64)), counts)
    ids = p[:, 1].copy()
    for q in range(Q):
        a, b = int(off[q]), int(off[q + 1])
        ids[a:b] = np.sort(ids[a:b])
    return off, ids


def oracle_state(nmax, updates):
    st = oracle.State(nmax)
    for ids, xy in updates:
        st.apply_updates(ids, xy)
    return st


def assert_same_csr(got, want, what=""):
    go, gi = got
    wo, wi = want
    assert go.shape == wo.shape, what
    if not np.array_equal(go, wo):
        q = int(np.nonzero(go != wo)[0][0])
        raise AssertionError("%s offsets differ first at query %d: %d vs %d" % (what, q, go[q], wo[q]))
    if not np.array_equal(gi, wi):
        k = int(np.nonzero(gi != wi)[0][0])
        q = int(np.searchsorted(wo, k, side="right") - 1)
        raise AssertionError("%s ids differ at %d (query %d)" % (what, k, q))
