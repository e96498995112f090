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


def expand_runs(elems, sorted_ids):
    """Covering-compressed elements (uint32[E, 2]) -> (qidx, id) pairs, in
    element order: a pair (q, id) stays, a run (q | 2^31, first) (count, 0)
    becomes (q, sorted_ids[first + j]) for j < count."""
    e = np.asarray(elems, dtype=np.uint32).reshape(-1, 2)
    run = (e[:, 0] & 0x80000000) != 0
    heads = np.nonzero(run)[0]
    counts = np.ones(e.shape[0], np.int64)
    counts[heads] = e[heads + 1, 0]
    counts[heads + 1] = 0
    total = int(counts.sum())
    q = np.repeat(e[:, 0] & 0x7fffffff, counts)
    cstart = np.concatenate([[0], np.cumsum(counts)[:-1]])
    first = np.where(run, e[:, 1], 0).astype(np.int64)
    pos = np.repeat(first - cstart, counts) + np.arange(total)
    vals = np.repeat(e[:, 1], counts)
    in_run = np.repeat(run, counts)
    vals[in_run] = sorted_ids[pos[in_run]]
    return np.stack([q, vals], axis=1).astype(np.uint32), counts


def gpu_runs_as_csr(idx, rects, dev):
    """RUNS output -> sorted CSR on the host (expanded with the tick's sorted
    ids); also checks the element offsets and the grouping by query."""
    res, offs = idx.tick(to_dev(rects, dev), kind="runs")
    e = res.cpu().numpy().view(np.uint32)
    eoff = offs.cpu().numpy().view(np.uint64).astype(np.int64)
    Q = rects.shape[0]
    assert eoff[-1] == e.shape[0]
    _, sid = idx.sorted_objects()
    pairs, counts = expand_runs(e, sid)
    # every element lies in its query's element range
    qe = (e[:, 0] & 0x7fffffff).astype(np.int64)
    heads = np.nonzero((e[:, 0] & 0x80000000) != 0)[0]
    assert np.all(e[heads + 1, 1] == 0) and np.all(e[heads + 1, 0] > 0)
    qe[heads + 1] = qe[heads]                                               # a run's second element
    assert np.array_equal(np.searchsorted(eoff, np.arange(e.shape[0]), side="right") - 1, qe)
    per_q = np.add.reduceat(np.append(counts, 0), eoff[:-1]) if Q else np.zeros(0, np.int64)
    per_q[eoff[:-1] == eoff[1:]] = 0
    off = np.concatenate([[0], np.cumsum(per_q)]).astype(np.uint64)
    ids = pairs[:, 1].copy()
    for q in range(Q):
        a, b = int(off[q]), int(off[q + 1])
        ids[a:b] = np.sort(ids[a:b])
    return off, ids, e


def gpu_atomic_as_csr(idx, rects, dev):
    """PAIRS_ATOMIC output (unordered pairs) -> sorted CSR on the host."""
    res, _ = idx.tick(to_dev(rects, dev), kind="pairs_atomic")
    p = res.cpu().numpy().view(np.uint32)
    Q = rects.shape[0]
    order = np.lexsort((p[:, 1], p[:, 0]))
    p = p[order]
    counts = np.bincount(p[:, 0], minlength=Q) if p.shape[0] else np.zeros(Q, np.int64)
    assert counts.shape[0] == Q
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.uint64)
    return off, p[:, 1].copy()
