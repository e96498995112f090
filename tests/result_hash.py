"""Order-independent per-query checksum of result pairs, on the host (test
infrastructure; the library never computes it).

The value of a result (query q, object id) is the output function of
splitmix64 (Steele, Lea & Flood 2014, with Vigna's published constants)
applied to (q << 32 | id); a query's checksum is the sum of its results'
values modulo 2^64.  The oracle computes the same checksum from its own Def. 1
result sets in C (count_grid(..., with_hash=True)), so comparing checksums
compares every query's complete id set without storing the oracle's lists."""
import numpy as np

_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


def mix64(z):
    """splitmix64's output function, elementwise on a uint64 array."""
    z = np.asarray(z, np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
    return z ^ (z >> np.uint64(31))


def per_query_hash(pairs_u32, offsets, chunk=1 << 25):
    """pairs_u32: uint32 [R, 2] (qidx, id) grouped by query in ascending
    qidx; offsets: uint64/int64 [Q + 1].  Returns uint64 [Q]."""
    off = np.asarray(offsets).astype(np.int64)
    Q = off.shape[0] - 1
    R = int(off[-1])
    vals = np.empty(R, np.uint64)
    for a in range(0, R, chunk):
        b = min(R, a + chunk)
        p = pairs_u32[a:b]
        key = (p[:, 0].astype(np.uint64) << np.uint64(32)) | p[:, 1].astype(np.uint64)
        vals[a:b] = mix64(key)
    out = np.zeros(Q, np.uint64)
    nz = np.nonzero(off[1:] > off[:-1])[0]
    if nz.size:
        with np.errstate(over="ignore"):
            out[nz] = np.add.reduceat(vals, off[nz])
    return out
