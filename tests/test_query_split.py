"""The query-splitting argument behind the candidate pass, on the host with
the oracle's own Morton code (Alg. 1, GPUcalculateMortonHash) and its mapping
g (Def. "Mapping functions"), independently of the CUDA path.

A query's cell rectangle is cut into at most 3 x 3 aligned blocks of side
2^k, k the smallest value with 2^(k+1) >= its extent; the candidate leaves of
a (query, block) pair are the leaves whose Morton interval meets
[z(lower-left), z(upper-right)] of the query's part of the block.  That is
exact because the Morton codes of an axis-aligned cell rectangle lie between
those of its two corners (bit interleaving is increasing in each coordinate),
so every leaf that meets the query inside the block meets that interval; in
particular the block holding the lower-left corner of leaf and query (the
block that keeps the subquery, Sec. 5.3 Fig. 8) lists the leaf."""
import numpy as np

import oracle
from paper_1411_3212_gb300 import workloads


def test_rectangle_codes_lie_between_corner_codes():
    g = 16
    codes = np.array([[oracle.morton(i, j) for j in range(g)] for i in range(g)], dtype=np.int64)
    for i0 in range(g):
        for i1 in range(i0, g):
            for j0 in range(g):
                for j1 in range(j0, g):
                    sub = codes[i0:i1 + 1, j0:j1 + 1]
                    assert sub.min() == codes[i0, j0] and sub.max() == codes[i1, j1]


def _blocks(i0, i1, j0, j1):
    e = max(i1 - i0, j1 - j0) + 1
    k = 0 if e <= 1 else int(e - 1).bit_length() - 1          # 2^(k+1) >= e > 2^k
    side = 1 << k
    out = []
    for bj in range(j0 >> k, (j1 >> k) + 1):
        for bi in range(i0 >> k, (i1 >> k) + 1):
            ci0, cj0 = max(i0, bi << k), max(j0, bj << k)
            ci1, cj1 = min(i1, (bi << k) + side - 1), min(j1, (bj << k) + side - 1)
            out.append(((bi << k, bj << k, side), oracle.morton(ci0, cj0), oracle.morton(ci1, cj1)))
    return out


def test_every_subquery_leaf_lies_in_its_blocks_trimmed_interval():
    rng = np.random.default_rng(5)
    xy = workloads.HotspotWalk(n=20_000, q=1, hotspots=6, seed=3).next_tick().xy
    st = oracle.State(xy.shape[0])
    st.apply_updates(np.arange(xy.shape[0], dtype=np.uint32), xy)
    leaves = oracle.quadtree(np.sort(oracle.keys(st)), 16)
    lo = (leaves["z"].astype(np.int64) << (2 * (15 - leaves["level"].astype(np.int64))))
    hi = lo + (np.int64(1) << (2 * (15 - leaves["level"].astype(np.int64)))) - 1
    sc = oracle.scale(0.0, 1.0)
    centres = xy[rng.integers(0, xy.shape[0], 300)]
    sides = np.exp(rng.uniform(np.log(0.0005), np.log(0.05), 300)).astype(np.float32)
    rects = workloads.squares_around(centres, sides)
    trimmed_total = whole_total = 0
    for r in rects:
        meet, _ = oracle.subqueries(leaves, r, skip_empty=False)
        i0, i1 = oracle.cell(float(r[0]), 0.0, sc), oracle.cell(float(r[2]), 0.0, sc)
        j0, j1 = oracle.cell(float(r[1]), 0.0, sc), oracle.cell(float(r[3]), 0.0, sc)
        blocks = _blocks(i0, i1, j0, j1)
        assert len(blocks) <= 9
        for li in meet:
            z0 = int(lo[li])
            bi0 = bj0 = 0
            for b in range(15):                                 # de-interleave the leaf's first cell
                bi0 |= ((z0 >> (2 * b)) & 1) << b
                bj0 |= ((z0 >> (2 * b + 1)) & 1) << b
            ci, cj = max(bi0, i0), max(bj0, j0)                 # lower-left corner of leaf and query
            owner = [blk for blk in blocks
                     if blk[0][0] <= ci < blk[0][0] + blk[0][2] and blk[0][1] <= cj < blk[0][1] + blk[0][2]]
            assert len(owner) == 1
            _, zlo, zhi = owner[0]
            assert lo[li] <= zhi and hi[li] >= zlo
        for (bi, bj, side), zlo, zhi in blocks:
            blo = oracle.morton(bi, bj)
            bhi = blo + side * side - 1
            assert blo <= zlo <= zhi <= bhi                      # a sub-interval of the block's
            trimmed_total += int(np.count_nonzero((lo <= zhi) & (hi >= zlo)))
            whole_total += int(np.count_nonzero((lo <= bhi) & (hi >= blo)))
    assert trimmed_total < whole_total
