// k_query.cu -- query indexing: splitting every query into subqueries over the
// leaves it meets (Def. "Mapping functions", function g), intersecting vs
// covering classification, the two-pass count/scan/write scheme of Sec. 5.3
// ("Indexing moving objects and queries"), and the grouping of intersecting
// subqueries by leaf (Sec. 5.3 "Sorting", replaced by a counting scatter).
//
// The leaves of a tick are contiguous Morton intervals [lo, hi] of the
// l_max grid, sorted.  Every query is cut into at most 3 x 3 aligned blocks;
// the leaves meeting a block are one contiguous range of the leaf table,
// found through a coarse lookup table (the paper's z_map, at a fixed coarse
// level).  All (query, candidate leaf) pairs are then classified in one flat,
// load-balanced pass (no per-query serial walk), and a leaf larger than a
// block is kept once, by the block holding the lower-left corner of its
// intersection with the query (the paper's minimal-grid-coordinates rule).
#include <algorithm>

#include "mqr_internal.cuh"

namespace mqr {

struct QCells {
    uint32_t i0, i1, j0, j1;
};

// Def. 1: a NaN corner or an inverted side admits no point.
__device__ __forceinline__ bool query_cells(float4 r, float x0, float y0, float sx, float sy, QCells &c) {
    if (isnan(r.x) || isnan(r.y) || isnan(r.z) || isnan(r.w)) return false;
    if (r.x > r.z || r.y > r.w) return false;
    c.i0 = cell_of(r.x, x0, sx);
    c.i1 = cell_of(r.z, x0, sx);
    c.j0 = cell_of(r.y, y0, sy);
    c.j1 = cell_of(r.w, y0, sy);
    return true;
}

// ---------------------------------------------------------------------------
// Coarse Morton lookup table: the paper's z_map (Sec. 5.3, "Building a lookup
// table to map coordinates to cells") kept at the fixed coarse level kZLevel
// instead of l_deep (4^15 entries would not fit): zmap[c] is the first leaf
// whose Morton interval ends at or after the first code of coarse cell c, and
// zmap[4^kZLevel] = L.  A lookup then only searches the leaves of one coarse
// cell.
// ---------------------------------------------------------------------------
__global__ void zmap_kernel(const uint32_t *__restrict__ leaf_hi, const Info *info,
                            uint32_t *__restrict__ zmap) {
    const uint32_t L = (uint32_t)info->n_leaves;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c <= kZCells; c += gridDim.x * blockDim.x) {
        if (c == kZCells) {
            zmap[c] = L;
            continue;
        }
        const uint32_t z = c << kZShift;
        uint32_t a = 0, b = L;
        while (a < b) {
            uint32_t m = (a + b) >> 1;
            if (__ldg(leaf_hi + m) >= z) b = m; else a = m + 1;
        }
        zmap[c] = a;
    }
}

// First leaf whose interval ends at or after code z1, and the same for z2
// (L if none), the two binary searches advancing together so that their
// dependent loads overlap.
__device__ __forceinline__ void leaves_at_or_after2(uint32_t z1, uint32_t z2, const uint32_t *__restrict__ leaf_hi,
                                                    const uint32_t *__restrict__ zmap, uint32_t &r1, uint32_t &r2) {
    uint32_t a1 = __ldg(zmap + (z1 >> kZShift)), b1 = __ldg(zmap + (z1 >> kZShift) + 1);
    uint32_t a2 = __ldg(zmap + (z2 >> kZShift)), b2 = __ldg(zmap + (z2 >> kZShift) + 1);
    while (a1 < b1 || a2 < b2) {
        const uint32_t m1 = (a1 + b1) >> 1, m2 = (a2 + b2) >> 1;
        const uint32_t v1 = a1 < b1 ? __ldg(leaf_hi + m1) : 0u;
        const uint32_t v2 = a2 < b2 ? __ldg(leaf_hi + m2) : 0u;
        if (a1 < b1) { if (v1 >= z1) b1 = m1; else a1 = m1 + 1; }
        if (a2 < b2) { if (v2 >= z2) b2 = m2; else a2 = m2 + 1; }
    }
    r1 = a1;
    r2 = a2;
}

// Query splitting works on aligned blocks of side 2^k cells, k the smallest
// value with 2^(k+1) >= the query's larger extent, so that a query meets at
// most 3 x 3 blocks.  The leaves meeting one block are a contiguous range of
// the leaf table (leaves and blocks are both aligned quadtree quadrants), and
// so are those meeting the query's part of the block.
__device__ __forceinline__ uint32_t block_log2(uint32_t i0, uint32_t i1, uint32_t j0, uint32_t j1) {
    const uint32_t e = max(i1 - i0, j1 - j0) + 1u;
    return e <= 1u ? 0u : 31u - __clz(e - 1u);       // = ceil(log2 e) - 1
}

__device__ __forceinline__ void unpack_cells(uint2 qc, uint32_t &i0, uint32_t &i1, uint32_t &j0, uint32_t &j1) {
    i0 = qc.x & 0xffffu; i1 = qc.x >> 16; j0 = qc.y & 0xffffu; j1 = qc.y >> 16;
}

// Candidate classification: 0 = no subquery, 1 = intersecting, 2 = covering.
// A leaf of block `blo` yields a subquery of the query iff its box meets the
// query's cell rectangle and the lower-left corner of that intersection lies
// in this block (so that a leaf larger than the block is emitted once: the
// paper's rule of keeping the subquery with the minimal grid coordinates,
// Sec. 5.3 Fig. 8).  Covering iff the leaf's cells lie strictly inside the
// rectangle on both axes (Def. "Mapping functions"): then every object of the
// leaf passes the FP32 test of Def. 1, the cell function being monotone.
// blk: the block's lower-left cell (i | j << 16); box: the leaf's lower-left
// cell (i | j << 16) and the log2 of its side in cells.
__device__ __forceinline__ int classify(uint32_t i0, uint32_t i1, uint32_t j0, uint32_t j1, uint32_t k,
                                        uint32_t blk, uint2 box) {
    const uint32_t bi0 = box.x & 0xffffu, bj0 = box.x >> 16;
    const uint32_t bi1 = bi0 + (1u << box.y) - 1u, bj1 = bj0 + (1u << box.y) - 1u;
    if (bi1 < i0 || bi0 > i1 || bj1 < j0 || bj0 > j1) return 0;
    const uint32_t ci = max(bi0, i0), cj = max(bj0, j0);
    const uint32_t Bi0 = blk & 0xffffu, Bj0 = blk >> 16;
    if (ci < Bi0 || ci > Bi0 + (1u << k) - 1u || cj < Bj0 || cj > Bj0 + (1u << k) - 1u) return 0;
    return (bi0 > i0 && bi1 < i1 && bj0 > j0 && bj1 < j1) ? 2 : 1;
}

// ---------------------------------------------------------------------------
// a5 + a6: per query, its blocks and their leaf ranges ("pairs") and the
// number of candidate leaves; single-pass scans give pair and candidate
// offsets (the paper's two-pass count / exclusive scan / write scheme, with
// the write of the pair records fused after the scan).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kQBThreads)
query_blocks_kernel(const float4 *__restrict__ rects, uint32_t Q, float x0, float y0, float sx, float sy,
                    Worlds worlds, const uint32_t *__restrict__ leaf_lo, const uint32_t *__restrict__ leaf_hi,
                    const uint32_t *__restrict__ zmap, uint2 *__restrict__ qcells,
                    unsigned long long *__restrict__ cand_off, uint32_t *__restrict__ pair_q,
                    uint32_t *__restrict__ pair_first, uint32_t *__restrict__ pair_blo,
                    unsigned long long *__restrict__ pair_off, uint32_t *__restrict__ qpair,
                    uint32_t *__restrict__ tile_p0, unsigned long long tile_cap, uint32_t *status_p,
                    unsigned long long *status_c, uint32_t *tile_counter, Info *info) {
    // one thread per (query, block slot): kQBQueries queries x 9 slots per block
    __shared__ uint32_t s_scan32[kQBThreads / 32 + 1];
    __shared__ unsigned long long s_scan64[kQBThreads / 32 + 1];
    __shared__ uint32_t s_tile, s_pp;
    __shared__ unsigned long long s_pc;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint32_t L = (uint32_t)info->n_leaves;
    const uint32_t slot = (uint32_t)tid % 9u, ql = (uint32_t)tid / 9u;
    const uint32_t q = tile * kQBQueries + ql;
    const bool qvalid = ql < (uint32_t)kQBQueries && q < Q;

    uint32_t f = 0, cnt = 0, blk = 0;
    QCells c;
    const bool qok = qvalid && L > 0 && query_cells(rects[q], x0, y0, sx, sy, c);
    if (qok && worlds.n) {      // the query's cells inside its world's node
        const uint32_t w = world_of(q, worlds.q_base, worlds.n);
        c.i0 = world_cell(c.i0, w, worlds.bits, 0);
        c.i1 = world_cell(c.i1, w, worlds.bits, 0);
        c.j0 = world_cell(c.j0, w, worlds.bits, 1);
        c.j1 = world_cell(c.j1, w, worlds.bits, 1);
    }
    if (qok) {
        const uint32_t k = block_log2(c.i0, c.i1, c.j0, c.j1);
        const uint32_t bi = (c.i0 >> k) + slot % 3u, bj = (c.j0 >> k) + slot / 3u;
        if (slot == 0) qcells[q] = make_uint2(c.i0 | (c.i1 << 16), c.j0 | (c.j1 << 16));
        if (bi <= (c.i1 >> k) && bj <= (c.j1 >> k)) {
            blk = (bi << k) | ((bj << k) << 16);
            // the leaves meeting the query inside this block lie in the Morton
            // interval of the query's part of the block (an axis-aligned cell
            // rectangle's codes lie between those of its lower-left and
            // upper-right cells), a sub-interval of the block's
            const uint32_t side = (1u << k) - 1u;
            const uint32_t zlo = morton2(max(c.i0, bi << k), max(c.j0, bj << k));
            const uint32_t zhi = morton2(min(c.i1, (bi << k) + side), min(c.j1, (bj << k) + side));
            uint32_t g;
            leaves_at_or_after2(zlo, zhi, leaf_hi, zmap, f, g);
            if (f < L && __ldg(leaf_lo + f) <= zhi) {
                const uint32_t last = (g < L && __ldg(leaf_lo + g) <= zhi) ? g : g - 1u;
                cnt = last - f + 1u;
            }
        }
    }
    const uint32_t has = cnt > 0u ? 1u : 0u;
    uint32_t tot_p;
    unsigned long long tot_c;
    const uint32_t off_p = block_excl_scan<kQBThreads>(has, &tot_p, s_scan32);
    const unsigned long long off_c = block_excl_scan<kQBThreads>((unsigned long long)cnt, &tot_c, s_scan64);
    if (tid < 32) {
        const uint32_t pp = lookback_warp<uint32_t>(status_p, tile, tot_p, &info->err);
        if (tid == 0) s_pp = pp;
    } else if (tid < 64) {
        const unsigned long long pc = lookback_warp<unsigned long long>(status_c, tile, tot_c, &info->err);
        if (tid == 32) s_pc = pc;
    }
    __syncthreads();
    const uint32_t p = s_pp + off_p;
    const unsigned long long co = s_pc + off_c;
    if (qvalid && slot == 0) {
        cand_off[q] = co;
        qpair[q] = p;
    }
    if (has) {
        pair_q[p] = q;
        pair_first[p] = f;
        pair_blo[p] = blk;
        pair_off[p] = co;
        // warp tiles of 32 candidates whose first candidate falls in this pair
        for (unsigned long long t = (co + 31) >> 5; (t << 5) < co + cnt && t < tile_cap; ++t) tile_p0[t] = p;
    }
    if (tid == 0 && (tile + 1) * (uint32_t)kQBQueries >= Q) {
        const uint32_t np = s_pp + tot_p;
        const unsigned long long nc = s_pc + tot_c;
        cand_off[Q] = nc;
        qpair[Q] = np;
        pair_off[np] = nc;
        info->n_pairs = np;
        info->n_cand = nc;
    }
}

void launch_zmap(cudaStream_t st, const uint32_t *leaf_hi, const Info *info, uint32_t *zmap) {
    zmap_kernel<<<(kZCells + 1 + 255) / 256, 256, 0, st>>>(leaf_hi, info, zmap);
}

void launch_query_blocks(cudaStream_t st, const float4 *rects, uint32_t Q, float x0, float y0, float sx,
                         float sy, Worlds worlds, const uint32_t *leaf_lo, const uint32_t *leaf_hi, const uint32_t *zmap,
                         uint2 *qcells, unsigned long long *cand_off, uint32_t *pair_q,
                         uint32_t *pair_first, uint32_t *pair_blo, unsigned long long *pair_off,
                         uint32_t *qpair, uint32_t *tile_p0, unsigned long long tile_cap,
                         uint32_t *status_p, unsigned long long *status_c, uint32_t *tile_counter,
                         Info *info) {
    if (Q == 0) return;
    uint32_t tiles = (Q + kQBQueries - 1) / kQBQueries;
    query_blocks_kernel<<<tiles, kQBThreads, 0, st>>>(rects, Q, x0, y0, sx, sy, worlds, leaf_lo, leaf_hi, zmap,
                                                      qcells, cand_off, pair_q, pair_first, pair_blo,
                                                      pair_off, qpair, tile_p0, tile_cap, status_p,
                                                      status_c, tile_counter, info);
}

// ---------------------------------------------------------------------------
// a7: candidate leaves -> subquery records, in warp tiles of 32 consecutive
// candidates.  The pairs touching a tile are the 32 pairs from tile_p0[t] on
// (every pair has >= 1 candidate); lane j loads pair tile_p0[t] + j, the pair
// starts inside the tile are gathered in one bit mask, and the pair of lane L
// is found by a popcount.  Consecutive covering leaves of one pair inside one
// tile form one covering run (their objects are one contiguous range of the
// sorted objects).
// One pass classifies and places the records: a block takes chunks of
// kCandChunkTiles consecutive tiles in ticket order (each warp kCandWarpTiles
// of them), gathers the chunk's records in shared memory in tile order, finds
// the chunk's first record by a decoupled look-back over the chunks before
// it, and stores the records there, coalesced.  Record k: sub_q[k] = query,
// sub_leaf[k] = first leaf (bit 31 set for a covering run), sub_len[k] = run
// length (covering) or the record's row in its leaf's list (intersecting: the
// rank drawn from the leaf's counter leaf_nsub), sub_res[k] = result count
// (covering: the run's objects; intersecting: 0, filled by the filter).
// Records are in query-major order.  pair_rec[p] = the index of pair p's
// first record (or of the record after it, if p has none).
// ---------------------------------------------------------------------------
struct CandLane {
    bool valid;
    int code;          // 0 none, 1 intersecting, 2 covering
    bool cont;         // covering and continuing the run of the previous lane
    uint32_t q, leaf, p_rel;
    uint32_t po_j;     // lane j's pair: offset of its first candidate in the tile
    bool pj_starts;    // lane j's pair starts inside this tile
};

// The loads of a tile's pairs (lane j: pair tile_p0[t] + j), issued one tile
// ahead of their use so that two tiles' load chains overlap in each warp.
struct PairLoad {
    uint32_t p0, po, q, f, b;
};

__device__ __forceinline__ PairLoad pair_load(unsigned long long t, uint32_t npairs,
                                              const uint32_t *__restrict__ tile_p0,
                                              const uint32_t *__restrict__ pair_q,
                                              const uint32_t *__restrict__ pair_first,
                                              const uint32_t *__restrict__ pair_blo,
                                              const unsigned long long *__restrict__ pair_off) {
    PairLoad L;
    L.p0 = __ldg(tile_p0 + t);
    const uint32_t pj = L.p0 + (threadIdx.x & 31);
    L.q = L.f = L.b = 0;
    L.po = 0xffffffffu;
    if (pj < npairs) {
        L.po = (uint32_t)__ldg(pair_off + pj);
        L.q = __ldg(pair_q + pj);
        L.f = __ldg(pair_first + pj);
        L.b = __ldg(pair_blo + pj);
    }
    return L;
}

__device__ __forceinline__ CandLane cand_lane(unsigned long long t, unsigned long long ncand, uint32_t npairs,
                                              int covering, const PairLoad &L,
                                              const uint2 *__restrict__ qcells,
                                              const uint2 *__restrict__ leaf_box) {
    // candidate indices fit 32 bits (at most kMaxCandTiles tiles of 32)
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t c0 = (uint32_t)t << 5;
    const uint32_t pj = L.p0 + lane;
    const uint32_t q_j = L.q, f_j = L.f, b_j = L.b, po = L.po;
    CandLane r;
    r.pj_starts = pj < npairs && po >= c0 && po < c0 + 32u;
    r.po_j = r.pj_starts ? po - c0 : 0u;
    const uint32_t bit = (r.pj_starts && lane > 0) ? (1u << r.po_j) : 0u;
    const uint32_t start_mask = __reduce_or_sync(0xffffffffu, bit);
    uint32_t le;
    asm("mov.u32 %0, %%lanemask_le;" : "=r"(le));
    r.p_rel = __popc(start_mask & le);
    const uint32_t c = c0 + lane;
    r.valid = c < ncand;
    r.q = __shfl_sync(0xffffffffu, q_j, r.p_rel);
    const uint32_t first = __shfl_sync(0xffffffffu, f_j, r.p_rel);
    const uint32_t blo = __shfl_sync(0xffffffffu, b_j, r.p_rel);   // block corner
    const uint32_t pstart = __shfl_sync(0xffffffffu, po, r.p_rel);
    r.code = 0;
    r.leaf = 0;
    if (r.valid) {
        r.leaf = first + (c - pstart);
        uint32_t i0, i1, j0, j1;
        unpack_cells(__ldg(qcells + r.q), i0, i1, j0, j1);
        r.code = classify(i0, i1, j0, j1, block_log2(i0, i1, j0, j1), blo, __ldg(leaf_box + r.leaf));
        if (r.code == 2 && !covering) r.code = 1;
    }
    const int prev = __shfl_up_sync(0xffffffffu, r.code, 1);
    const bool is_start = r.valid && c == pstart;
    r.cont = r.code == 2 && lane > 0 && !is_start && prev == 2;
    return r;
}

__global__ void __launch_bounds__(256)
cand_write_kernel(int covering, const uint32_t *__restrict__ tile_p0, const uint32_t *__restrict__ pair_q,
                  const uint32_t *__restrict__ pair_first, const uint32_t *__restrict__ pair_blo,
                  const unsigned long long *__restrict__ pair_off, const uint2 *__restrict__ qcells,
                  const uint2 *__restrict__ leaf_box, const uint32_t *__restrict__ leaf_beg,
                  uint32_t *__restrict__ leaf_nsub, uint32_t *__restrict__ pair_rec,
                  uint32_t *__restrict__ sub_q, uint32_t *__restrict__ sub_leaf, uint32_t *__restrict__ sub_len,
                  uint32_t *__restrict__ sub_res, unsigned long long *status, uint32_t *chunk_counter, Caps caps,
                  Info *info) {
    constexpr int NW = 256 / 32;
    static_assert(kCandChunkTiles == NW * kCandWarpTiles, "a chunk is the block's warps' tiles");
    __shared__ uint4 s_rec[NW][kCandWarpTiles * 32];     // the warp's records, in tile order
    __shared__ uint32_t s_warp[NW];
    __shared__ uint32_t s_chunk;
    __shared__ unsigned long long s_prefix;
    __shared__ unsigned long long s_red[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 2) s_red[tid] = 0;
    __syncthreads();
    const unsigned long long ncand = info->n_cand;
    const uint32_t npairs = (uint32_t)info->n_pairs;
    const unsigned long long ntiles = (ncand + 31) >> 5;
    const unsigned long long nchunks = (ntiles + kCandChunkTiles - 1) / kCandChunkTiles;
    const uint32_t lt = lanemask_lt();
    uint4 *my = s_rec[warp];
    unsigned long long n_i = 0, n_c = 0;
    // every block takes the same branch (ntiles and the capacity are uniform)
    while (ntiles <= caps.cand_tiles) {
        if (tid == 0) s_chunk = atomicAdd(chunk_counter, 1u);
        __syncthreads();
        const uint32_t chunk = s_chunk;
        if (chunk >= nchunks) break;
        const unsigned long long t0 = (unsigned long long)chunk * kCandChunkTiles + warp * kCandWarpTiles;
        // prel[j]: the first record of the lane's pair starting in tile j,
        // counted from the warp's first record (~0u: no pair starts there)
        uint32_t prel[kCandWarpTiles];
        uint32_t wcnt = 0;
        // a record is stored one tile later, so that the latency of its leaf
        // counter atomic (or of its run's leaf bounds) overlaps the next
        // tile's loads and classification
        bool pend = false;
        uint32_t pend_pos = 0;
        uint4 pend_rec = make_uint4(0u, 0u, 0u, 0u);
        PairLoad cur{};
        if (t0 < ntiles) cur = pair_load(t0, npairs, tile_p0, pair_q, pair_first, pair_blo, pair_off);
#pragma unroll
        for (int j = 0; j < kCandWarpTiles; ++j) {
            const unsigned long long t = t0 + j;
            prel[j] = ~0u;
            if (t < ntiles) {                                   // warp-uniform
                PairLoad nxt = cur;
                if (j + 1 < kCandWarpTiles && t + 1 < ntiles)
                    nxt = pair_load(t + 1, npairs, tile_p0, pair_q, pair_first, pair_blo, pair_off);
                const CandLane r = cand_lane(t, ncand, npairs, covering, cur, qcells, leaf_box);
                const bool rec = r.code == 1 || (r.code == 2 && !r.cont);
                const uint32_t m = __ballot_sync(0xffffffffu, rec);
                const uint32_t notcont = __ballot_sync(0xffffffffu, !(r.valid && r.cont));
                if (r.pj_starts) prel[j] = wcnt + __popc(m & ((1u << r.po_j) - 1u));
                if (pend) my[pend_pos] = pend_rec;
                pend = false;
                if (r.code == 1) {
                    ++n_i;
                    pend = true;
                    pend_pos = wcnt + __popc(m & lt);
                    pend_rec = make_uint4(r.q, r.leaf, atomicAdd(leaf_nsub + r.leaf, 1u), 0u);
                } else if (r.code == 2) {
                    ++n_c;
                    if (!r.cont) {
                        const uint32_t after = notcont & ~(lt | (1u << lane));   // later lanes that end the run
                        const uint32_t end = after ? (uint32_t)(__ffs(after) - 1) : 32u;
                        const uint32_t len = end - lane;
                        pend = true;
                        pend_pos = wcnt + __popc(m & lt);
                        pend_rec = make_uint4(r.q, r.leaf | 0x80000000u, len,
                                              __ldg(leaf_beg + r.leaf + len) - __ldg(leaf_beg + r.leaf));
                    }
                }
                wcnt += __popc(m);
                cur = nxt;
            }
        }
        if (pend) my[pend_pos] = pend_rec;
        if (lane == 0) s_warp[warp] = wcnt;
        __syncthreads();
        uint32_t woff = 0, total = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const uint32_t v = s_warp[w];
            if (w < warp) woff += v;
            total += v;
        }
        if (warp == 0) {
            const unsigned long long pre =
                lookback_warp<unsigned long long>(status, chunk, (unsigned long long)total, &info->err);
            if (lane == 0) s_prefix = pre;
        }
        __syncthreads();
        const unsigned long long base = s_prefix + woff;
        for (uint32_t i = lane; i < wcnt; i += 32) {
            const unsigned long long k = base + i;
            if (k < caps.sub) {
                const uint4 v = my[i];
                sub_q[k] = v.x;
                sub_leaf[k] = v.y;
                sub_len[k] = v.z;
                sub_res[k] = v.w;
            }
        }
#pragma unroll
        for (int j = 0; j < kCandWarpTiles; ++j)
            if (prel[j] != ~0u) pair_rec[__ldg(tile_p0 + t0 + j) + lane] = (uint32_t)(base + prel[j]);
        if (tid == 0 && chunk + 1 == nchunks) info->n_sub = s_prefix + total;
        __syncthreads();            // s_chunk, s_warp, s_prefix and s_rec are reused by the next chunk
    }
    n_i = warp_sum(n_i); n_c = warp_sum(n_c);
    if (lane == 0) {
        if (n_i) atomicAdd(&s_red[0], n_i);
        if (n_c) atomicAdd(&s_red[1], n_c);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_red[0]) atomicAdd(&info->n_sub_i, s_red[0]);
        if (s_red[1]) atomicAdd(&info->n_sub_c, s_red[1]);
    }
}

void launch_candidates(cudaStream_t st, int grid_blocks, int covering, const uint32_t *tile_p0,
                       const uint32_t *pair_q, const uint32_t *pair_first, const uint32_t *pair_blo,
                       const unsigned long long *pair_off, const uint2 *qcells, const uint2 *leaf_box,
                       const uint32_t *leaf_beg, uint32_t *leaf_nsub, uint32_t *pair_rec, uint32_t *sub_q,
                       uint32_t *sub_leaf, uint32_t *sub_len, uint32_t *sub_res, unsigned long long *status,
                       uint32_t *chunk_counter, Caps caps, Info *info) {
    cand_write_kernel<<<grid_blocks, 256, 0, st>>>(covering, tile_p0, pair_q, pair_first, pair_blo, pair_off,
                                                   qcells, leaf_box, leaf_beg, leaf_nsub, pair_rec, sub_q,
                                                   sub_leaf, sub_len, sub_res, status, chunk_counter, caps, info);
}

// ---------------------------------------------------------------------------
// a8: per-leaf scans.  For leaf l with n objects and s intersecting
// subqueries: its subquery list starts at leaf_sub_off[l]; its bitmap (s rows
// of ceil(n/32) words, row-major: the linearized layout of Sec. 5.4) starts
// at leaf_word_off[l]; its filter work items (ceil(n/256) object chunks x
// ceil(s/32) subquery groups) start at leaf_item_off[l].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kLeafScanThreads)
leaf_scan_kernel(const uint32_t *__restrict__ leaf_beg, const uint32_t *__restrict__ leaf_nsub,
                 uint32_t *__restrict__ leaf_sub_off, uint32_t *__restrict__ leaf_word_off,
                 uint32_t *__restrict__ leaf_item_off,
                 uint32_t *__restrict__ item_leaf, uint32_t *status3, uint32_t num_tiles,
                 uint32_t *tile_counter, Caps caps, Info *info) {
    constexpr int NW = kLeafScanThreads / 32;
    __shared__ uint3 s_warp[NW];
    __shared__ uint32_t s_tile, s_p[3];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t L = (uint32_t)info->n_leaves;
    // the grid is a few blocks per SM; each takes tiles from the counter in
    // order (a tile's look-back only waits for tiles already taken)
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        const uint32_t base = tile * kLeafScanTile;
        if (base >= L) break;
        const uint32_t lb = base + tid * kLeafScanItems;

        uint32_t ns[kLeafScanItems], nw[kLeafScanItems], ni[kLeafScanItems];
        uint32_t t_s = 0, t_w = 0, t_i = 0;
        unsigned long long objs = 0, tests = 0;
#pragma unroll
        for (int e = 0; e < kLeafScanItems; ++e) {
            uint32_t l = lb + e;
            ns[e] = nw[e] = ni[e] = 0;
            if (l < L) {
                uint32_t sq = leaf_nsub[l];
                uint32_t n = leaf_beg[l + 1] - leaf_beg[l];
                ns[e] = sq;
                nw[e] = sq * ((n + 31u) >> 5);
                ni[e] = sq ? ((n + 255u) >> 8) * ((sq + 31u) >> 5) : 0u;
                if (sq) objs += (unsigned long long)n * ((sq + 31u) >> 5);
                tests += (unsigned long long)n * sq;                 // containment tests of the leaf
            }
            t_s += ns[e]; t_w += nw[e]; t_i += ni[e];
        }
        // one block scan of the three counts together
        uint32_t i_s = warp_incl_scan(t_s), i_w = warp_incl_scan(t_w), i_i = warp_incl_scan(t_i);
        if (lane == 31) s_warp[warp] = make_uint3(i_s, i_w, i_i);
        objs = warp_sum(objs);
        tests = warp_sum(tests);
        if (lane == 0 && objs) atomicAdd(&info->n_item_objs, objs);
        if (lane == 0 && tests) atomicAdd(&info->n_tests, tests);
        __syncthreads();
        uint32_t w_s = 0, w_w = 0, w_i = 0, tot_s = 0, tot_w = 0, tot_i = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const uint3 v = s_warp[w];
            if (w < warp) { w_s += v.x; w_w += v.y; w_i += v.z; }
            tot_s += v.x; tot_w += v.y; tot_i += v.z;
        }
        uint32_t o_s = w_s + i_s - t_s, o_w = w_w + i_w - t_w, o_i = w_i + i_i - t_i;
        if (tid < 96) {
            const uint32_t agg = warp == 0 ? tot_s : (warp == 1 ? tot_w : tot_i);
            const uint32_t pre = lookback_warp<uint32_t>(status3 + (size_t)warp * num_tiles, tile, agg, &info->err);
            if (lane == 0) s_p[warp] = pre;
        }
        __syncthreads();
        o_s += s_p[0]; o_w += s_p[1]; o_i += s_p[2];
#pragma unroll
        for (int e = 0; e < kLeafScanItems; ++e) {
            uint32_t l = lb + e;
            if (l < L) {
                leaf_sub_off[l] = o_s;
                leaf_word_off[l] = o_w;
                leaf_item_off[l] = o_i;
                for (uint32_t t = 0; t < ni[e]; ++t)
                    if (o_i + t < caps.items) item_leaf[o_i + t] = l;
            }
            o_s += ns[e]; o_w += nw[e]; o_i += ni[e];
        }
        if (tid == 0 && base + kLeafScanTile >= L) {
            leaf_sub_off[L] = s_p[0] + tot_s;
            leaf_word_off[L] = s_p[1] + tot_w;
            leaf_item_off[L] = s_p[2] + tot_i;
            info->n_words = s_p[1] + tot_w;
            info->n_items = s_p[2] + tot_i;
        }
        __syncthreads();            // s_tile, s_warp and s_p are reused by the next tile
    }
}

void launch_leaf_scan(cudaStream_t st, int num_sms, uint32_t nmax, const uint32_t *leaf_beg,
                      const uint32_t *leaf_nsub, uint32_t *leaf_sub_off, uint32_t *leaf_word_off,
                      uint32_t *leaf_item_off, uint32_t *item_leaf,
                      uint32_t *status3, uint32_t *tile_counter, Caps caps, Info *info) {
    if (nmax == 0) return;
    uint32_t tiles = (nmax + kLeafScanTile - 1) / kLeafScanTile;
    const uint32_t grid = std::min<uint32_t>(tiles, (uint32_t)num_sms * 2u);
    leaf_scan_kernel<<<grid, kLeafScanThreads, 0, st>>>(leaf_beg, leaf_nsub, leaf_sub_off,
                                                        leaf_word_off, leaf_item_off,
                                                        item_leaf, status3, tiles, tile_counter, caps,
                                                        info);
}

// ---------------------------------------------------------------------------
// a8: every intersecting record takes its place in its leaf's list: isub[
// leaf_sub_off[leaf] + row] = k, with row the rank the candidate pass drew
// from the leaf's counter (kept in sub_len: the record's bitmap row in the
// leaf).  Four records per thread per step, their loads issued together.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
leaf_lists_kernel(const uint32_t *__restrict__ sub_leaf, const uint32_t *__restrict__ sub_len,
                  const uint32_t *__restrict__ leaf_sub_off, uint32_t *__restrict__ isub, Caps caps,
                  const Info *info) {
    constexpr int U = 4;
    const unsigned long long nsub = info->n_sub;
    if (nsub > caps.sub || info->n_sub_i > caps.sub_i) return;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long k0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k0 < nsub;
         k0 += U * stride) {
        uint32_t leaf[U], row[U], off[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const unsigned long long k = k0 + u * stride;
            leaf[u] = k < nsub ? __ldg(sub_leaf + k) : 0x80000000u;
            row[u] = k < nsub ? __ldg(sub_len + k) : 0u;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (!(leaf[u] & 0x80000000u)) off[u] = __ldg(leaf_sub_off + leaf[u]);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (!(leaf[u] & 0x80000000u)) isub[off[u] + row[u]] = (uint32_t)(k0 + u * stride);
    }
}

void launch_leaf_lists(cudaStream_t st, int grid_blocks, const uint32_t *sub_leaf, const uint32_t *sub_len,
                       const uint32_t *leaf_sub_off, uint32_t *isub, Caps caps, const Info *info) {
    leaf_lists_kernel<<<grid_blocks, 256, 0, st>>>(sub_leaf, sub_len, leaf_sub_off, isub, caps, info);
}

}  // namespace mqr
