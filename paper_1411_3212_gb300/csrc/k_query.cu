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

// First leaf whose interval ends at or after code z (L if none).
__device__ __forceinline__ uint32_t leaf_at_or_after(uint32_t z, const uint32_t *__restrict__ leaf_hi,
                                                     const uint32_t *__restrict__ zmap) {
    const uint32_t c = z >> kZShift;
    uint32_t a = __ldg(zmap + c), b = __ldg(zmap + c + 1);
    while (a < b) {
        uint32_t m = (a + b) >> 1;
        if (__ldg(leaf_hi + m) >= z) b = m; else a = m + 1;
    }
    return a;
}

// Query splitting works on aligned blocks of side 2^k cells, k the smallest
// value with 2^(k+1) >= the query's larger extent, so that a query meets at
// most 3 x 3 blocks.  The leaves meeting one block are a contiguous range of
// the leaf table (leaves and blocks are both aligned quadtree quadrants).
__device__ __forceinline__ uint32_t block_log2(uint32_t i0, uint32_t i1, uint32_t j0, uint32_t j1) {
    const uint32_t e = max(i1 - i0, j1 - j0) + 1u;
    uint32_t k = 0;
    while ((2u << k) < e) ++k;
    return k;
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
__device__ __forceinline__ int classify(uint32_t i0, uint32_t i1, uint32_t j0, uint32_t j1, uint32_t k,
                                        uint32_t blo, uint32_t lo, uint32_t hi) {
    const uint32_t span = hi - lo + 1u;
    const uint32_t s = (31u - __clz(span)) >> 1;
    const uint32_t bi0 = compact15(lo), bj0 = compact15(lo >> 1);
    const uint32_t bi1 = bi0 + (1u << s) - 1u, bj1 = bj0 + (1u << s) - 1u;
    if (bi1 < i0 || bi0 > i1 || bj1 < j0 || bj0 > j1) return 0;
    const uint32_t ci = max(bi0, i0), cj = max(bj0, j0);
    const uint32_t Bi0 = compact15(blo), Bj0 = compact15(blo >> 1);
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
                    const uint32_t *__restrict__ leaf_lo, const uint32_t *__restrict__ leaf_hi,
                    const uint32_t *__restrict__ zmap, uint2 *__restrict__ qcells,
                    unsigned long long *__restrict__ cand_off, uint32_t *__restrict__ pair_q,
                    uint32_t *__restrict__ pair_first, uint32_t *__restrict__ pair_blo,
                    unsigned long long *__restrict__ pair_off, uint32_t *status_p,
                    unsigned long long *status_c, uint32_t *tile_counter, Info *info) {
    __shared__ uint32_t s_scan32[kQBThreads / 32 + 1];
    __shared__ unsigned long long s_scan64[kQBThreads / 32 + 1];
    __shared__ uint32_t s_tile, s_pp;
    __shared__ unsigned long long s_pc;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint32_t L = (uint32_t)info->n_leaves;
    const uint32_t q = tile * kQBThreads + tid;

    uint32_t first[9], cnt[9], blo9[9];
    uint32_t npairs = 0;
    unsigned long long ncand = 0;
#pragma unroll
    for (int b = 0; b < 9; ++b) cnt[b] = 0;
    QCells c;
    if (q < Q && L > 0 && query_cells(rects[q], x0, y0, sx, sy, c)) {
        const uint32_t k = block_log2(c.i0, c.i1, c.j0, c.j1);
        const uint32_t bi_lo = c.i0 >> k, bi_hi = c.i1 >> k, bj_lo = c.j0 >> k, bj_hi = c.j1 >> k;
        qcells[q] = make_uint2(c.i0 | (c.i1 << 16), c.j0 | (c.j1 << 16));
#pragma unroll
        for (int dj = 0; dj < 3; ++dj) {
#pragma unroll
            for (int di = 0; di < 3; ++di) {
                const int b = dj * 3 + di;
                if (bi_lo + di > bi_hi || bj_lo + dj > bj_hi) continue;
                const uint32_t blo = morton2((bi_lo + di) << k, (bj_lo + dj) << k);
                const uint32_t bhi = blo + ((1u << (2 * k)) - 1u);
                const uint32_t f = leaf_at_or_after(blo, leaf_hi, zmap);
                if (f >= L || __ldg(leaf_lo + f) > bhi) continue;
                const uint32_t g = leaf_at_or_after(bhi, leaf_hi, zmap);
                const uint32_t last = (g < L && __ldg(leaf_lo + g) <= bhi) ? g : g - 1u;
                first[b] = f;
                cnt[b] = last - f + 1u;
                blo9[b] = blo;
                ++npairs;
                ncand += cnt[b];
            }
        }
    }
    uint32_t tot_p;
    unsigned long long tot_c;
    const uint32_t off_p = block_excl_scan<kQBThreads>(npairs, &tot_p, s_scan32);
    const unsigned long long off_c = block_excl_scan<kQBThreads>(ncand, &tot_c, s_scan64);
    if (tid == 0) {
        s_pp = lookback<uint32_t>(status_p, tile, tot_p, &info->err);
        s_pc = lookback<unsigned long long>(status_c, tile, tot_c, &info->err);
    }
    __syncthreads();
    uint32_t p = s_pp + off_p;
    unsigned long long co = s_pc + off_c;
    if (q < Q) cand_off[q] = co;
#pragma unroll
    for (int b = 0; b < 9; ++b) {
        if (cnt[b] == 0) continue;
        pair_q[p] = q;
        pair_first[p] = first[b];
        pair_blo[p] = blo9[b];
        pair_off[p] = co;
        co += cnt[b];
        ++p;
    }
    if (tid == 0 && (tile + 1) * (uint32_t)kQBThreads >= Q) {
        const uint32_t np = s_pp + tot_p;
        const unsigned long long nc = s_pc + tot_c;
        cand_off[Q] = nc;
        pair_off[np] = nc;
        info->n_pairs = np;
        info->n_cand = nc;
    }
}

void launch_zmap(cudaStream_t st, const uint32_t *leaf_hi, const Info *info, uint32_t *zmap) {
    zmap_kernel<<<(kZCells + 1 + 255) / 256, 256, 0, st>>>(leaf_hi, info, zmap);
}

void launch_query_blocks(cudaStream_t st, const float4 *rects, uint32_t Q, float x0, float y0, float sx,
                         float sy, const uint32_t *leaf_lo, const uint32_t *leaf_hi, const uint32_t *zmap,
                         uint2 *qcells, unsigned long long *cand_off, uint32_t *pair_q,
                         uint32_t *pair_first, uint32_t *pair_blo, unsigned long long *pair_off,
                         uint32_t *status_p, unsigned long long *status_c, uint32_t *tile_counter,
                         Info *info) {
    if (Q == 0) return;
    uint32_t tiles = (Q + kQBThreads - 1) / kQBThreads;
    query_blocks_kernel<<<tiles, kQBThreads, 0, st>>>(rects, Q, x0, y0, sx, sy, leaf_lo, leaf_hi, zmap,
                                                      qcells, cand_off, pair_q, pair_first, pair_blo,
                                                      pair_off, status_p, status_c, tile_counter, info);
}

// ---------------------------------------------------------------------------
// a7: candidate leaves -> subquery records.  Tiles of kCandTile candidates
// (taken in order by a persistent grid) map each candidate to its pair,
// classify it, and compact the subqueries with a single-pass scan into
// records in query-major order.  Consecutive covering leaves of one pair form
// one covering run (their objects are one contiguous range of the sorted
// objects).  Record k: sub_q[k] = query, sub_leaf[k] = first leaf (bit 31 set
// for a covering run), sub_len[k] = run length, sub_res[k] = result count
// (covering: the run's objects; intersecting: 0, filled by the filter).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int classify_candidate(unsigned long long cand, uint32_t p,
                                                  const uint32_t *__restrict__ pair_q,
                                                  const uint32_t *__restrict__ pair_first,
                                                  const uint32_t *__restrict__ pair_blo,
                                                  const unsigned long long *__restrict__ pair_off,
                                                  const uint2 *__restrict__ qcells,
                                                  const uint32_t *__restrict__ leaf_lo,
                                                  const uint32_t *__restrict__ leaf_hi, int covering) {
    uint32_t i0, i1, j0, j1;
    unpack_cells(__ldg(qcells + __ldg(pair_q + p)), i0, i1, j0, j1);
    const uint32_t l = __ldg(pair_first + p) + (uint32_t)(cand - __ldg(pair_off + p));
    int cl = classify(i0, i1, j0, j1, block_log2(i0, i1, j0, j1), __ldg(pair_blo + p), __ldg(leaf_lo + l),
                      __ldg(leaf_hi + l));
    return (cl == 2 && !covering) ? 1 : cl;
}

__global__ void __launch_bounds__(kCandThreads)
candidates_kernel(uint32_t Q, int covering, const uint32_t *__restrict__ leaf_lo,
                  const uint32_t *__restrict__ leaf_hi, const uint32_t *__restrict__ leaf_beg,
                  const uint2 *__restrict__ qcells, const unsigned long long *__restrict__ cand_off,
                  const uint32_t *__restrict__ pair_q, const uint32_t *__restrict__ pair_first,
                  const uint32_t *__restrict__ pair_blo, const unsigned long long *__restrict__ pair_off,
                  uint32_t *__restrict__ sub_q, uint32_t *__restrict__ sub_leaf,
                  uint32_t *__restrict__ sub_len, uint32_t *__restrict__ sub_res,
                  uint32_t *__restrict__ sub_off, uint32_t *__restrict__ leaf_nsub, uint32_t *status,
                  uint32_t *tile_counter, Caps caps, Info *info) {
    constexpr int T = kCandTile, PER = kCandItems;
    __shared__ unsigned long long s_poff[T + 2];
    __shared__ uint32_t s_pq[T + 1], s_pfirst[T + 1], s_pblo[T + 1];
    __shared__ uint8_t s_code[T];
    __shared__ uint16_t s_pj[T];
    __shared__ uint32_t s_rec[T + 1];
    __shared__ uint32_t s_scan[kCandThreads / 32 + 1];
    __shared__ unsigned long long s_red[4];
    __shared__ uint32_t s_tile, s_p0, s_prefix, s_qa;
    __shared__ int s_prev_cov;

    const int tid = threadIdx.x;
    const unsigned long long ncand = info->n_cand;
    const uint32_t npairs = (uint32_t)info->n_pairs;
    if (ncand == 0) {
        for (uint32_t q = blockIdx.x * blockDim.x + tid; q <= Q; q += gridDim.x * blockDim.x) sub_off[q] = 0;
        return;
    }
    const unsigned long long ntiles = (ncand + T - 1) / T;
    if (ntiles > caps.cand_tiles) return;     // the host sees n_cand, grows the status array, retries
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
        if (tid < 4) s_red[tid] = 0;
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles) break;
        const unsigned long long c0 = (unsigned long long)tile * T;
        const uint32_t cn = (uint32_t)min((unsigned long long)T, ncand - c0);
        if (tid == 0) {
            // last pair with pair_off[p] <= c0
            uint32_t a = 0, b = npairs;
            while (b - a > 1) {
                uint32_t m = (a + b) >> 1;
                if (pair_off[m] <= c0) a = m; else b = m;
            }
            s_p0 = a;
        }
        __syncthreads();
        const uint32_t p0 = s_p0;
        const uint32_t np = min((uint32_t)T + 1u, npairs - p0);      // pairs p0 .. p0+np-1
        for (uint32_t j = tid; j <= np; j += kCandThreads) {
            s_poff[j] = pair_off[p0 + j];                                // pair_off[npairs] = ncand
            if (j < np) {
                s_pq[j] = pair_q[p0 + j];
                s_pfirst[j] = pair_first[p0 + j];
                s_pblo[j] = pair_blo[p0 + j];
            }
        }
        if (tid == 0) {
            // classification of the candidate just before the tile, if it belongs to pair p0
            s_prev_cov = 0;
            if (c0 > 0 && c0 - 1 >= pair_off[p0])
                s_prev_cov = classify_candidate(c0 - 1, p0, pair_q, pair_first, pair_blo, pair_off, qcells,
                                                leaf_lo, leaf_hi, covering) == 2;
        }
        __syncthreads();

        // classify this thread's candidates (blocked: tid*PER .. +PER)
        uint32_t nrec = 0;
        unsigned long long n_i = 0, n_c = 0, tests = 0;
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            const uint32_t loc = tid * PER + e;
            if (loc >= cn) break;
            const unsigned long long cand = c0 + loc;
            uint32_t a = 0, b = np;                                   // last j with s_poff[j] <= cand
            while (b - a > 1) {
                uint32_t m = (a + b) >> 1;
                if (s_poff[m] <= cand) a = m; else b = m;
            }
            uint32_t i0, i1, j0, j1;
            unpack_cells(__ldg(qcells + s_pq[a]), i0, i1, j0, j1);
            const uint32_t l = s_pfirst[a] + (uint32_t)(cand - s_poff[a]);
            int cl = classify(i0, i1, j0, j1, block_log2(i0, i1, j0, j1), s_pblo[a], __ldg(leaf_lo + l),
                              __ldg(leaf_hi + l));
            if (cl == 2 && !covering) cl = 1;
            s_code[loc] = (uint8_t)cl;
            s_pj[loc] = (uint16_t)a;
        }
        __syncthreads();
        // records: intersecting candidates and heads of covering runs
        uint32_t rflags = 0;
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            const uint32_t loc = tid * PER + e;
            if (loc >= cn) break;
            const int cl = s_code[loc];
            bool rec = false;
            if (cl == 1) {
                rec = true;
            } else if (cl == 2) {
                const unsigned long long cand = c0 + loc;
                const uint32_t a = s_pj[loc];
                bool cont;
                if (cand == s_poff[a]) cont = false;                     // first candidate of its pair
                else if (loc == 0) cont = s_prev_cov;
                else cont = s_code[loc - 1] == 2;
                rec = !cont;
            }
            if (rec) {
                rflags |= 1u << e;
                ++nrec;
            }
        }
        uint32_t total;
        uint32_t off = block_excl_scan<kCandThreads>(nrec, &total, s_scan);
        if (tid == 0) s_prefix = lookback<uint32_t>(status, tile, total, &info->err);
        // exclusive record prefix at every candidate position of the tile
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            const uint32_t loc = tid * PER + e;
            if (loc < cn) s_rec[loc] = off;
            if (rflags & (1u << e)) ++off;
        }
        if (tid == 0) s_rec[cn] = total;
        __syncthreads();
        const uint32_t prefix = s_prefix;

        // write the records
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            const uint32_t loc = tid * PER + e;
            if (loc >= cn) break;
            const int cl = s_code[loc];
            if (cl == 2) ++n_c;
            if (!(rflags & (1u << e))) continue;
            const unsigned long long cand = c0 + loc;
            const uint32_t a = s_pj[loc];
            const uint32_t q = s_pq[a];
            const uint32_t l = s_pfirst[a] + (uint32_t)(cand - s_poff[a]);
            const uint32_t k = prefix + s_rec[loc];
            if (cl == 1) {
                ++n_i;
                atomicAdd(leaf_nsub + l, 1u);
                tests += __ldg(leaf_beg + l + 1) - __ldg(leaf_beg + l);
                if (k < caps.sub) {
                    sub_q[k] = q;
                    sub_leaf[k] = l;
                    sub_len[k] = 1;
                    sub_res[k] = 0;
                }
            } else {
                // run length: following candidates of the same pair that are covering
                uint32_t len = 1;
                const unsigned long long pend = s_poff[a + 1];
                unsigned long long nx = cand + 1;
                while (nx < pend) {
                    int cl2;
                    if (nx < c0 + cn) cl2 = s_code[nx - c0];
                    else cl2 = classify_candidate(nx, p0 + a, pair_q, pair_first, pair_blo, pair_off, qcells,
                                                  leaf_lo, leaf_hi, covering);
                    if (cl2 != 2) break;
                    ++len;
                    ++nx;
                }
                if (k < caps.sub) {
                    sub_q[k] = q;
                    sub_leaf[k] = l | 0x80000000u;
                    sub_len[k] = len;
                    sub_res[k] = __ldg(leaf_beg + l + len) - __ldg(leaf_beg + l);
                }
            }
        }
        n_i = warp_sum(n_i); n_c = warp_sum(n_c); tests = warp_sum(tests);
        if ((tid & 31) == 0) {
            atomicAdd(&s_red[0], n_i);
            atomicAdd(&s_red[1], n_c);
            atomicAdd(&s_red[3], tests);
        }
        // per-query first record: queries whose first candidate lies in this tile
        if (tid == 0) {
            uint32_t a = 0, b = Q;                                     // first q with cand_off[q] >= c0
            while (a < b) {
                uint32_t m = (a + b) >> 1;
                if (cand_off[m] >= c0) b = m; else a = m + 1;
            }
            s_qa = a;
        }
        __syncthreads();
        const bool last_tile = c0 + cn == ncand;
        for (uint32_t q = s_qa + tid; q <= Q; q += kCandThreads) {
            const unsigned long long co = cand_off[q];
            if (co >= c0 + cn && !(last_tile && co == ncand)) break;
            sub_off[q] = prefix + (co >= c0 + cn ? total : s_rec[co - c0]);
        }
        if (tid == 0) {
            if (s_red[0]) atomicAdd(&info->n_sub_i, s_red[0]);
            if (s_red[1]) atomicAdd(&info->n_sub_c, s_red[1]);
            if (s_red[3]) atomicAdd(&info->n_tests, s_red[3]);
            if (total > s_red[0]) atomicAdd(&info->n_runs, (unsigned long long)(total - s_red[0]));
            if (last_tile) info->n_sub = prefix + total;
        }
        __syncthreads();
    }
}

void launch_candidates(cudaStream_t st, int num_sms, uint32_t Q, int covering, const uint32_t *leaf_lo,
                       const uint32_t *leaf_hi, const uint32_t *leaf_beg, const uint2 *qcells,
                       const unsigned long long *cand_off, const uint32_t *pair_q,
                       const uint32_t *pair_first, const uint32_t *pair_blo,
                       const unsigned long long *pair_off, uint32_t *sub_q, uint32_t *sub_leaf,
                       uint32_t *sub_len, uint32_t *sub_res, uint32_t *sub_off, uint32_t *leaf_nsub,
                       uint32_t *status, uint32_t *tile_counter, Caps caps, Info *info) {
    candidates_kernel<<<num_sms * 4, kCandThreads, 0, st>>>(Q, covering, leaf_lo, leaf_hi, leaf_beg, qcells,
                                                            cand_off, pair_q, pair_first, pair_blo, pair_off,
                                                            sub_q, sub_leaf, sub_len, sub_res, sub_off,
                                                            leaf_nsub, status, tile_counter, caps, info);
}

// ---------------------------------------------------------------------------
// a8: per-leaf scans.  For leaf l with n objects and s intersecting
// subqueries: its subquery list starts at leaf_sub_off[l]; its bitmap (s rows
// of ceil(n/32) words, row-major: the linearized layout of Sec. 5.5) starts
// at leaf_word_off[l]; its filter work items (ceil(n/256) object chunks x
// ceil(s/32) subquery groups) start at leaf_item_off[l].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kLeafScanThreads)
leaf_scan_kernel(const uint32_t *__restrict__ leaf_beg, const uint32_t *__restrict__ leaf_nsub,
                 uint32_t *__restrict__ leaf_sub_off, uint32_t *__restrict__ leaf_word_off,
                 uint32_t *__restrict__ leaf_item_off, uint32_t *__restrict__ leaf_cursor,
                 uint32_t *status3, uint32_t num_tiles, uint32_t *tile_counter, Info *info) {
    __shared__ uint32_t s_scan[kLeafScanThreads / 32 + 1];
    __shared__ uint32_t s_tile, s_p[3];
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint32_t L = (uint32_t)info->n_leaves;
    const uint32_t base = tile * kLeafScanTile;
    if (base >= L) return;
    const uint32_t lb = base + tid * kLeafScanItems;

    uint32_t ns[kLeafScanItems], nw[kLeafScanItems], ni[kLeafScanItems];
    uint32_t t_s = 0, t_w = 0, t_i = 0;
    unsigned long long objs = 0;
#pragma unroll
    for (int e = 0; e < kLeafScanItems; ++e) {
        uint32_t l = lb + e;
        ns[e] = nw[e] = ni[e] = 0;
        if (l < L) {
            uint32_t s = leaf_nsub[l];
            uint32_t n = leaf_beg[l + 1] - leaf_beg[l];
            ns[e] = s;
            nw[e] = s * ((n + 31u) >> 5);
            ni[e] = s ? ((n + 255u) >> 8) * ((s + 31u) >> 5) : 0u;
            if (s) objs += (unsigned long long)n * ((s + 31u) >> 5);
        }
        t_s += ns[e]; t_w += nw[e]; t_i += ni[e];
    }
    uint32_t tot_s, tot_w, tot_i;
    uint32_t o_s = block_excl_scan<kLeafScanThreads>(t_s, &tot_s, s_scan);
    uint32_t o_w = block_excl_scan<kLeafScanThreads>(t_w, &tot_w, s_scan);
    uint32_t o_i = block_excl_scan<kLeafScanThreads>(t_i, &tot_i, s_scan);
    objs = warp_sum(objs);
    if ((tid & 31) == 0 && objs) atomicAdd(&info->n_item_objs, objs);
    if (tid < 3) {
        uint32_t agg = tid == 0 ? tot_s : (tid == 1 ? tot_w : tot_i);
        s_p[tid] = lookback<uint32_t>(status3 + (size_t)tid * num_tiles, tile, agg, &info->err);
    }
    __syncthreads();
    o_s += s_p[0]; o_w += s_p[1]; o_i += s_p[2];
#pragma unroll
    for (int e = 0; e < kLeafScanItems; ++e) {
        uint32_t l = lb + e;
        if (l < L) {
            leaf_sub_off[l] = o_s;
            leaf_cursor[l] = o_s;
            leaf_word_off[l] = o_w;
            leaf_item_off[l] = o_i;
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
}

void launch_leaf_scan(cudaStream_t st, uint32_t nmax, const uint32_t *leaf_beg,
                      const uint32_t *leaf_nsub, uint32_t *leaf_sub_off, uint32_t *leaf_word_off,
                      uint32_t *leaf_item_off, uint32_t *leaf_cursor, uint32_t *status3,
                      uint32_t *tile_counter, Info *info) {
    if (nmax == 0) return;
    uint32_t tiles = (nmax + kLeafScanTile - 1) / kLeafScanTile;
    leaf_scan_kernel<<<tiles, kLeafScanThreads, 0, st>>>(leaf_beg, leaf_nsub, leaf_sub_off,
                                                         leaf_word_off, leaf_item_off, leaf_cursor,
                                                         status3, tiles, tile_counter, info);
}

// ---------------------------------------------------------------------------
// a8 (scatter): intersecting subqueries into their leaf's list, each with the
// offset of its bitmap row (row = rank in the leaf's list).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
scatter_kernel(const uint32_t *__restrict__ sub_leaf, const uint32_t *__restrict__ leaf_beg,
               const uint32_t *__restrict__ leaf_sub_off, const uint32_t *__restrict__ leaf_word_off,
               uint32_t *__restrict__ leaf_cursor, uint32_t *__restrict__ sub_bm,
               uint32_t *__restrict__ isub, Caps caps, const Info *info) {
    if (info->n_sub > caps.sub || info->n_sub_i > caps.sub_i || info->n_words > caps.words) return;
    const uint32_t nsub = (uint32_t)info->n_sub;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nsub; k += gridDim.x * blockDim.x) {
        const uint32_t sl = sub_leaf[k];
        if (sl & 0x80000000u) continue;
        const uint32_t pos = atomicAdd(leaf_cursor + sl, 1u);
        const uint32_t n = __ldg(leaf_beg + sl + 1) - __ldg(leaf_beg + sl);
        isub[pos] = k;
        sub_bm[k] = __ldg(leaf_word_off + sl) + (pos - __ldg(leaf_sub_off + sl)) * ((n + 31u) >> 5);
    }
}

void launch_scatter(cudaStream_t st, int num_sms, const uint32_t *sub_leaf, const uint32_t *leaf_beg,
                    const uint32_t *leaf_sub_off, const uint32_t *leaf_word_off, uint32_t *leaf_cursor,
                    uint32_t *sub_bm, uint32_t *isub, Caps caps, const Info *info) {
    scatter_kernel<<<num_sms * 8, 256, 0, st>>>(sub_leaf, leaf_beg, leaf_sub_off, leaf_word_off, leaf_cursor,
                                                sub_bm, isub, caps, info);
}

}  // namespace mqr
