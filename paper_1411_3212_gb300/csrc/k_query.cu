// k_query.cu -- query indexing: splitting every query into subqueries over the
// leaves it meets (Def. "Mapping functions", function g), intersecting vs
// covering classification, the two-pass count/scan/write scheme of Sec. 5.3
// ("Indexing moving objects and queries"), and the grouping of intersecting
// subqueries by leaf (Sec. 5.3 "Sorting", replaced by a counting scatter).
//
// The leaves of a tick are contiguous Morton intervals [lo, hi] of the
// l_max grid, sorted.  Instead of the paper's z_map table (4^l_deep entries),
// a query walks the leaf table along the Z-order curve restricted to its cell
// rectangle: find the first leaf ending at or after the current in-box code,
// emit it if its box meets the rectangle, then jump to the smallest Morton
// code inside the rectangle that follows the leaf (BIGMIN).  Each (query,
// leaf) pair is visited once, which is the paper's duplicate elimination
// (one subquery per cell, Fig. 8) by construction.
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

// Smallest idx >= from with hi[idx] >= z (galloping search), or L.
__device__ __forceinline__ uint32_t first_hi_ge(const uint32_t *__restrict__ hi, uint32_t L,
                                                uint32_t from, uint32_t z) {
    if (from >= L) return L;
    if (__ldg(hi + from) >= z) return from;
    uint32_t a = from, step = 1, b;
    for (;;) {
        b = a + step;
        if (b >= L) { b = L; break; }
        if (__ldg(hi + b) >= z) break;
        a = b;
        step <<= 1;
    }
    uint32_t lo = a + 1;
    while (lo < b) {
        uint32_t m = (lo + b) >> 1;
        if (__ldg(hi + m) >= z) b = m; else lo = m + 1;
    }
    return lo;
}

// BIGMIN: the smallest Morton code >= z whose cell lies in the rectangle with
// corner codes zmin = z(i0, j0), zmax = z(i1, j1).  Bits are examined from the
// top; `lower` selects the lower bits of the same axis as bit b.
__device__ __forceinline__ bool next_in_box(uint32_t z, uint32_t zmin, uint32_t zmax, uint32_t &out) {
    uint32_t mn = zmin, mx = zmax, best = 0;
    bool have = false;
    for (int b = 2 * kLevels - 1; b >= 0; --b) {
        const uint32_t bit = 1u << b;
        const uint32_t lower = ((b & 1) ? 0xAAAAAAAAu : 0x55555555u) & (bit - 1u);
        const uint32_t sel = ((z >> b) & 1u) << 2 | ((mn >> b) & 1u) << 1 | ((mx >> b) & 1u);
        switch (sel) {
            case 1:  // z in the lower half, the box spans both: upper half is a candidate
                best = (mn | bit) & ~lower;
                have = true;
                mx = (mx & ~bit) | lower;
                break;
            case 3:  // the whole remaining box lies above z
                out = mn;
                return true;
            case 4:  // the whole remaining box lies below z
                if (have) { out = best; return true; }
                return false;
            case 5:  // z in the upper half: restrict the box to it
                mn = (mn | bit) & ~lower;
                break;
            case 2:
            case 6:  // cannot happen for a valid box
                if (have) { out = best; return true; }
                return false;
            default:
                break;
        }
    }
    out = z;
    return true;
}

// Walk the leaves meeting the query's cell rectangle in Morton order and call
// emit(leaf, covering).  Covering iff the leaf's cells lie strictly inside
// the rectangle on both axes: then every object of the leaf passes the FP32
// test of Def. 1, because the cell function is monotone.
template <class F>
__device__ __forceinline__ void walk_leaves(const QCells &c, const uint32_t *__restrict__ leaf_lo,
                                            const uint32_t *__restrict__ leaf_hi, uint32_t L, F &&emit) {
    const uint32_t zmin = morton2(c.i0, c.j0), zmax = morton2(c.i1, c.j1);
    uint32_t z = zmin, idx = 0;
    for (;;) {
        idx = first_hi_ge(leaf_hi, L, idx, z);
        if (idx >= L) break;
        const uint32_t lo = __ldg(leaf_lo + idx), hi = __ldg(leaf_hi + idx);
        if (lo > zmax) break;
        const uint32_t span = hi - lo + 1u;                 // 4^s cells
        const uint32_t s = (31u - __clz(span)) >> 1;
        const uint32_t bi0 = compact15(lo), bj0 = compact15(lo >> 1);
        const uint32_t bi1 = bi0 + (1u << s) - 1u, bj1 = bj0 + (1u << s) - 1u;
        if (!(bi1 < c.i0 || bi0 > c.i1 || bj1 < c.j0 || bj0 > c.j1))
            emit(idx, bi0 > c.i0 && bi1 < c.i1 && bj0 > c.j0 && bj1 < c.j1);
        if (hi >= zmax) break;
        uint32_t nz;
        if (!next_in_box(hi + 1u, zmin, zmax, nz)) break;
        z = nz;
        ++idx;
    }
}

// Emission state: consecutive covering leaves (leaf indices l, l+1, ...) form
// one covering run, whose objects are one contiguous range of the sorted
// object array.
struct RunState {
    uint32_t first, len;
    bool open;
};

// ---------------------------------------------------------------------------
// a5 + a6: count pass with fused single-pass scan -> sub_off[Q+1].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kQueryThreads)
query_count_kernel(const float4 *__restrict__ rects, uint32_t Q, float x0, float y0, float sx,
                   float sy, const uint32_t *__restrict__ leaf_lo, const uint32_t *__restrict__ leaf_hi,
                   const uint32_t *__restrict__ leaf_beg, int covering, uint32_t *__restrict__ sub_off,
                   uint32_t *__restrict__ leaf_nsub, uint32_t *status, uint32_t *tile_counter,
                   Info *info) {
    __shared__ uint32_t s_scan[kQueryThreads / 32 + 1];
    __shared__ unsigned long long s_red[4];
    __shared__ uint32_t s_tile, s_prefix;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
    if (tid < 4) s_red[tid] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint32_t L = (uint32_t)info->n_leaves;
    const uint32_t qbase = tile * kQueryTile + tid * kQueryItems;

    uint32_t cnt[kQueryItems];
    unsigned long long n_i = 0, n_c = 0, n_runs = 0, tests = 0;
#pragma unroll
    for (int e = 0; e < kQueryItems; ++e) {
        cnt[e] = 0;
        uint32_t q = qbase + e;
        if (q >= Q) continue;
        QCells c;
        if (!query_cells(rects[q], x0, y0, sx, sy, c)) continue;
        RunState rs{0, 0, false};
        uint32_t k = 0;
        walk_leaves(c, leaf_lo, leaf_hi, L, [&](uint32_t leaf, bool cov) {
            if (cov && covering) {
                ++n_c;
                if (rs.open && leaf == rs.first + rs.len) { ++rs.len; return; }
                rs = RunState{leaf, 1, true};
                ++k;
                ++n_runs;
            } else {
                rs.open = false;
                ++k;
                ++n_i;
                atomicAdd(leaf_nsub + leaf, 1u);
                tests += __ldg(leaf_beg + leaf + 1) - __ldg(leaf_beg + leaf);
            }
        });
        cnt[e] = k;
    }
    uint32_t local = 0;
#pragma unroll
    for (int e = 0; e < kQueryItems; ++e) local += cnt[e];
    uint32_t total;
    uint32_t off = block_excl_scan<kQueryThreads>(local, &total, s_scan);
    if (tid == 0) s_prefix = lookback<uint32_t>(status, tile, total, &info->err);
    n_i = warp_sum(n_i); n_c = warp_sum(n_c); n_runs = warp_sum(n_runs); tests = warp_sum(tests);
    if ((tid & 31) == 0) {
        atomicAdd(&s_red[0], n_i); atomicAdd(&s_red[1], n_c);
        atomicAdd(&s_red[2], n_runs); atomicAdd(&s_red[3], tests);
    }
    __syncthreads();
    uint32_t run = s_prefix + off;
#pragma unroll
    for (int e = 0; e < kQueryItems; ++e) {
        uint32_t q = qbase + e;
        if (q < Q) sub_off[q] = run;
        run += cnt[e];
    }
    if (tid == 0) {
        if (s_red[0]) atomicAdd(&info->n_sub_i, s_red[0]);
        if (s_red[1]) atomicAdd(&info->n_sub_c, s_red[1]);
        if (s_red[2]) atomicAdd(&info->n_runs, s_red[2]);
        if (s_red[3]) atomicAdd(&info->n_tests, s_red[3]);
        if ((tile + 1) * (uint32_t)kQueryTile >= Q) {
            sub_off[Q] = s_prefix + total;
            info->n_sub = s_prefix + total;
        }
    }
}

void launch_query_count(cudaStream_t st, const float4 *rects, uint32_t Q, float x0, float y0,
                        float sx, float sy, const uint32_t *leaf_lo, const uint32_t *leaf_hi,
                        const uint32_t *leaf_beg, int covering, uint32_t *sub_off,
                        uint32_t *leaf_nsub, uint32_t *status, uint32_t *tile_counter, Info *info) {
    if (Q == 0) return;
    uint32_t tiles = (Q + kQueryTile - 1) / kQueryTile;
    query_count_kernel<<<tiles, kQueryThreads, 0, st>>>(rects, Q, x0, y0, sx, sy, leaf_lo, leaf_hi,
                                                        leaf_beg, covering, sub_off, leaf_nsub,
                                                        status, tile_counter, info);
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
        }
        t_s += ns[e]; t_w += nw[e]; t_i += ni[e];
    }
    uint32_t tot_s, tot_w, tot_i;
    uint32_t o_s = block_excl_scan<kLeafScanThreads>(t_s, &tot_s, s_scan);
    uint32_t o_w = block_excl_scan<kLeafScanThreads>(t_w, &tot_w, s_scan);
    uint32_t o_i = block_excl_scan<kLeafScanThreads>(t_i, &tot_i, s_scan);
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
// a7: write pass.  Same walk as the count pass; subquery record k of query q
// (k in [sub_off[q], sub_off[q+1])) holds q, its first leaf (bit 31 set for
// a covering run), the run length in leaves, and its result count
// (covering: the run's object count; intersecting: 0, filled by the filter).
// Intersecting subqueries are scattered into their leaf's list and get the
// offset of their bitmap row.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kQueryThreads)
query_write_kernel(const float4 *__restrict__ rects, uint32_t Q, float x0, float y0, float sx,
                   float sy, const uint32_t *__restrict__ leaf_lo, const uint32_t *__restrict__ leaf_hi,
                   const uint32_t *__restrict__ leaf_beg, int covering,
                   const uint32_t *__restrict__ sub_off, const uint32_t *__restrict__ leaf_sub_off,
                   const uint32_t *__restrict__ leaf_word_off, uint32_t *__restrict__ leaf_cursor,
                   uint32_t *__restrict__ sub_q, uint32_t *__restrict__ sub_leaf,
                   uint32_t *__restrict__ sub_len, uint32_t *__restrict__ sub_res,
                   uint32_t *__restrict__ sub_bm, uint32_t *__restrict__ isub, Caps caps,
                   const Info *info) {
    if (info->n_sub > caps.sub || info->n_sub_i > caps.sub_i || info->n_words > caps.words) return;
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    QCells c;
    if (!query_cells(rects[q], x0, y0, sx, sy, c)) return;
    const uint32_t L = (uint32_t)info->n_leaves;
    uint32_t k = sub_off[q];
    const uint32_t kend = sub_off[q + 1];
    RunState rs{0, 0, false};
    auto close_run = [&]() {
        if (rs.open) {
            sub_q[k] = q;
            sub_leaf[k] = rs.first | 0x80000000u;
            sub_len[k] = rs.len;
            sub_res[k] = __ldg(leaf_beg + rs.first + rs.len) - __ldg(leaf_beg + rs.first);
            ++k;
            rs.open = false;
        }
    };
    walk_leaves(c, leaf_lo, leaf_hi, L, [&](uint32_t leaf, bool cov) {
        if (cov && covering) {
            if (rs.open && leaf == rs.first + rs.len) { ++rs.len; return; }
            close_run();
            rs = RunState{leaf, 1, true};
        } else {
            close_run();
            uint32_t pos = atomicAdd(leaf_cursor + leaf, 1u);
            uint32_t n = __ldg(leaf_beg + leaf + 1) - __ldg(leaf_beg + leaf);
            sub_q[k] = q;
            sub_leaf[k] = leaf;
            sub_len[k] = 1;
            sub_res[k] = 0;
            sub_bm[k] = leaf_word_off[leaf] + (pos - leaf_sub_off[leaf]) * ((n + 31u) >> 5);
            isub[pos] = k;
            ++k;
        }
    });
    close_run();
    (void)kend;
}

void launch_query_write(cudaStream_t st, const float4 *rects, uint32_t Q, float x0, float y0,
                        float sx, float sy, const uint32_t *leaf_lo, const uint32_t *leaf_hi,
                        const uint32_t *leaf_beg, int covering, const uint32_t *sub_off,
                        const uint32_t *leaf_sub_off, const uint32_t *leaf_word_off,
                        uint32_t *leaf_cursor, uint32_t *sub_q, uint32_t *sub_leaf,
                        uint32_t *sub_len, uint32_t *sub_res, uint32_t *sub_bm, uint32_t *isub,
                        Caps caps, Info *info) {
    if (Q == 0) return;
    const int T = 128;
    query_write_kernel<<<(Q + T - 1) / T, T, 0, st>>>(rects, Q, x0, y0, sx, sy, leaf_lo, leaf_hi,
                                                      leaf_beg, covering, sub_off, leaf_sub_off,
                                                      leaf_word_off, leaf_cursor, sub_q, sub_leaf,
                                                      sub_len, sub_res, sub_bm, isub, caps, info);
}

}  // namespace mqr
