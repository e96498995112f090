// mqr_internal.cuh -- shared device helpers and kernel launchers of libmqr.
//
// Layout in HBM (one context, N = max_objects slots):
//   pos      float2[N]      last-known position per object id (Sec. 2.2)
//   stamp    u64[N]         (update epoch << 32 | index) of the winning update;
//                           0 = object never updated (absent)
//   keysA/B  u64[N]         radix-sort ping-pong: (morton30 << 32) | id, bit 62
//                           set for absent slots so they sort last
//   skey/sid u32[N]         Morton-sorted keys and ids of present objects
//   sxy      float2[N]      positions in Morton-sorted order (SoA-by-record,
//                           Sec. 4.4 structure of vectors)
//   leaf_lo/hi u32[L]       Morton interval [lo, hi] of each non-empty leaf
//   leaf_beg u32[L+1]       first sorted object of each leaf (cell boundary
//                           table, Sec. 4.4)
//   leaf_box uint2[L]       lower-left cell (i | j << 16) and log2 side of each
//                           leaf
//   per query, per subquery and per leaf work arrays (see mqr_api.cu)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace mqr {

constexpr int kLevels = 15;                 // l_max: 15 bits per axis, 30-bit keys
constexpr uint32_t kCells = 1u << kLevels;  // cells per axis of the l_max grid
constexpr uint32_t kAbsentKey = 1u << 30;   // key of an absent slot (sorts last)

// Sticky error bits reported through Info::err.
constexpr unsigned long long kErrTimeout = 1ull;   // a bounded wait gave up
constexpr unsigned long long kErrBadId = 2ull;     // update id >= max_objects
constexpr unsigned long long kErrInternal = 4ull;  // an index left its range

// Device-side counters of one tick (zeroed at the start of every tick).
struct Info {
    unsigned long long n_present;
    unsigned long long n_leaves;
    unsigned long long max_level;
    unsigned long long n_sub;       // subquery records (intersecting + covering runs)
    unsigned long long n_sub_i;     // intersecting subqueries
    unsigned long long n_sub_c;     // covering subqueries counted per leaf
    unsigned long long n_runs;      // covering runs
    unsigned long long n_tests;     // containment tests of the filter
    unsigned long long n_items;     // filter work items
    unsigned long long n_words;     // bitmap words
    unsigned long long n_results;   // R
    unsigned long long n_results_cov;
    unsigned long long err;
    unsigned long long n_item_objs;  // objects loaded by the filter (sum over items)
    unsigned long long n_pairs;      // (query, block) pairs of query splitting
    unsigned long long n_cand;       // candidate (query, leaf) pairs
    unsigned long long n_out;        // output elements (R, or R_I + 2 per covering run for the run kind)
    unsigned long long emit_end;     // admission: 0 = emit all, else (bit 63 |) emit records [0, low 32 bits) only
    unsigned long long admitted;     // admission: queries [0, admitted) answered
    unsigned long long admitted_out; // admission: their output elements
};

// Capacities of the growable per-tick buffers (host-chosen, passed by value).
struct Caps {
    unsigned long long sub;      // subquery records
    unsigned long long sub_i;    // intersecting subqueries (isub list)
    unsigned long long words;    // bitmap words
    unsigned long long out;      // output elements (pairs / ids / bitmap words)
    unsigned long long cand_tiles;  // warp tiles (32 candidates) the candidate buffers can hold
    unsigned long long items;       // filter work items (item -> leaf map)
};

// ---------------------------------------------------------------------------
// Cell function and Morton codes (Alg. 1 GPUcalculateMortonHash)
// ---------------------------------------------------------------------------
// i = min(floor((v - lo) * scale), 2^15 - 1), NaN and negatives to 0; the two
// roundings are explicit so that objects and query corners share one
// monotone map (exact containment follows from monotonicity).
__device__ __forceinline__ uint32_t cell_of(float v, float lo, float scale) {
    float t = __fmul_rn(__fsub_rn(v, lo), scale);
    if (!(t >= 0.0f)) return 0u;
    if (t >= 32767.0f) return kCells - 1;
    return (uint32_t)t;
}

// Spread the 15 low bits of v to the even bit positions.
__host__ __device__ __forceinline__ uint32_t spread15(uint32_t v) {
    v &= 0x7fffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}
__host__ __device__ __forceinline__ uint32_t compact15(uint32_t v) {
    v &= 0x55555555u;
    v = (v | (v >> 1)) & 0x33333333u;
    v = (v | (v >> 2)) & 0x0f0f0f0fu;
    v = (v | (v >> 4)) & 0x00ff00ffu;
    v = (v | (v >> 8)) & 0x0000ffffu;
    return v;
}

// Independent worlds sharing one index: world w (0 <= w < 4^bits) owns the
// object ids [obj_base[w], obj_base[w+1]) and the queries [q_base[w],
// q_base[w+1]).  Its quadtree is the node of depth `bits` whose Morton prefix
// is w, so a world's cells are its own l_max cells shifted right by `bits`
// and placed in that node; leaves never lie above depth `bits`.  n == 0: one
// world, the whole grid.
constexpr uint32_t kMaxWorlds = 16384;     // 4^7: at least 8 levels left per world
// Per-region leaf capacities: the nodes of depth region_bits <= 4 (at most
// 256 regions), each capacity at most kLeafCapSmem (shared-memory window table).
constexpr uint32_t kMaxRegionBits = 4;
// Per-region work statistics of a tick (mqr_region_work), in this order.
enum RegionStat { kRsObjects, kRsLeaves, kRsQueries, kRsSideLog2, kRsSubI, kRsSubC, kRsTests, kRsResI, kRsResC,
                  kRegionStats };
struct Worlds {
    const uint32_t *obj_base;
    const uint32_t *q_base;
    uint32_t n;       // number of worlds (0: not batched)
    uint32_t bits;    // levels above the worlds' roots (4^bits >= n)
};

// The world of item i: the largest w with base[w] <= i.
__device__ __forceinline__ uint32_t world_of(uint32_t i, const uint32_t *__restrict__ base, uint32_t n) {
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1u) {
        const uint32_t m = (lo + hi) >> 1;
        if (__ldg(base + m) <= i) lo = m; else hi = m;
    }
    return lo;
}

// An l_max cell of world w on one axis (odd = y) -> its cell in the batched grid.
__device__ __forceinline__ uint32_t world_cell(uint32_t c, uint32_t w, uint32_t bits, int odd) {
    const uint32_t wc = compact15(odd ? (w >> 1) : w);
    return (wc << (kLevels - bits)) | (c >> bits);
}
// x index in the even bits, y index in the odd bits.
__host__ __device__ __forceinline__ uint32_t morton2(uint32_t i, uint32_t j) {
    return spread15(i) | (spread15(j) << 1);
}

// Depth of the deepest quadtree node containing both keys (0..15).
__device__ __forceinline__ uint32_t shared_depth(uint32_t a, uint32_t b) {
    uint32_t x = a ^ b;
    return x == 0u ? 15u : (uint32_t)(__clz(x) - 2) >> 1;
}

// ---------------------------------------------------------------------------
// Warp / block scans
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += u;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// Exclusive scan over the block (NT threads); *total receives the sum.
// smem: at least NT/32 + 1 elements.  Contains __syncthreads.
template <int NT, typename T>
__device__ __forceinline__ T block_excl_scan(T v, T *total, T *smem) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31) smem[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T s = lane < NT / 32 ? smem[lane] : T(0);
        T si = warp_incl_scan(s);
        if (lane < NT / 32) smem[lane] = si - s;
        if (lane == NT / 32 - 1) smem[NT / 32] = si;
    }
    __syncthreads();
    T res = smem[warp] + inc - v;
    *total = smem[NT / 32];
    __syncthreads();
    return res;
}

// ---------------------------------------------------------------------------
// Decoupled look-back for single-pass scans.  A status word packs a 2-bit
// flag (1 = tile aggregate, 2 = inclusive prefix) above the value.  Tiles are
// numbered in the order their blocks start (an atomic counter), so a tile
// only ever waits for tiles already running.  Waits are bounded by a
// wall-clock deadline; on expiry the kernel records kErrTimeout and carries on
// with a partial sum (its output is then discarded by the host).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s

template <typename T> struct StatusBits;
template <> struct StatusBits<uint32_t> {
    static constexpr uint32_t kShift = 30, kMask = (1u << 30) - 1;
};
template <> struct StatusBits<unsigned long long> {
    static constexpr unsigned kShift = 62;
    static constexpr unsigned long long kMask = (1ull << 62) - 1;
};

__device__ __forceinline__ uint32_t status_load(const uint32_t *p) {
    return *(const volatile uint32_t *)p;
}
__device__ __forceinline__ unsigned long long status_load(const unsigned long long *p) {
    return *(const volatile unsigned long long *)p;
}
__device__ __forceinline__ void status_store(uint32_t *p, uint32_t v) { atomicExch(p, v); }
__device__ __forceinline__ void status_store(unsigned long long *p, unsigned long long v) { atomicExch(p, v); }

// Warp-wide look-back, called by all 32 lanes of one warp of tile `tile`:
// publishes `agg`, examines the 32 nearest earlier tiles per step (one per
// lane), and returns (to every lane) the exclusive prefix of all earlier
// tiles, then publishes the inclusive prefix.
template <typename T>
__device__ T lookback_warp(T *status, uint32_t tile, T agg, unsigned long long *err,
                           unsigned long long wait_ns = kWaitNs) {
    using B = StatusBits<T>;
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) status_store(status, (T(2) << B::kShift) | agg);
        return T(0);
    }
    if (lane == 0) status_store(status + tile, (T(1) << B::kShift) | agg);
    T sum = 0;
    long j = (long)tile - 1;
    unsigned long long t0 = 0;
    unsigned spins = 0;
    bool expired = false;
    for (;;) {
        const long idx = j - lane;
        T v = idx < 0 ? (T(2) << B::kShift) : status_load(status + idx);
        for (;;) {
            const bool inval = (v >> B::kShift) == 0;
            if (!__any_sync(0xffffffffu, inval)) break;
            __nanosleep(64);
            if (inval) v = status_load(status + idx);
            if ((++spins & 63u) == 0) {
                if (lane == 0) {
                    unsigned long long now = global_ns();
                    if (t0 == 0) t0 = now;
                    else if (now - t0 > wait_ns) expired = true;
                }
                expired = __shfl_sync(0xffffffffu, expired, 0);
                if (expired) break;
            }
        }
        if (expired) {
            if (lane == 0) atomicOr(err, kErrTimeout);
            break;
        }
        const T flag = v >> B::kShift, val = v & B::kMask;
        const uint32_t incl = __ballot_sync(0xffffffffu, flag == 2);
        if (incl) {
            const int first = __ffs(incl) - 1;
            sum += warp_sum(lane <= first ? val : T(0));
            break;
        }
        sum += warp_sum(val);
        j -= 32;
    }
    if (lane == 0) status_store(status + tile, (T(2) << B::kShift) | (sum + agg));
    return sum;
}

// Per-thread look-back for the radix sort, where every thread scans the
// status of its own digit (consecutive tiles adjacent in memory).
template <typename T>
__device__ T lookback1(T *status, uint32_t tile, T agg, unsigned long long *err) {
    using B = StatusBits<T>;
    if (tile == 0) {
        status_store(status, (T(2) << B::kShift) | agg);
        return T(0);
    }
    status_store(status + tile, (T(1) << B::kShift) | agg);
    T sum = 0;
    long j = (long)tile - 1;
    unsigned long long t0 = 0;
    unsigned spins = 0;
    while (j >= 0) {
        const T v = status_load(status + j);
        const T flag = v >> B::kShift;
        if (flag == 0) {
            if ((++spins & 63u) == 0) {
                const unsigned long long now = global_ns();
                if (t0 == 0) t0 = now;
                else if (now - t0 > kWaitNs) {
                    atomicOr(err, kErrTimeout);
                    break;
                }
            }
            __nanosleep(32);
            continue;
        }
        sum += v & B::kMask;
        if (flag == 2) break;
        --j;
    }
    status_store(status + tile, (T(2) << B::kShift) | (sum + agg));
    return sum;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Message returned by mqr_last_error() on the calling thread.
void set_last_error(const std::string &msg);

// ---------------------------------------------------------------------------
// Launchers (host functions; all enqueue on `st`)
// ---------------------------------------------------------------------------
// a1: apply updates, last occurrence wins.
void launch_apply_updates(cudaStream_t st, const uint32_t *ids, const float2 *xy, uint32_t n,
                          uint32_t nmax, unsigned long long epoch, unsigned long long *stamp,
                          float2 *pos, unsigned long long *err);

// a2: Morton keys of every slot + digit histograms of the 4 sort passes.
void launch_state_flags(cudaStream_t st, const unsigned long long *stamp, uint32_t nmax, uint8_t *present);
void launch_state_stamps(cudaStream_t st, const uint8_t *present, uint32_t nmax, unsigned long long epoch,
                         unsigned long long *stamp);
// tile_counts: the first sort pass's per-tile digit counts (256 x tiles).
void launch_morton_keys(cudaStream_t st, const float2 *pos, const unsigned long long *stamp,
                        uint32_t nmax, float x0, float y0, float sx, float sy, Worlds worlds,
                        unsigned long long *keys, uint32_t *hist4x256, uint32_t *tile_counts, Info *info);

// a3: one onesweep pass over n u64 keys, 8-bit digit at `shift`.  The final
// pass of the object sort (`final_obj`) writes skey/sid/sxy instead of `out`.
constexpr int kSortThreads = 512, kSortItems = 8, kSortTile = kSortThreads * kSortItems;
void launch_onesweep_pass(cudaStream_t st, const unsigned long long *in, unsigned long long *out,
                          uint32_t n, int shift, const uint32_t *hist256, uint32_t *status,
                          uint32_t *tile_counter, unsigned long long *err, bool final_obj,
                          const float2 *pos, uint32_t *skey, uint32_t *sid, float2 *sxy);
// The same pass without look-back: per-tile digit counts (counts/offs hold
// 256 x ceil(n / kSortTile) u32 each), a per-digit scan over the tiles, then
// the rank-and-scatter tile kernel with the precomputed offsets.
// counts_ready: `counts` already holds the pass's per-tile digit counts.
void launch_sort_pass_pre(cudaStream_t st, const unsigned long long *in, unsigned long long *out, uint32_t n,
                          int shift, const uint32_t *hist256, uint32_t *counts, uint32_t *offs,
                          unsigned long long *err, bool final_obj, const float2 *pos, uint32_t *skey,
                          uint32_t *sid, float2 *sxy, bool counts_ready);
// Histograms (nd digit passes at shifts[]) of n u64 keys, for generic sorts.
void launch_key_histograms(cudaStream_t st, const unsigned long long *keys, uint32_t n,
                           const int *shifts_host, int nd, uint32_t *hist);

// a4: leaves.  level_mode: 0 = quadtree (capacity rule), 1 = uniform grid at
// `grid_level`; no leaf above depth min_level (the batched worlds' roots);
// region_bits > 0: per-region capacities region_cap[4^region_bits] (no leaf
// above depth region_bits).
// Writes leaf_lo/leaf_hi/leaf_beg and Info::n_leaves/max_level.
constexpr int kLeafThreads = 256, kLeafTile = 2048, kLeafCapSmem = 16384;
cudaError_t launch_region_work(cudaStream_t st, int num_sms, const uint32_t *leaf_lo, const uint32_t *leaf_beg,
                               uint32_t n_leaves, const uint32_t *sub_leaf, const uint32_t *sub_len,
                               const uint32_t *sub_res, unsigned long long n_sub, const float4 *rects, uint32_t Q,
                               float x0, float y0, float sx, float sy, uint32_t region_bits, double *out);
// The last tick's leaf footprint: leaves producing results and their objects
// (out[0], out[1]), tested leaves and their objects (out[2], out[3]); mark
// holds (n_leaves + 3) & ~3 bytes.
cudaError_t launch_footprint(cudaStream_t st, int num_sms, const uint32_t *sub_leaf, const uint32_t *sub_len,
                             const uint32_t *sub_res, unsigned long long n_sub, const uint32_t *leaf_beg,
                             uint32_t n_leaves, uint8_t *mark, unsigned long long *out);
cudaError_t launch_region_counts(cudaStream_t st, const uint32_t *skey, uint32_t n, uint32_t region_bits,
                                 uint32_t *counts);
void launch_build_leaves(cudaStream_t st, const uint32_t *skey, uint32_t nmax, uint32_t cap,
                         int uniform_grid, uint32_t grid_level, uint32_t min_level, uint32_t region_bits,
                         const uint32_t *region_cap, uint8_t *mk_a, uint8_t *mk_b,
                         uint32_t *status, uint32_t *tile_counter, uint32_t *leaf_lo,
                         uint32_t *leaf_hi, uint32_t *leaf_beg, uint32_t *leaf_nsub, uint2 *leaf_box,
                         Info *info);

// Query splitting (a5-a7).  Coarse lookup level and tile shapes.
constexpr int kZLevel = 8;
constexpr uint32_t kZCells = 1u << (2 * kZLevel);
constexpr int kZShift = 2 * (kLevels - kZLevel);
constexpr int kQBThreads = 256;                       // threads per block of query_blocks
constexpr int kQBQueries = kQBThreads / 9;            // queries per block (9 block slots each)
constexpr unsigned long long kMaxCandTiles = (1ull << 27) - 1;   // candidates and record indices fit 32 bits
constexpr int kCandWarpTiles = 8;                     // warp tiles of one warp in one chunk of the candidate pass
constexpr int kCandChunkTiles = 8 * kCandWarpTiles;   // warp tiles of one chunk (a block of 256 threads)

void launch_zmap(cudaStream_t st, const uint32_t *leaf_hi, const Info *info, uint32_t *zmap);
// a5 + a6: blocks, leaf ranges and candidate counts per query, scanned.
void launch_query_blocks(cudaStream_t st, const float4 *rects, uint32_t Q, float x0, float y0, float sx,
                         float sy, Worlds worlds, const uint32_t *leaf_lo, const uint32_t *leaf_hi, const uint32_t *zmap,
                         uint2 *qcells, unsigned long long *cand_off, uint32_t *pair_q,
                         uint32_t *pair_first, uint32_t *pair_blo, unsigned long long *pair_off,
                         uint32_t *qpair, uint32_t *tile_p0, unsigned long long tile_cap,
                         uint32_t *status_p, unsigned long long *status_c, uint32_t *tile_counter,
                         Info *info);
// a7: candidates (warp tiles of 32) -> subquery records (query-major),
// placed in one pass (chunks of tiles in ticket order, a look-back over the
// chunks' record counts in status[]), the first record of every pair
// (pair_rec[npairs+1]) and the per-leaf counts leaf_nsub.
// The work-item kernels (candidates, leaf lists, filter, emit) take their
// grid in blocks: they draw work from counters (or stride over it), so the
// grid only sets how many blocks are resident (mqr_set_launch_config).
constexpr int kDefaultBlocksPerSM = 8;
void launch_candidates(cudaStream_t st, int grid_blocks, int covering, const uint32_t *tile_p0,
                       const uint32_t *pair_q, const uint32_t *pair_first, const uint32_t *pair_blo,
                       const unsigned long long *pair_off, const uint2 *qcells, const uint2 *leaf_box,
                       const uint32_t *leaf_beg, uint32_t *leaf_nsub, uint32_t *pair_rec, uint32_t *sub_q,
                       uint32_t *sub_leaf, uint32_t *sub_len, uint32_t *sub_res, unsigned long long *status,
                       uint32_t *chunk_counter, Caps caps, Info *info);

// a8: scans over leaves -> leaf_sub_off, leaf_word_off, leaf_item_off, item_leaf.
constexpr int kLeafScanThreads = 256, kLeafScanItems = 8, kLeafScanTile = kLeafScanThreads * kLeafScanItems;
void launch_leaf_scan(cudaStream_t st, int num_sms, uint32_t nmax, const uint32_t *leaf_beg,
                      const uint32_t *leaf_nsub, uint32_t *leaf_sub_off, uint32_t *leaf_word_off,
                      uint32_t *leaf_item_off, uint32_t *item_leaf,
                      uint32_t *status3, uint32_t *tile_counter, Caps caps, Info *info);

// a8: the intersecting records into their leaves' lists (isub).
void launch_leaf_lists(cudaStream_t st, int grid_blocks, const uint32_t *sub_leaf, const uint32_t *sub_len,
                       const uint32_t *leaf_sub_off, uint32_t *isub, Caps caps, const Info *info);

// a10: filtering into bitmap words + per-subquery counts.
void launch_filter(cudaStream_t st, int grid_blocks, const float4 *rects, const float2 *sxy,
                   const uint32_t *leaf_beg, const uint32_t *leaf_sub_off,
                   const uint32_t *leaf_word_off, const uint32_t *leaf_item_off,
                   const uint32_t *item_leaf, const uint32_t *isub, const uint32_t *sub_q,
                   uint32_t *sub_res, uint32_t *bitmap, uint32_t *ticket, Caps caps, const Info *info);

// a11: result offsets out_off[k] (u64, exclusive) over subquery records.
// stall_test: the failure-handling test hook (mqr_debug_stall_scan): tile 0
// withholds its look-back status and the other tiles wait kStallWaitNs only,
// so their bounded waits run out and the tick reports a timeout.
constexpr int kResThreads = 256, kResItems = 8, kResTile = kResThreads * kResItems;
constexpr unsigned long long kStallWaitNs = 1000000ull;   // 1 ms
void launch_result_scan(cudaStream_t st, unsigned long long sub_cap, const uint32_t *sub_res,
                        const uint32_t *sub_leaf, unsigned long long *out_off,
                        unsigned long long *status, uint32_t *tile_counter, uint32_t run_elems, Caps caps, Info *info,
                        bool stall_test = false);

// a12 + a13: emit results in query-major order.
enum EmitKind { kEmitPairs = 0, kEmitIds = 1, kEmitBitmap = 2, kEmitKeys64 = 3, kEmitRuns = 4,
                kEmitAtomic = 5 /* the atomic-append baseline (no bitmaps, unordered pairs) */ };
void launch_emit(cudaStream_t st, int grid_blocks, int emit_kind, const uint32_t *sub_q,
                 const uint32_t *sub_leaf, const uint32_t *sub_len, const uint32_t *leaf_word_off,
                 const unsigned long long *out_off, const uint32_t *leaf_beg,
                 const uint32_t *sid, const uint32_t *bitmap, void *out, uint32_t bitmap_words_per_row,
                 uint32_t *ticket, Caps caps, const Info *info);

// The atomic-append baseline filtering (Alg. 3) and its covering runs.
void launch_atomic_baseline(cudaStream_t st, int num_sms, const float4 *rects, const float2 *sxy,
                            const uint32_t *sid, const uint32_t *leaf_beg, const uint32_t *leaf_sub_off,
                            const uint32_t *leaf_item_off, const uint32_t *item_leaf, const uint32_t *isub,
                            const uint32_t *sub_q, const uint32_t *sub_leaf, const uint32_t *sub_len, void *out,
                            unsigned long long cap, uint32_t *ticket, Caps caps, Info *info);

// Learned tick-cost model (k_cost.cu): MLP 5 -> 64 -> 64 -> 1.
size_t cost_param_count();
cudaError_t launch_cost_train(cudaStream_t st, float *params, float *m, float *v, uint32_t step0, const float *X,
                              const float *y, uint32_t n, uint32_t epochs, float lr, float *loss, float *grad);
cudaError_t launch_cost_predict(cudaStream_t st, const float *params, const float *X, uint32_t n, float *out);

// Admission by output memory: queries [0, A) whose output fits cap elements.
void launch_admit(cudaStream_t st, uint32_t Q, const unsigned long long *offsets, unsigned long long cap,
                  const uint32_t *qpair, const uint32_t *pair_rec, Caps caps, Info *info);

// Per-query offsets: off[q] = out_off[pair_rec[qpair[q]]].
void launch_query_offsets(cudaStream_t st, uint32_t Q, const uint32_t *qpair, const uint32_t *pair_rec,
                          const unsigned long long *out_off, unsigned long long *offsets, Caps caps,
                          const Info *info);

// (qidx << 32 | id) keys -> pairs (qidx, id) or ids.
void launch_keys_to_output(cudaStream_t st, const unsigned long long *keys, uint64_t n,
                           int as_pairs, void *out);

}  // namespace mqr
