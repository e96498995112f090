// mqr_api.cu -- the C ABI of libmqr (declared in include/mqr.h): context,
// device memory, and the per-tick pipeline
//   a2 Morton keys -> a3 onesweep sort (4 passes) -> a4 leaves ->
//   a5/a6 query count + scan -> a8 leaf scans -> a7 query write ->
//   a10 filter -> a11 result scan -> a12/a13 emit (-> a14 sort/layout)
// all enqueued on the context's stream with one host synchronisation at the
// end of the tick (the result count sizes the caller's output).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/mqr.h"
#include "mqr_internal.cuh"

using namespace mqr;

namespace {

thread_local std::string g_err;

mqr_status fail(mqr_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

mqr_status cuda_fail(cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(e == cudaErrorMemoryAllocation ? MQR_ERR_OOM : MQR_ERR_CUDA, m);
}

#define MQR_CUDA(call)                                         \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);    \
    } while (0)

// Bumped whenever any device buffer is (re)allocated or freed: a captured
// tick graph holds raw pointers, so it is only replayed while this is unchanged.
std::atomic<unsigned long long> g_buf_gen{0};
// Fault injection (mqr_debug_fail_allocation): the number of device buffer
// allocations still to succeed before one fails; negative: disarmed.
std::atomic<long long> g_fail_alloc_after{-1};
// Failure-handling test hook (mqr_debug_stall_scan): the next result scan
// runs with a withheld look-back status and a 1 ms wait limit.
std::atomic<bool> g_stall_scan{false};

// A device buffer that only grows (contents are not preserved on growth).
template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    cudaError_t ensure(size_t want) {
        if (want <= n) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        ++g_buf_gen;
        if (g_fail_alloc_after.load() >= 0 && g_fail_alloc_after.fetch_sub(1) == 0)
            return cudaErrorMemoryAllocation;      // injected failure (the hook disarms itself)
        cudaError_t e = cudaMalloc(&p, want * sizeof(T));
        if (e == cudaSuccess) n = want;
        return e;
    }
    void release() {
        if (p) { cudaFree(p); ++g_buf_gen; }
        p = nullptr;
        n = 0;
    }
};

size_t grow_to(unsigned long long need) { return (size_t)(need + need / 4 + 1024); }

}  // namespace

void mqr::set_last_error(const std::string &msg) { g_err = msg; }

struct mqr_ctx {
    int device = 0;
    int num_sms = 148;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    mqr_config cfg{};
    mqr_rect bounds{};
    float sx = 0.f, sy = 0.f;
    uint32_t nmax = 0;
    unsigned long long epoch = 0;

    // resident state
    DevBuf<float2> pos;
    DevBuf<unsigned long long> stamp;
    // sort
    DevBuf<unsigned long long> keysA, keysB;
    DevBuf<uint32_t> skey, sid, sort_counts, sort_offs;
    DevBuf<float2> sxy;
    // leaves
    DevBuf<uint32_t> leaf_lo, leaf_hi, leaf_beg, leaf_nsub, leaf_sub_off, leaf_word_off,
        leaf_item_off;
    DevBuf<uint8_t> mk_a, mk_b;
    DevBuf<uint2> leaf_box;
    // per query / subquery
    DevBuf<uint32_t> sub_q, sub_leaf, sub_len, sub_res, isub, bitmap, item_leaf;
    DevBuf<unsigned long long> out_off;
    // query splitting: coarse lookup table, per-query cells, (query, block) pairs
    DevBuf<uint32_t> zmap, pair_q, pair_first, pair_blo, pair_rec, qpair, tile_p0;
    DevBuf<uint2> qcells;
    DevBuf<unsigned long long> cand_off, pair_off;
    unsigned long long cand_tiles = 0;
    // zero-initialised arena: Info, histograms, tile counters, look-back status
    DevBuf<unsigned char> arena;
    // staging for the host-buffer entry points and the sorted output kinds
    DevBuf<uint32_t> up_ids;
    DevBuf<float2> up_xy;
    DevBuf<float4> q_rects;
    DevBuf<unsigned char> out_stage, out_stage2;     // host-output staging (two for the async path)
    DevBuf<unsigned long long> off_stage, off_stage2, sortA, sortB;
    cudaStream_t copy_stream = nullptr;              // device-to-host copies of mqr_tick_host_async
    DevBuf<uint32_t> sid_stage, sid_stage2;          // sorted-id snapshots copied by mqr_get_sorted_async
    cudaEvent_t snap_done = nullptr;
    cudaEvent_t copy_done[2] = {nullptr, nullptr};
    bool copy_pending[2] = {false, false};
    int next_stage = 0;
    DevBuf<unsigned char> sort_arena;
    DevBuf<unsigned long long> upd_err;  // sticky error word of the update kernels
    // captured tick (mqr_set_graph): replayed while its inputs are unchanged
    bool graph_on = false;
    // captured ticks, replayed while their inputs are unchanged: a few are
    // kept (least recently used evicted), so that ticks alternating between
    // output buffers (the two staging buffers of the asynchronous host path)
    // replay too
    static constexpr int kGraphCache = 4;
    struct GraphKey {
        const void *rects, *out, *offsets;
        unsigned long long Q, out_cap, gen, n_worlds;
        int emit_kind;
        uint32_t timing_mask;       // phases timed by event nodes of the graph (0: none)
        bool operator==(const GraphKey &o) const {
            return rects == o.rects && out == o.out && offsets == o.offsets && Q == o.Q &&
                   out_cap == o.out_cap && gen == o.gen && n_worlds == o.n_worlds && emit_kind == o.emit_kind &&
                   timing_mask == o.timing_mask;
        }
    };
    struct GraphEntry {
        GraphKey key{};
        cudaGraphExec_t exec = nullptr;
        Caps caps{};
        bool ev_phase[MQR_NUM_PHASES] = {};
        uint64_t ev_launches[MQR_NUM_PHASES] = {};
        uint64_t launches[MQR_NUM_PHASES] = {};
        unsigned long long used = 0;
    } graphs[kGraphCache];
    unsigned long long graph_clock = 0;
    unsigned long long graph_replays = 0, graph_captures = 0;
    // phase timing inside a captured tick: the timed phases' events are
    // external event-record nodes of the graph (recorded by every replay);
    // the other phases' launches are counted once at capture and added per replay
    bool capturing = false;
    bool graph_ev_phase[MQR_NUM_PHASES] = {};
    uint64_t graph_ev_launches[MQR_NUM_PHASES] = {};
    uint64_t graph_launches[MQR_NUM_PHASES] = {};
    // batched independent worlds (mqr_set_worlds): id and query ranges per world
    uint32_t n_worlds = 0, world_bits = 0;
    DevBuf<uint32_t> world_obj, world_q;
    // per-region leaf capacities (mqr_set_region_caps): 4^region_bits entries
    uint32_t region_bits = 0;
    DevBuf<uint32_t> region_cap, region_cnt;
    DevBuf<double> region_stats;
    DevBuf<uint8_t> fp_mark;        // mqr_result_footprint: leaf marks and the two sums
    DevBuf<unsigned long long> fp_sum;
    DevBuf<uint8_t> state_flags;    // staging of mqr_export_state / mqr_import_state
    int last_emit_kind = -1;
    // blocks per SM of the work-item kernels (mqr_set_launch_config)
    uint32_t bps_cand = kDefaultBlocksPerSM, bps_compact = kDefaultBlocksPerSM, bps_filter = kDefaultBlocksPerSM,
             bps_emit = kDefaultBlocksPerSM;
    unsigned long long world_q_total = 0;
    bool world_q_set = false;

    Info *info_host = nullptr;  // pinned
    Info last{};
    // per-phase timing (mqr_set_timing)
    bool timing = false;            // launch counting on (mqr_set_timing / mqr_set_timing_phases)
    uint32_t timing_mask = 0;       // the phases timed with events
    cudaEvent_t ev[MQR_NUM_PHASES][2] = {};
    bool ev_used[MQR_NUM_PHASES] = {};
    uint64_t ev_launches[MQR_NUM_PHASES] = {};
    static constexpr int kMaxPendingUpdates = 64;
    cudaEvent_t up_ev[kMaxPendingUpdates][2] = {};
    int up_pending = 0;
    uint64_t up_launches = 0;
    mqr_timing acc{};
    unsigned long long last_q = 0, retries = 0;
    bool have_tick = false;
    bool bad_id = false;   // an update id >= max_objects was seen since the last report
    // snapshots and join slots (mqr_snapshot, mqr_slot_*): a context's index is
    // shared read-only by its slots; snap_info holds the index counters of the
    // last snapshot (objects present, leaves, deepest level, error bits)
    cudaEvent_t snap_ready = nullptr;
    DevBuf<unsigned long long> snap_info;
    bool have_snapshot = false;
    bool snap_pending = false;      // a snapshot was enqueued after the last completed tick
    bool index_valid = false;       // c->last's index counters describe the current index
    std::vector<mqr_ctx *> slots;
    // a slot: its context, the event after its last join, the pending join
    mqr_ctx *parent = nullptr;
    cudaEvent_t slot_done = nullptr;
    bool slot_busy = false;
    struct SlotJob {
        const float4 *rects;
        uint32_t Q;
        int emit_kind, kind;
        void *out;
        unsigned long long cap;
        unsigned long long *offsets;
        Caps caps;
    } job{};
};

namespace {

// The object sort runs its passes with look-back up to this many tiles.
constexpr uint32_t kSortLookbackTiles = 16;

// Arena layout for one tick.
struct Arena {
    size_t info, hist, counters, st_sort, st_leaf, st_lscan, st_qb_p, st_qb_c, st_cand, st_res, total;
    uint32_t sort_tiles, leaf_tiles, lscan_tiles, qb_tiles, res_tiles;
    unsigned long long cand_tiles;
};

Arena arena_layout(uint32_t nmax, uint32_t Q, unsigned long long sub_cap, unsigned long long cand_tiles) {
    Arena a{};
    a.sort_tiles = (nmax + kSortTile - 1) / kSortTile;
    a.leaf_tiles = (nmax + kLeafTile - 1) / kLeafTile;
    a.lscan_tiles = (nmax + kLeafScanTile - 1) / kLeafScanTile;
    a.qb_tiles = (Q + kQBQueries - 1) / kQBQueries;
    a.cand_tiles = cand_tiles;
    a.res_tiles = (uint32_t)((sub_cap + kResTile - 1) / kResTile) + 1;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o += (bytes + 255) & ~(size_t)255;
        return r;
    };
    a.info = take(sizeof(Info));
    a.hist = take(8 * 256 * sizeof(uint32_t));
    a.counters = take(16 * sizeof(uint32_t));
    // look-back status of the object sort's four passes, when it runs them
    // with look-back (a few tiles: see enqueue_index)
    a.st_sort = take(a.sort_tiles <= kSortLookbackTiles ? (size_t)4 * 256 * a.sort_tiles * sizeof(uint32_t) : 0);
    a.st_leaf = take((size_t)a.leaf_tiles * sizeof(uint32_t));
    a.st_lscan = take((size_t)3 * a.lscan_tiles * sizeof(uint32_t));
    a.st_qb_p = take((size_t)a.qb_tiles * sizeof(uint32_t));
    a.st_qb_c = take((size_t)a.qb_tiles * sizeof(unsigned long long));
    a.st_cand = take((size_t)((a.cand_tiles + kCandChunkTiles - 1) / kCandChunkTiles + 1) *
                     sizeof(unsigned long long));
    a.st_res = take((size_t)a.res_tiles * sizeof(unsigned long long));
    a.total = o;
    return a;
}

template <typename T>
T *at(mqr_ctx *c, size_t off) {
    return reinterpret_cast<T *>(c->arena.p + off);
}

mqr_status check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, what);
    return MQR_OK;
}

// Phase timing: events around the kernels of the phases in timing_mask;
// launches are counted for every phase while timing is on.
// While a tick is captured into a graph, the records become external
// event-record nodes, so that every replay records them.
void record_phase_event(mqr_ctx *c, cudaEvent_t ev) {
    if (c->capturing) cudaEventRecordWithFlags(ev, c->stream, cudaEventRecordExternal);
    else cudaEventRecord(ev, c->stream);
}
void phase_begin(mqr_ctx *c, int p) {
    if (!c->timing || !(c->timing_mask & (1u << p))) return;
    record_phase_event(c, c->ev[p][0]);
}
void phase_end(mqr_ctx *c, int p, uint64_t launches) {
    if (!c->timing) return;
    if (c->timing_mask & (1u << p)) {
        record_phase_event(c, c->ev[p][1]);
        if (c->capturing) {
            c->graph_ev_phase[p] = true;
            c->graph_ev_launches[p] = launches;
        } else {
            c->ev_used[p] = true;
            c->ev_launches[p] = launches;
        }
    } else if (c->capturing) {
        c->graph_launches[p] += launches;
    } else {
        c->acc.launches[p] += launches;
    }
}
// After a graph launch: the replay recorded the timed phases' events and
// launched the captured kernels.
void phases_replayed(mqr_ctx *c, const mqr_ctx::GraphEntry &g) {
    if (!c->timing) return;
    for (int p = 0; p < MQR_NUM_PHASES; ++p) {
        if (g.ev_phase[p]) {
            c->ev_used[p] = true;
            c->ev_launches[p] = g.ev_launches[p];
        }
        c->acc.launches[p] += g.launches[p];
    }
}

void free_graphs(mqr_ctx *c) {
    for (auto &g : c->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = mqr_ctx::GraphEntry{};
    }
}
// Called after the stream has been synchronised: fold the recorded phases
// (and the update calls since the last tick) into the accumulators.
void phases_collect(mqr_ctx *c, bool count_tick) {
    if (!c->timing) return;
    for (int p = 0; p < MQR_NUM_PHASES; ++p) {
        if (!c->ev_used[p]) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev[p][0], c->ev[p][1]) == cudaSuccess) {
            c->acc.ms[p] += ms;
            c->acc.launches[p] += c->ev_launches[p];
        }
        c->ev_used[p] = false;
    }
    for (int k = 0; k < c->up_pending; ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->up_ev[k][0], c->up_ev[k][1]) == cudaSuccess)
            c->acc.ms[MQR_PHASE_UPDATES] += ms;
    }
    c->acc.launches[MQR_PHASE_UPDATES] += c->up_launches;
    c->up_pending = 0;
    c->up_launches = 0;
    if (count_tick) c->acc.ticks++;
}

bool finite_rect(const mqr_rect &b) {
    return std::isfinite(b.xmin) && std::isfinite(b.ymin) && std::isfinite(b.xmax) &&
           std::isfinite(b.ymax) && b.xmax > b.xmin && b.ymax > b.ymin;
}

// scale = 2^15 / (hi - lo), each operation rounded to float32.
float fp32_scale(float lo, float hi) {
    volatile float w = hi - lo;
    volatile float s = 32768.0f / w;
    return s;
}

uint32_t bitmap_words_per_row(uint32_t nmax) { return (nmax + 31u) / 32u; }

size_t out_elem_bytes(int kind) {
    switch (kind) {
        case MQR_OUT_PAIRS:
        case MQR_OUT_PAIRS_SORTED:
        case MQR_OUT_RUNS:
        case MQR_OUT_PAIRS_ATOMIC: return 8;
        case MQR_OUT_CSR:
        case MQR_OUT_CSR_SORTED: return 4;
        default: return 4;
    }
}

// Wait (on the context's stream) until no slot still reads the index that
// the next index build overwrites.
mqr_status wait_for_slots(mqr_ctx *c) {
    for (mqr_ctx *sl : c->slots)
        if (sl->slot_done) MQR_CUDA(cudaStreamWaitEvent(c->stream, sl->slot_done, 0));
    return MQR_OK;
}

// a2 - a4: Morton keys, the onesweep sort and the leaves of the current
// state, then the snapshot's counters for the slots.  The arena is zeroed and
// the update kernels' error bits carried in first.
mqr_status enqueue_index(mqr_ctx *c, const Arena &a) {
    cudaStream_t st = c->stream;
    Info *info = at<Info>(c, a.info);
    uint32_t *hist = at<uint32_t>(c, a.hist);
    uint32_t *ctr = at<uint32_t>(c, a.counters);
    unsigned long long *err = &info->err;
    const float x0 = c->bounds.xmin, y0 = c->bounds.ymin;
    const uint32_t nmax = c->nmax;
    mqr_status s = wait_for_slots(c);
    if (s != MQR_OK) return s;
    MQR_CUDA(cudaMemsetAsync(c->arena.p, 0, a.total, st));
    // Carry the update kernels' sticky error bits into this tick.
    MQR_CUDA(cudaMemcpyAsync(&info->err, c->upd_err.p, sizeof(unsigned long long),
                             cudaMemcpyDeviceToDevice, st));
    MQR_CUDA(cudaMemsetAsync(c->upd_err.p, 0, sizeof(unsigned long long), st));

    // a2 + a3: keys and the 4-pass onesweep sort of (key << 32 | id).
    phase_begin(c, MQR_PHASE_KEYS);
    const Worlds worlds{c->world_obj.p, c->world_q.p, c->n_worlds, c->world_bits};
    launch_morton_keys(st, c->pos.p, c->stamp.p, nmax, x0, y0, c->sx, c->sy, worlds, c->keysA.p, hist,
                       c->sort_counts.p, info);
    phase_end(c, MQR_PHASE_KEYS, nmax ? 1 : 0);
    unsigned long long *src = c->keysA.p, *dst = c->keysB.p;
    phase_begin(c, MQR_PHASE_SORT);
    // A few tiles: each pass's tiles look back over one another (one launch
    // per pass; the walk is short); more: the look-back-free passes (tile
    // counts, digit scan, rank and scatter), whose tiles need not wait.
    const bool sort_lookback = a.sort_tiles <= kSortLookbackTiles;
    uint32_t *st_sort = at<uint32_t>(c, a.st_sort);
    for (int p = 0; p < 4; ++p) {
        const bool fin = p == 3;
        if (sort_lookback)
            launch_onesweep_pass(st, src, dst, nmax, 32 + 8 * p, hist + 256 * p,
                                 st_sort + (size_t)256 * a.sort_tiles * p, ctr + p, err, fin, c->pos.p, c->skey.p,
                                 c->sid.p, c->sxy.p);
        else
            launch_sort_pass_pre(st, src, dst, nmax, 32 + 8 * p, hist + 256 * p, c->sort_counts.p,
                                 c->sort_offs.p, err, fin, c->pos.p, c->skey.p, c->sid.p, c->sxy.p, p == 0);
        std::swap(src, dst);
    }
    // the look-back-free passes: the first pass's tile counts come from the key kernel
    phase_end(c, MQR_PHASE_SORT, nmax ? (sort_lookback ? 4 : 11) : 0);
    // a4
    phase_begin(c, MQR_PHASE_LEAVES);
    const uint32_t cap = c->cfg.leaf_cap;
    const bool ug = c->cfg.index_kind == MQR_INDEX_UNIFORM_GRID;
    const uint32_t rbits = ug ? 0 : c->region_bits;          // region capacities refine the quadtree only
    launch_build_leaves(st, c->skey.p, nmax, cap, ug, c->cfg.grid_level, std::max(c->world_bits, rbits), rbits,
                        c->region_cap.p, c->mk_a.p, c->mk_b.p,
                        at<uint32_t>(c, a.st_leaf), ctr + 4, c->leaf_lo.p, c->leaf_hi.p, c->leaf_beg.p,
                        c->leaf_nsub.p, c->leaf_box.p, info);
    uint64_t leaf_launches = nmax ? 1 : 0;
    if (nmax && !ug && !rbits && cap > (uint32_t)kLeafCapSmem && cap < nmax) {
        int kexp = 0;
        while ((2ull << kexp) <= (unsigned long long)cap + 1) ++kexp;
        leaf_launches += 1 + kexp;
    }
    phase_end(c, MQR_PHASE_LEAVES, leaf_launches);
    if (!c->slots.empty()) {
        // the index counters (n_present, n_leaves, max_level) and the error bits for the slots
        MQR_CUDA(cudaMemcpyAsync(c->snap_info.p, info, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st));
        MQR_CUDA(cudaMemcpyAsync(c->snap_info.p + 3, &info->err, sizeof(unsigned long long),
                                 cudaMemcpyDeviceToDevice, st));
        MQR_CUDA(cudaEventRecord(c->snap_ready, st));
    }
    return check_launch("index kernels");
}

// a5 - a14 for Q queries against the index of ix (ix == c for a plain tick,
// the slot's context for a slot): query splitting, grouping, filtering, the
// result scan and the emit.  admit: the output is limited to the longest
// prefix of queries that fits out_cap_elems (per-query offsets, then the
// admission kernel, then the emit of the admitted records: no host round
// trip); offsets is then required.
mqr_status enqueue_join(mqr_ctx *c, const mqr_ctx *ix, const float4 *rects, uint32_t Q, int emit_kind, void *out,
                        unsigned long long out_cap_elems, unsigned long long *offsets, const Arena &a, Caps &caps,
                        bool admit) {
    cudaStream_t st = c->stream;
    Info *info = at<Info>(c, a.info);
    // tile/ticket counters: 0-3 sort passes, 4 leaves, 5 query blocks, 6 leaf scan, 7 result scan,
    // 8 candidate scan, 9 emit batches, 10 filter items; 12-13 the output sort's error word
    uint32_t *ctr = at<uint32_t>(c, a.counters);
    const float x0 = c->bounds.xmin, y0 = c->bounds.ymin;
    const uint32_t nmax = c->nmax;
    const int cov = c->cfg.covering ? 1 : 0;
    const Worlds worlds{ix->world_obj.p, ix->world_q.p, ix->n_worlds, ix->world_bits};
    // a5 + a6: coarse lookup table, blocks and candidate counts per query
    caps.sub = c->sub_q.n;
    caps.sub_i = c->isub.n;
    caps.words = std::min<size_t>(c->bitmap.n, 0xffffffffull);
    caps.out = out_cap_elems;
    caps.cand_tiles = a.cand_tiles;
    caps.items = c->item_leaf.n;
    phase_begin(c, MQR_PHASE_QUERY_BLOCKS);
    launch_zmap(st, ix->leaf_hi.p, info, c->zmap.p);
    launch_query_blocks(st, rects, Q, x0, y0, c->sx, c->sy, worlds, ix->leaf_lo.p, ix->leaf_hi.p, c->zmap.p,
                        c->qcells.p, c->cand_off.p, c->pair_q.p, c->pair_first.p, c->pair_blo.p,
                        c->pair_off.p, c->qpair.p, c->tile_p0.p, a.cand_tiles,
                        at<uint32_t>(c, a.st_qb_p), at<unsigned long long>(c, a.st_qb_c), ctr + 5, info);
    phase_end(c, MQR_PHASE_QUERY_BLOCKS, Q ? 2 : 1);
    // a7: candidates -> subquery records
    phase_begin(c, MQR_PHASE_CANDIDATES);
    if (c != ix)      // a slot's per-leaf subquery counts start at zero (the index build zeroes its own)
        MQR_CUDA(cudaMemsetAsync(c->leaf_nsub.p, 0, (size_t)std::max<uint32_t>(nmax, 1) * sizeof(uint32_t), st));
    launch_candidates(st, c->num_sms * (int)c->bps_cand, cov, c->tile_p0.p, c->pair_q.p, c->pair_first.p, c->pair_blo.p,
                      c->pair_off.p, c->qcells.p, ix->leaf_box.p, ix->leaf_beg.p, c->leaf_nsub.p, c->pair_rec.p,
                      c->sub_q.p, c->sub_leaf.p, c->sub_len.p, c->sub_res.p,
                      at<unsigned long long>(c, a.st_cand), ctr + 8, caps, info);
    phase_end(c, MQR_PHASE_CANDIDATES, 1);
    // a8: group intersecting subqueries by leaf: the leaves' list offsets,
    // then every intersecting record into its leaf's list
    phase_begin(c, MQR_PHASE_GROUP);
    launch_leaf_scan(st, c->num_sms, nmax, ix->leaf_beg.p, c->leaf_nsub.p, c->leaf_sub_off.p, c->leaf_word_off.p,
                     c->leaf_item_off.p, c->item_leaf.p, at<uint32_t>(c, a.st_lscan), ctr + 6, caps, info);
    launch_leaf_lists(st, c->num_sms * (int)c->bps_compact, c->sub_leaf.p, c->sub_len.p, c->leaf_sub_off.p,
                      c->isub.p, caps, info);
    phase_end(c, MQR_PHASE_GROUP, nmax ? 2 : 1);
    // a10
    if (emit_kind == kEmitAtomic) {
        // the atomic-append baseline: no bitmaps, no result scan, no decoding
        phase_begin(c, MQR_PHASE_FILTER);
        launch_atomic_baseline(st, c->num_sms, rects, ix->sxy.p, ix->sid.p, ix->leaf_beg.p, c->leaf_sub_off.p,
                               c->leaf_item_off.p, c->item_leaf.p, c->isub.p, c->sub_q.p, c->sub_leaf.p,
                               c->sub_len.p, out, out ? out_cap_elems : 0, ctr + 10, caps, info);
        phase_end(c, MQR_PHASE_FILTER, 2);
        return check_launch("tick kernels");
    }
    phase_begin(c, MQR_PHASE_FILTER);
    launch_filter(st, c->num_sms * (int)c->bps_filter, rects, ix->sxy.p, ix->leaf_beg.p, c->leaf_sub_off.p,
                  c->leaf_word_off.p, c->leaf_item_off.p, c->item_leaf.p, c->isub.p, c->sub_q.p, c->sub_res.p,
                  c->bitmap.p, ctr + 10, caps, info);
    phase_end(c, MQR_PHASE_FILTER, 1);
    // a11
    phase_begin(c, MQR_PHASE_RESULT_SCAN);
    launch_result_scan(st, caps.sub, c->sub_res.p, c->sub_leaf.p, c->out_off.p,
                       at<unsigned long long>(c, a.st_res), ctr + 7, emit_kind == kEmitRuns ? 2u : 0u, caps,
                       info, g_stall_scan.exchange(false));
    phase_end(c, MQR_PHASE_RESULT_SCAN, 1);
    if (admit) {
        // per-query offsets, then the longest prefix of queries that fits
        phase_begin(c, MQR_PHASE_OFFSETS);
        launch_query_offsets(st, Q, c->qpair.p, c->pair_rec.p, c->out_off.p, offsets, caps, info);
        launch_admit(st, Q, offsets, out ? out_cap_elems : 0, c->qpair.p, c->pair_rec.p, caps, info);
        phase_end(c, MQR_PHASE_OFFSETS, 2);
    }
    // a12 + a13
    if (out != nullptr && emit_kind >= 0) {
        phase_begin(c, MQR_PHASE_EMIT);
        launch_emit(st, c->num_sms * (int)c->bps_emit, emit_kind, c->sub_q.p, c->sub_leaf.p, c->sub_len.p, c->leaf_word_off.p,
                    c->out_off.p, ix->leaf_beg.p, ix->sid.p, c->bitmap.p, out,
                    bitmap_words_per_row(nmax), ctr + 9, caps, info);
        phase_end(c, MQR_PHASE_EMIT, 1);
    }
    if (offsets != nullptr && !admit) {
        phase_begin(c, MQR_PHASE_OFFSETS);
        launch_query_offsets(st, Q, c->qpair.p, c->pair_rec.p, c->out_off.p, offsets, caps, info);
        phase_end(c, MQR_PHASE_OFFSETS, 1);
    }
    return check_launch("tick kernels");
}

// The whole pipeline of a plain tick: the index, then the join.  Returns
// after enqueueing.
mqr_status enqueue_tick(mqr_ctx *c, const float4 *rects, uint32_t Q, int emit_kind, void *out,
                        unsigned long long out_cap_elems, unsigned long long *offsets,
                        const Arena &a, Caps &caps, bool admit) {
    mqr_status s = enqueue_index(c, a);
    if (s != MQR_OK) return s;
    return enqueue_join(c, c, rects, Q, emit_kind, out, out_cap_elems, offsets, a, caps, admit);
}

// A slot's join against its context's last snapshot: the slot waits for the
// snapshot, takes its index counters and error bits, then runs the join on
// its own stream and buffers.
mqr_status enqueue_slot(mqr_ctx *c, const float4 *rects, uint32_t Q, int emit_kind, void *out,
                        unsigned long long out_cap_elems, unsigned long long *offsets, const Arena &a, Caps &caps) {
    const mqr_ctx *ix = c->parent;
    Info *info = at<Info>(c, a.info);
    MQR_CUDA(cudaMemsetAsync(c->arena.p, 0, a.total, c->stream));
    MQR_CUDA(cudaStreamWaitEvent(c->stream, ix->snap_ready, 0));
    MQR_CUDA(cudaMemcpyAsync(info, ix->snap_info.p, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                             c->stream));
    MQR_CUDA(cudaMemcpyAsync(&info->err, ix->snap_info.p + 3, sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                             c->stream));
    return enqueue_join(c, ix, rects, Q, emit_kind, out, out_cap_elems, offsets, a, caps, true);
}

// Make sure every per-tick buffer that depends on Q or on the capacities
// exists.
mqr_status ensure_tick_buffers(mqr_ctx *c, uint32_t Q) {
    size_t sub0 = std::max<size_t>(4096, (size_t)Q * 4);
    MQR_CUDA(c->zmap.ensure(kZCells + 1));
    MQR_CUDA(c->qcells.ensure(std::max<size_t>(Q, 1)));
    MQR_CUDA(c->cand_off.ensure((size_t)Q + 1));
    MQR_CUDA(c->qpair.ensure((size_t)Q + 1));
    MQR_CUDA(c->pair_q.ensure((size_t)Q * 9 + 1));
    MQR_CUDA(c->pair_first.ensure((size_t)Q * 9 + 1));
    MQR_CUDA(c->pair_blo.ensure((size_t)Q * 9 + 1));
    MQR_CUDA(c->pair_off.ensure((size_t)Q * 9 + 1));
    MQR_CUDA(c->pair_rec.ensure((size_t)Q * 9 + 2));
    c->cand_tiles = std::min<unsigned long long>(
        std::max<unsigned long long>(c->cand_tiles, std::max<unsigned long long>(1 << 16, 2ull * Q)), kMaxCandTiles);
    MQR_CUDA(c->tile_p0.ensure(c->cand_tiles));
    if (c->sub_q.n == 0) {
        MQR_CUDA(c->sub_q.ensure(sub0));
        MQR_CUDA(c->sub_leaf.ensure(sub0));
        MQR_CUDA(c->sub_len.ensure(sub0));
        MQR_CUDA(c->sub_res.ensure(sub0));
        MQR_CUDA(c->out_off.ensure(sub0 + 1));
        MQR_CUDA(c->isub.ensure(sub0));
        MQR_CUDA(c->bitmap.ensure(std::max<size_t>(1 << 16, (size_t)Q * 16)));
        MQR_CUDA(c->item_leaf.ensure(std::max<size_t>(1 << 16, (size_t)Q)));
    }
    return MQR_OK;
}

mqr_status grow_sub(mqr_ctx *c, unsigned long long need) {
    size_t n = grow_to(need);
    c->sub_q.release(); c->sub_leaf.release(); c->sub_len.release(); c->sub_res.release();
    c->out_off.release();
    MQR_CUDA(c->sub_q.ensure(n));
    MQR_CUDA(c->sub_leaf.ensure(n));
    MQR_CUDA(c->sub_len.ensure(n));
    MQR_CUDA(c->sub_res.ensure(n));
    MQR_CUDA(c->out_off.ensure(n + 1));
    return MQR_OK;
}

// Enqueue the tick's kernels, or, in graph mode (and without phase timing),
// replay the tick captured for the same inputs and buffers: one graph launch
// instead of ~20 kernel launches.  The first tick of a new shape is captured
// (relaxed capture mode), instantiated and launched.
mqr_status enqueue_or_replay(mqr_ctx *c, const float4 *rects, uint32_t Q, int emit_kind, void *out,
                             unsigned long long out_cap_elems, unsigned long long *offsets, const Arena &a,
                             Caps &caps, bool admit) {
    // slots wait on the index build through events, which a replayed graph does not record
    if (!c->graph_on || g_stall_scan.load() || !c->slots.empty() || admit)
        return enqueue_tick(c, rects, Q, emit_kind, out, out_cap_elems, offsets, a, caps, admit);
    // The captured tick reads the queries from the context's own buffer, so a
    // caller that passes each tick's queries in a different buffer still
    // replays the same graph (one device-to-device copy of 16 B per query).
    MQR_CUDA(c->q_rects.ensure(std::max<size_t>(Q, 1)));
    const float4 *staged = reinterpret_cast<const float4 *>(c->q_rects.p);
    if (Q && rects != staged)
        MQR_CUDA(cudaMemcpyAsync(c->q_rects.p, rects, (size_t)Q * sizeof(float4), cudaMemcpyDeviceToDevice,
                                 c->stream));
    rects = staged;
    const mqr_ctx::GraphKey key{rects, out, offsets, Q, out_cap_elems, g_buf_gen.load(), c->n_worlds, emit_kind,
                                c->timing ? c->timing_mask : 0u};
    mqr_ctx::GraphEntry *ge = nullptr;
    for (auto &g : c->graphs)
        if (g.exec && g.key == key) ge = &g;
    if (!ge) {
        ge = &c->graphs[0];                   // a free entry, else the least recently used
        for (auto &g : c->graphs)
            if (!g.exec || (ge->exec && g.used < ge->used)) ge = &g;
        if (ge->exec) cudaGraphExecDestroy(ge->exec);
        *ge = mqr_ctx::GraphEntry{};
        MQR_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
        std::memset(c->graph_ev_phase, 0, sizeof(c->graph_ev_phase));
        std::memset(c->graph_ev_launches, 0, sizeof(c->graph_ev_launches));
        std::memset(c->graph_launches, 0, sizeof(c->graph_launches));
        c->capturing = true;
        mqr_status s = enqueue_tick(c, rects, Q, emit_kind, out, out_cap_elems, offsets, a, caps, false);
        c->capturing = false;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (s != MQR_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&ge->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            ge->exec = nullptr;
            return cuda_fail(e, "cudaGraphInstantiate");
        }
        ge->key = key;
        ge->caps = caps;
        std::memcpy(ge->ev_phase, c->graph_ev_phase, sizeof(ge->ev_phase));
        std::memcpy(ge->ev_launches, c->graph_ev_launches, sizeof(ge->ev_launches));
        std::memcpy(ge->launches, c->graph_launches, sizeof(ge->launches));
        ++c->graph_captures;
    } else {
        caps = ge->caps;
        ++c->graph_replays;
    }
    ge->used = ++c->graph_clock;
    MQR_CUDA(cudaGraphLaunch(ge->exec, c->stream));
    phases_replayed(c, *ge);
    return MQR_OK;
}

// One attempt of a tick (or of a slot's join): enqueue its kernels and the
// copy of its counters to the host.  Returns after enqueueing.
mqr_status attempt_enqueue(mqr_ctx *c, const float4 *rects, uint32_t Q, int emit_kind, void *out,
                           unsigned long long out_cap_elems, unsigned long long *offsets, bool admit, Caps &caps) {
    Arena a = arena_layout(c->nmax, Q, c->sub_q.n, c->cand_tiles);
    MQR_CUDA(c->arena.ensure(a.total));
    caps = Caps{};
    mqr_status s = c->parent ? enqueue_slot(c, rects, Q, emit_kind, out, out_cap_elems, offsets, a, caps)
                             : enqueue_or_replay(c, rects, Q, emit_kind, out, out_cap_elems, offsets, a, caps, admit);
    if (s != MQR_OK) return s;
    MQR_CUDA(cudaMemcpyAsync(c->info_host, c->arena.p + a.info, sizeof(Info), cudaMemcpyDeviceToHost, c->stream));
    return MQR_OK;
}

// After the stream has completed an attempt: its errors, and whether an
// internal buffer was too small (then it is grown and *again is set: the
// attempt must be repeated).
mqr_status attempt_check(mqr_ctx *c, uint32_t Q, int emit_kind, const Caps &caps, bool *again) {
    *again = false;
    Info in = *c->info_host;
    c->last = in;
    c->last_q = Q;
    c->last_emit_kind = emit_kind;
    c->have_tick = true;
    c->index_valid = true;
    c->snap_pending = false;
    if (in.err & kErrTimeout) return fail(MQR_ERR_TIMEOUT, "a device-side wait exceeded its deadline");
    if (in.err & kErrInternal) return fail(MQR_ERR_INTERNAL, "device index out of range");
    if (in.err & kErrBadId) c->bad_id = true;
    const unsigned long long need_tiles = (in.n_cand + 31) / 32;
    if (need_tiles > caps.cand_tiles) {
        if (need_tiles > kMaxCandTiles)
            return fail(MQR_ERR_INVALID_ARG, "too many candidate leaves in one tick (limit 2^32)");
        c->cand_tiles = std::min<unsigned long long>(grow_to(need_tiles), kMaxCandTiles);
        c->tile_p0.release();
        MQR_CUDA(c->tile_p0.ensure(c->cand_tiles));
        *again = true;
    } else if (in.n_sub > caps.sub) {
        mqr_status s = grow_sub(c, in.n_sub);
        if (s != MQR_OK) return s;
        *again = true;
    } else {
        if (in.n_sub_i > caps.sub_i) {
            c->isub.release();
            MQR_CUDA(c->isub.ensure(grow_to(in.n_sub_i)));
            *again = true;
        }
        if (in.n_items > caps.items) {
            c->item_leaf.release();
            MQR_CUDA(c->item_leaf.ensure(grow_to(in.n_items)));
            *again = true;
        }
        if (in.n_words > caps.words) {
            if (in.n_words > 0xffffffffull)
                return fail(MQR_ERR_CAPACITY, "more than 2^32 bitmap words in one tick");
            c->bitmap.release();
            MQR_CUDA(c->bitmap.ensure(grow_to(in.n_words)));
            *again = true;
        }
    }
    return MQR_OK;
}

// Run the pipeline until every internal buffer was large enough; leaves the
// tick's device state valid and c->last filled.  `out` may be null (then
// nothing is emitted).  admit: see enqueue_join.
mqr_status run_tick(mqr_ctx *c, const float4 *rects, uint32_t Q, int emit_kind, void *out,
                    unsigned long long out_cap_elems, unsigned long long *offsets, bool admit = false) {
    mqr_status s = ensure_tick_buffers(c, Q);
    if (s != MQR_OK) return s;
    c->retries = 0;
    for (int attempt = 0; attempt < 8; ++attempt) {
        Caps caps{};
        s = attempt_enqueue(c, rects, Q, emit_kind, out, out_cap_elems, offsets, admit, caps);
        if (s != MQR_OK) return s;
        MQR_CUDA(cudaStreamSynchronize(c->stream));
        bool again = false;
        s = attempt_check(c, Q, emit_kind, caps, &again);
        if (s != MQR_OK) return s;
        if (!again) {
            phases_collect(c, true);
            return MQR_OK;
        }
        ++c->retries;
    }
    return fail(MQR_ERR_INTERNAL, "buffer growth did not converge");
}

// Sort n keys (qidx << 32 | id) in sortA: digits over the id bits and the
// qidx bits only.  Result ends in *result.
mqr_status sort_result_keys(mqr_ctx *c, uint64_t n, uint32_t Q, unsigned long long **result) {
    *result = c->sortA.p;
    if (n <= 1) return MQR_OK;
    int shifts[8], nd = 0;
    uint32_t idbits = 1;
    while (idbits < 32 && (1ull << idbits) < c->nmax) ++idbits;
    uint32_t qbits = 1;
    while (qbits < 32 && (1ull << qbits) < Q) ++qbits;
    for (uint32_t b = 0; b < idbits; b += 8) shifts[nd++] = (int)b;
    for (uint32_t b = 0; b < qbits; b += 8) shifts[nd++] = 32 + (int)b;
    uint32_t tiles = (uint32_t)((n + kSortTile - 1) / kSortTile);
    size_t hist_off = 0, ctr_off = 8 * 256 * sizeof(uint32_t);
    size_t st_off = ctr_off + 256;
    size_t total = st_off + (size_t)nd * 256 * tiles * sizeof(uint32_t);
    MQR_CUDA(c->sort_arena.ensure(total));
    MQR_CUDA(cudaMemsetAsync(c->sort_arena.p, 0, total, c->stream));
    uint32_t *hist = reinterpret_cast<uint32_t *>(c->sort_arena.p + hist_off);
    uint32_t *ctr = reinterpret_cast<uint32_t *>(c->sort_arena.p + ctr_off);
    uint32_t *stp = reinterpret_cast<uint32_t *>(c->sort_arena.p + st_off);
    launch_key_histograms(c->stream, c->sortA.p, (uint32_t)n, shifts, nd, hist);
    unsigned long long *src = c->sortA.p, *dst = c->sortB.p;
    // error word of this sort: a dedicated slot in its counters block
    unsigned long long *err = reinterpret_cast<unsigned long long *>(ctr + 12);
    for (int d = 0; d < nd; ++d) {
        launch_onesweep_pass(c->stream, src, dst, (uint32_t)n, shifts[d], hist + 256 * d,
                             stp + (size_t)256 * tiles * d, ctr + d, err, false, nullptr, nullptr,
                             nullptr, nullptr);
        std::swap(src, dst);
    }
    *result = src;
    mqr_status s = check_launch("result sort");
    if (s != MQR_OK) return s;
    unsigned long long herr = 0;
    MQR_CUDA(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, c->stream));
    MQR_CUDA(cudaStreamSynchronize(c->stream));
    if (herr & kErrTimeout) return fail(MQR_ERR_TIMEOUT, "a device-side wait exceeded its deadline");
    if (herr) return fail(MQR_ERR_INTERNAL, "device index out of range in the result sort");
    return MQR_OK;
}

// The index counters of the latest index build (a tick's or a snapshot's)
// in c->last; waits for a pending snapshot.
mqr_status index_ready(mqr_ctx *c) {
    if (c->snap_pending) {
        unsigned long long h[4] = {0, 0, 0, 0};
        MQR_CUDA(cudaMemcpyAsync(h, c->snap_info.p, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
        MQR_CUDA(cudaStreamSynchronize(c->stream));
        c->last.n_present = h[0];
        c->last.n_leaves = h[1];
        c->last.max_level = h[2];
        c->snap_pending = false;
        c->index_valid = true;
        c->have_tick = false;       // the join records no longer match the index
    }
    if (!c->index_valid) return fail(MQR_ERR_INVALID_ARG, "no tick or snapshot has completed yet");
    return MQR_OK;
}

// Queries answered and output elements written by an admitted tick: the
// admission kernel marks emit_end (bit 63 set) when the output had to be cut.
void admission_counts(const Info &in, uint32_t Q, uint32_t *admitted, uint64_t *out_count) {
    if (in.emit_end) {
        *admitted = (uint32_t)in.admitted;
        *out_count = in.admitted_out;
    } else {
        *admitted = Q;
        *out_count = in.n_out;
    }
}

mqr_status tick_device_impl(mqr_ctx *c, const float *rects_dev, uint32_t Q, int kind, void *out_dev,
                            uint64_t cap_bytes, uint64_t *out_count, uint64_t *offsets_dev) {
    const float4 *rects = reinterpret_cast<const float4 *>(rects_dev);
    unsigned long long *offs = reinterpret_cast<unsigned long long *>(offsets_dev);
    const uint32_t wpr = bitmap_words_per_row(c->nmax);
    if (kind == MQR_OUT_BITMAP) {
        uint64_t words = (uint64_t)Q * wpr;
        *out_count = words;
        if (cap_bytes < words * 4) return fail(MQR_ERR_CAPACITY, "bitmap output buffer too small");
        if (words && out_dev == nullptr) return fail(MQR_ERR_INVALID_ARG, "out_dev is NULL");
        if (words) MQR_CUDA(cudaMemsetAsync(out_dev, 0, words * 4, c->stream));
        return run_tick(c, rects, Q, kEmitBitmap, out_dev, words, offs);
    }
    if (kind == MQR_OUT_COUNT) {
        mqr_status s = run_tick(c, rects, Q, -1, nullptr, 0, offs);
        *out_count = c->last.n_results;
        return s;
    }
    if (kind == MQR_OUT_PAIRS_ATOMIC) {
        if (offs) return fail(MQR_ERR_INVALID_ARG, "the unordered PAIRS_ATOMIC kind has no per-query offsets");
        if (out_dev && (reinterpret_cast<uintptr_t>(out_dev) & 15u))
            return fail(MQR_ERR_INVALID_ARG, "out_dev must be 16-byte aligned");
        const unsigned long long cap_elems = cap_bytes / 8;
        mqr_status s = run_tick(c, rects, Q, kEmitAtomic, out_dev, out_dev ? cap_elems : 0, nullptr);
        c->last.n_results = c->last.n_out;
        *out_count = c->last.n_out;
        if (s != MQR_OK) return s;
        if (c->last.n_out > cap_elems || (c->last.n_out && out_dev == nullptr))
            return fail(MQR_ERR_CAPACITY, "output buffer too small for the tick's results");
        return MQR_OK;
    }
    if (kind == MQR_OUT_PAIRS || kind == MQR_OUT_CSR || kind == MQR_OUT_RUNS) {
        if (out_dev && (reinterpret_cast<uintptr_t>(out_dev) & 15u))
            return fail(MQR_ERR_INVALID_ARG, "out_dev must be 16-byte aligned");
        const size_t eb = out_elem_bytes(kind);
        unsigned long long cap_elems = cap_bytes / eb;
        const int ek = kind == MQR_OUT_PAIRS ? kEmitPairs : (kind == MQR_OUT_CSR ? kEmitIds : kEmitRuns);
        mqr_status s = run_tick(c, rects, Q, ek, out_dev, out_dev ? cap_elems : 0, offs);
        *out_count = c->last.n_out;
        if (s != MQR_OK) return s;
        if (c->last.n_out > cap_elems || (c->last.n_out && out_dev == nullptr))
            return fail(MQR_ERR_CAPACITY, "output buffer too small for the tick's results");
        return MQR_OK;
    }
    // sorted kinds: count first, then emit (qidx, id) keys, sort, lay out.
    mqr_status s = run_tick(c, rects, Q, -1, nullptr, 0, offs);
    *out_count = c->last.n_results;
    if (s != MQR_OK) return s;
    const uint64_t R = c->last.n_results;
    const size_t eb = out_elem_bytes(kind);
    if (R > cap_bytes / eb || (R && out_dev == nullptr))
        return fail(MQR_ERR_CAPACITY, "output buffer too small for the tick's results");
    if (R >= (1ull << 30)) return fail(MQR_ERR_INVALID_ARG, "sorted output kinds are limited to R < 2^30");
    if (R == 0) return MQR_OK;
    MQR_CUDA(c->sortA.ensure(R));
    MQR_CUDA(c->sortB.ensure(R));
    Arena a = arena_layout(c->nmax, Q, c->sub_q.n, c->cand_tiles);
    Caps caps{c->sub_q.n, c->isub.n, std::min<size_t>(c->bitmap.n, 0xffffffffull), R, c->cand_tiles,
              c->item_leaf.n};
    Info *info = at<Info>(c, a.info);
    phase_begin(c, MQR_PHASE_OUTPUT_SORT);
    launch_emit(c->stream, c->num_sms * (int)c->bps_emit, kEmitKeys64, c->sub_q.p, c->sub_leaf.p, c->sub_len.p,
                c->leaf_word_off.p, c->out_off.p, c->leaf_beg.p, c->sid.p, c->bitmap.p, c->sortA.p, wpr,
                at<uint32_t>(c, a.counters) + 9, caps, info);
    s = check_launch("emit keys");
    if (s != MQR_OK) return s;
    unsigned long long *sorted = nullptr;
    s = sort_result_keys(c, R, Q, &sorted);
    if (s != MQR_OK) return s;
    launch_keys_to_output(c->stream, sorted, R, kind == MQR_OUT_PAIRS_SORTED, out_dev);
    phase_end(c, MQR_PHASE_OUTPUT_SORT, 0);
    s = check_launch("layout");
    if (s != MQR_OK) return s;
    MQR_CUDA(cudaStreamSynchronize(c->stream));
    phases_collect(c, false);
    return MQR_OK;
}

// The tick itself, then the deferred report of ignored update ids (the tick
// was answered completely, without those updates).
mqr_status tick_device(mqr_ctx *c, const float *rects_dev, uint32_t Q, int kind, void *out_dev,
                       uint64_t cap_bytes, uint64_t *out_count, uint64_t *offsets_dev) {
    mqr_status s = tick_device_impl(c, rects_dev, Q, kind, out_dev, cap_bytes, out_count, offsets_dev);
    if (s == MQR_OK && c->bad_id) {
        c->bad_id = false;
        return fail(MQR_ERR_INVALID_ARG,
                    "an update id was >= max_objects (ignored); the tick was answered without it");
    }
    return s;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *mqr_last_error(void) { return g_err.c_str(); }

struct mqr_cost {
    int device = 0;
    cudaStream_t stream = nullptr;
    DevBuf<float> params, m, v, X, y, out, loss;
    uint32_t steps = 0;
};

uint32_t mqr_cost_param_count(void) { return (uint32_t)cost_param_count(); }

mqr_status mqr_cost_create(mqr_cost **out) {
    if (!out) return fail(MQR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    mqr_cost *m = new (std::nothrow) mqr_cost();
    if (!m) return fail(MQR_ERR_OOM, "host allocation failed");
    const size_t P = cost_param_count();
    cudaError_t e = cudaGetDevice(&m->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = m->params.ensure(P);
    if (e == cudaSuccess) e = m->m.ensure(P);
    if (e == cudaSuccess) e = m->v.ensure(P);
    if (e == cudaSuccess) e = m->loss.ensure(1);
    if (e == cudaSuccess) e = cudaMemset(m->params.p, 0, P * 4);
    if (e == cudaSuccess) e = cudaMemset(m->m.p, 0, P * 4);
    if (e == cudaSuccess) e = cudaMemset(m->v.p, 0, P * 4);
    if (e != cudaSuccess) {
        mqr_cost_destroy(m);
        return cuda_fail(e, "mqr_cost_create");
    }
    *out = m;
    return MQR_OK;
}

mqr_status mqr_cost_set_params(mqr_cost *m, const float *params_host, uint32_t n_params) {
    if (!m || !params_host) return fail(MQR_ERR_INVALID_ARG, "NULL argument");
    if (n_params != cost_param_count()) return fail(MQR_ERR_INVALID_ARG, "wrong parameter count");
    MQR_CUDA(cudaSetDevice(m->device));
    MQR_CUDA(cudaMemcpy(m->params.p, params_host, (size_t)n_params * 4, cudaMemcpyHostToDevice));
    MQR_CUDA(cudaMemset(m->m.p, 0, (size_t)n_params * 4));
    MQR_CUDA(cudaMemset(m->v.p, 0, (size_t)n_params * 4));
    m->steps = 0;
    return MQR_OK;
}

mqr_status mqr_cost_get_params(mqr_cost *m, float *params_host, uint32_t n_params) {
    if (!m || !params_host) return fail(MQR_ERR_INVALID_ARG, "NULL argument");
    if (n_params != cost_param_count()) return fail(MQR_ERR_INVALID_ARG, "wrong parameter count");
    MQR_CUDA(cudaSetDevice(m->device));
    MQR_CUDA(cudaStreamSynchronize(m->stream));
    MQR_CUDA(cudaMemcpy(params_host, m->params.p, (size_t)n_params * 4, cudaMemcpyDeviceToHost));
    return MQR_OK;
}

mqr_status mqr_cost_train(mqr_cost *m, const float *X_host, const float *y_host, uint32_t n, uint32_t epochs,
                          float lr, float *loss_out) {
    if (!m || (n && (!X_host || !y_host))) return fail(MQR_ERR_INVALID_ARG, "NULL argument");
    if (n == 0 || epochs == 0) return MQR_OK;
    if (!(lr > 0.f)) return fail(MQR_ERR_INVALID_ARG, "lr must be > 0");
    MQR_CUDA(cudaSetDevice(m->device));
    MQR_CUDA(m->X.ensure((size_t)n * 5));
    MQR_CUDA(m->y.ensure(n));
    MQR_CUDA(cudaMemcpyAsync(m->X.p, X_host, (size_t)n * 5 * 4, cudaMemcpyHostToDevice, m->stream));
    MQR_CUDA(cudaMemcpyAsync(m->y.p, y_host, (size_t)n * 4, cudaMemcpyHostToDevice, m->stream));
    MQR_CUDA(launch_cost_train(m->stream, m->params.p, m->m.p, m->v.p, m->steps, m->X.p, m->y.p, n, epochs, lr,
                               m->loss.p, nullptr));
    m->steps += epochs;
    float l = 0.f;
    MQR_CUDA(cudaMemcpyAsync(&l, m->loss.p, 4, cudaMemcpyDeviceToHost, m->stream));
    MQR_CUDA(cudaStreamSynchronize(m->stream));
    if (loss_out) *loss_out = l;
    return MQR_OK;
}

mqr_status mqr_cost_gradient(mqr_cost *m, const float *X_host, const float *y_host, uint32_t n, float *grad_host,
                             float *loss_out) {
    if (!m || !grad_host || (n && (!X_host || !y_host))) return fail(MQR_ERR_INVALID_ARG, "NULL argument");
    if (n == 0) return fail(MQR_ERR_INVALID_ARG, "n must be >= 1");
    const size_t P = cost_param_count();
    MQR_CUDA(cudaSetDevice(m->device));
    MQR_CUDA(m->X.ensure((size_t)n * 5));
    MQR_CUDA(m->y.ensure(n));
    MQR_CUDA(m->out.ensure(std::max<size_t>(P, n)));
    MQR_CUDA(cudaMemcpyAsync(m->X.p, X_host, (size_t)n * 5 * 4, cudaMemcpyHostToDevice, m->stream));
    MQR_CUDA(cudaMemcpyAsync(m->y.p, y_host, (size_t)n * 4, cudaMemcpyHostToDevice, m->stream));
    MQR_CUDA(launch_cost_train(m->stream, m->params.p, m->m.p, m->v.p, m->steps, m->X.p, m->y.p, n, 1, 1.f,
                               m->loss.p, m->out.p));
    float l = 0.f;
    MQR_CUDA(cudaMemcpyAsync(grad_host, m->out.p, P * 4, cudaMemcpyDeviceToHost, m->stream));
    MQR_CUDA(cudaMemcpyAsync(&l, m->loss.p, 4, cudaMemcpyDeviceToHost, m->stream));
    MQR_CUDA(cudaStreamSynchronize(m->stream));
    if (loss_out) *loss_out = l;
    return MQR_OK;
}

mqr_status mqr_cost_predict(mqr_cost *m, const float *X_host, uint32_t n, float *out_host) {
    if (!m || (n && (!X_host || !out_host))) return fail(MQR_ERR_INVALID_ARG, "NULL argument");
    if (n == 0) return MQR_OK;
    MQR_CUDA(cudaSetDevice(m->device));
    MQR_CUDA(m->X.ensure((size_t)n * 5));
    MQR_CUDA(m->out.ensure(n));
    MQR_CUDA(cudaMemcpyAsync(m->X.p, X_host, (size_t)n * 5 * 4, cudaMemcpyHostToDevice, m->stream));
    MQR_CUDA(launch_cost_predict(m->stream, m->params.p, m->X.p, n, m->out.p));
    MQR_CUDA(cudaMemcpyAsync(out_host, m->out.p, (size_t)n * 4, cudaMemcpyDeviceToHost, m->stream));
    MQR_CUDA(cudaStreamSynchronize(m->stream));
    return MQR_OK;
}

void mqr_cost_destroy(mqr_cost *m) {
    if (!m) return;
    cudaSetDevice(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    m->params.release(); m->m.release(); m->v.release(); m->X.release(); m->y.release();
    m->out.release(); m->loss.release();
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

mqr_status mqr_set_index(mqr_ctx *c, int index_kind, uint32_t leaf_cap, uint32_t grid_level) {
    if (!c) return fail(MQR_ERR_INVALID_ARG, "ctx is NULL");
    if (index_kind != MQR_INDEX_QUADTREE && index_kind != MQR_INDEX_UNIFORM_GRID)
        return fail(MQR_ERR_INVALID_ARG, "unknown index kind");
    if (index_kind == MQR_INDEX_QUADTREE && leaf_cap == 0) return fail(MQR_ERR_INVALID_ARG, "leaf_cap must be >= 1");
    if (index_kind == MQR_INDEX_UNIFORM_GRID && (grid_level < 1 || grid_level > 15 || grid_level < c->world_bits))
        return fail(MQR_ERR_INVALID_ARG, "grid_level must be in 1..15 (and >= the worlds' levels)");
    MQR_CUDA(cudaSetDevice(c->device));
    MQR_CUDA(cudaStreamSynchronize(c->stream));
    if (index_kind == MQR_INDEX_QUADTREE && leaf_cap > (uint32_t)kLeafCapSmem && leaf_cap < c->nmax) {
        const size_t n = c->nmax;                  // the global window tables of large capacities
        MQR_CUDA(c->mk_a.ensure(2 * n + 2));
        MQR_CUDA(c->mk_b.ensure(2 * n + 2));
    }
    c->cfg.index_kind = index_kind;
    if (index_kind == MQR_INDEX_QUADTREE) c->cfg.leaf_cap = leaf_cap;
    else c->cfg.grid_level = grid_level;
    ++g_buf_gen;                                   // a captured tick holds the old configuration
    return MQR_OK;
}

mqr_status mqr_set_launch_config(mqr_ctx *c, const mqr_launch_config *lc) {
    if (!c || !lc) return fail(MQR_ERR_INVALID_ARG, "NULL argument");
    const uint32_t v[4] = {lc->candidate_blocks_per_sm, lc->compact_blocks_per_sm, lc->filter_blocks_per_sm,
                           lc->emit_blocks_per_sm};
    for (uint32_t x : v)
        if (x > 64) return fail(MQR_ERR_INVALID_ARG, "blocks per SM must be 0 (default) .. 64");
    MQR_CUDA(cudaSetDevice(c->device));
    MQR_CUDA(cudaStreamSynchronize(c->stream));
    auto pick = [](uint32_t x) { return x ? x : (uint32_t)kDefaultBlocksPerSM; };
    c->bps_cand = pick(v[0]);
    c->bps_compact = pick(v[1]);
    c->bps_filter = pick(v[2]);
    c->bps_emit = pick(v[3]);
    ++g_buf_gen;                                   // a captured tick holds the old launch shapes
    return MQR_OK;
}

mqr_status mqr_set_region_caps(mqr_ctx *c, uint32_t region_bits, const uint32_t *caps_host) {
    if (!c) return fail(MQR_ERR_INVALID_ARG, "ctx is NULL");
    if (region_bits > kMaxRegionBits) return fail(MQR_ERR_INVALID_ARG, "region_bits must be 0..4");
    const size_t n = (size_t)1 << (2 * region_bits);
    if (region_bits) {
        if (!caps_host) return fail(MQR_ERR_INVALID_ARG, "caps_host is NULL");
        for (size_t r = 0; r < n; ++r)
            if (caps_host[r] < 1 || caps_host[r] > (uint32_t)kLeafCapSmem)
                return fail(MQR_ERR_INVALID_ARG, "region capacities must be in 1..16384");
    }
    if (!region_bits && !c->region_bits) return MQR_OK;     // nothing changes
    MQR_CUDA(cudaSetDevice(c->device));
    MQR_CUDA(cudaStreamSynchronize(c->stream));
    if (region_bits) {
        MQR_CUDA(c->region_cap.ensure(n));
        MQR_CUDA(cudaMemcpy(c->region_cap.p, caps_host, n * sizeof(uint32_t), cudaMemcpyHostToDevice));
    }
    c->region_bits = region_bits;
    ++g_buf_gen;                                   // a captured tick holds the old configuration
    return MQR_OK;
}

mqr_status mqr_config_default(mqr_config *cfg) {
    if (!cfg) return fail(MQR_ERR_INVALID_ARG, "cfg is NULL");
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->max_objects = 1u << 20;
    cfg->leaf_cap = 128;
    cfg->index_kind = MQR_INDEX_QUADTREE;
    cfg->grid_level = 8;
    cfg->covering = 1;
    return MQR_OK;
}

void mqr_destroy(mqr_ctx *c) {
    if (!c) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->parent) {                       // a slot leaves its context's list
        auto &v = c->parent->slots;
        v.erase(std::remove(v.begin(), v.end(), c), v.end());
    }
    for (mqr_ctx *sl : c->slots) {         // slots outliving their context become unusable
        if (sl->stream) cudaStreamSynchronize(sl->stream);
        sl->parent = nullptr;
    }
    c->slots.clear();
    if (c->slot_done) cudaEventDestroy(c->slot_done);
    if (c->snap_ready) cudaEventDestroy(c->snap_ready);
    c->snap_info.release();
    DevBuf<float2> *f2[] = {&c->pos, &c->sxy, &c->up_xy};
    for (auto *b : f2) b->release();
    free_graphs(c);
    c->world_obj.release();
    c->world_q.release();
    c->region_cap.release();
    c->region_cnt.release();
    c->region_stats.release();
    c->state_flags.release();
    DevBuf<unsigned long long> *u64s[] = {&c->stamp, &c->keysA, &c->keysB, &c->out_off, &c->off_stage,
                                          &c->sortA, &c->sortB};
    for (auto *b : u64s) b->release();
    DevBuf<uint32_t> *u32s[] = {&c->skey, &c->sid, &c->sort_counts, &c->sort_offs, &c->leaf_lo, &c->leaf_hi, &c->leaf_beg, &c->leaf_nsub,
                                &c->leaf_sub_off, &c->leaf_word_off, &c->leaf_item_off,
                                &c->sub_q, &c->sub_leaf, &c->sub_len, &c->sub_res,
                                &c->isub, &c->bitmap, &c->item_leaf, &c->up_ids, &c->zmap, &c->pair_q,
                                &c->pair_first, &c->pair_blo, &c->pair_rec, &c->qpair, &c->tile_p0};
    for (auto *b : u32s) b->release();
    c->qcells.release();
    c->leaf_box.release();
    c->cand_off.release();
    c->pair_off.release();
    c->mk_a.release();
    c->mk_b.release();
    c->arena.release();
    c->sort_arena.release();
    c->upd_err.release();
    c->q_rects.release();
    for (int b = 0; b < 2; ++b)
        if (c->copy_done[b]) { cudaEventSynchronize(c->copy_done[b]); cudaEventDestroy(c->copy_done[b]); }
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->snap_done) cudaEventDestroy(c->snap_done);
    c->sid_stage.release();
    c->sid_stage2.release();
    c->out_stage.release();
    c->out_stage2.release();
    c->off_stage2.release();
    for (int p = 0; p < MQR_NUM_PHASES; ++p)
        for (int k = 0; k < 2; ++k)
            if (c->ev[p][k]) cudaEventDestroy(c->ev[p][k]);
    for (int p = 0; p < mqr_ctx::kMaxPendingUpdates; ++p)
        for (int k = 0; k < 2; ++k)
            if (c->up_ev[p][k]) cudaEventDestroy(c->up_ev[p][k]);
    if (c->info_host) cudaFreeHost(c->info_host);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    cudaSetDevice(prev);
    delete c;
}

mqr_status mqr_create_ex(mqr_rect bounds, const mqr_config *cfg, void *cuda_stream, mqr_ctx **out) {
    if (!out) return fail(MQR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(MQR_ERR_INVALID_ARG, "cfg is NULL");
    if (!finite_rect(bounds)) return fail(MQR_ERR_INVALID_ARG, "bounds must be finite with xmax > xmin, ymax > ymin");
    if (cfg->leaf_cap == 0) return fail(MQR_ERR_INVALID_ARG, "leaf_cap must be >= 1");
    if (cfg->index_kind != MQR_INDEX_QUADTREE && cfg->index_kind != MQR_INDEX_UNIFORM_GRID)
        return fail(MQR_ERR_INVALID_ARG, "unknown index_kind");
    if (cfg->index_kind == MQR_INDEX_UNIFORM_GRID && (cfg->grid_level < 1 || cfg->grid_level > 15))
        return fail(MQR_ERR_INVALID_ARG, "grid_level must be in 1..15");
    if (cfg->max_objects >= (1u << 30)) return fail(MQR_ERR_INVALID_ARG, "max_objects must be < 2^30");
    if (cfg->reserved[0] || cfg->reserved[1] || cfg->reserved[2])
        return fail(MQR_ERR_INVALID_ARG, "reserved fields must be 0");
    float sx = fp32_scale(bounds.xmin, bounds.xmax), sy = fp32_scale(bounds.ymin, bounds.ymax);
    if (!std::isfinite(sx) || !std::isfinite(sy) || !(sx > 0.f) || !(sy > 0.f))
        return fail(MQR_ERR_INVALID_ARG, "bounds too small for float32 cell scaling");

    mqr_ctx *c = new (std::nothrow) mqr_ctx();
    if (!c) return fail(MQR_ERR_OOM, "host allocation failed");
    c->cfg = *cfg;
    c->bounds = bounds;
    c->sx = sx;
    c->sy = sy;
    c->nmax = cfg->max_objects;
    auto bail = [&](cudaError_t e, const char *what) {
        mqr_status s = cuda_fail(e, what);
        mqr_destroy(c);
        return s;
    };
    cudaError_t e;
    if ((e = cudaGetDevice(&c->device)) != cudaSuccess) return bail(e, "cudaGetDevice");
    if ((e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device)) != cudaSuccess)
        return bail(e, "cudaDeviceGetAttribute");
    if (cuda_stream) {
        c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    } else {
        if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess)
            return bail(e, "cudaStreamCreate");
        c->own_stream = true;
    }
    const size_t n = std::max<size_t>(c->nmax, 1);
    if ((e = c->pos.ensure(n)) || (e = c->stamp.ensure(n)) || (e = c->keysA.ensure(n)) ||
        (e = c->keysB.ensure(n)) || (e = c->skey.ensure(n)) || (e = c->sid.ensure(n)) ||
        (e = c->sxy.ensure(n)) || (e = c->leaf_lo.ensure(n)) || (e = c->leaf_hi.ensure(n)) ||
        (e = c->leaf_beg.ensure(n + 1)) || (e = c->leaf_nsub.ensure(n)) ||
        (e = c->leaf_sub_off.ensure(n + 1)) || (e = c->leaf_word_off.ensure(n + 1)) ||
        (e = c->leaf_item_off.ensure(n + 1)) ||
        (e = c->sort_counts.ensure((size_t)256 * ((n + kSortTile - 1) / kSortTile))) ||
        (e = c->sort_offs.ensure((size_t)256 * ((n + kSortTile - 1) / kSortTile))) ||
        (e = c->upd_err.ensure(1)) || (e = c->leaf_box.ensure(n)))
        return bail(e, "cudaMalloc (object state)");
    if (cfg->index_kind == MQR_INDEX_QUADTREE && cfg->leaf_cap > (uint32_t)kLeafCapSmem &&
        cfg->leaf_cap < c->nmax) {
        if ((e = c->mk_a.ensure(2 * n + 2)) || (e = c->mk_b.ensure(2 * n + 2)))
            return bail(e, "cudaMalloc (window tables)");
    }
    if ((e = cudaMemsetAsync(c->stamp.p, 0, n * sizeof(unsigned long long), c->stream)) ||
        (e = cudaMemsetAsync(c->pos.p, 0, n * sizeof(float2), c->stream)) ||
        (e = cudaMemsetAsync(c->upd_err.p, 0, sizeof(unsigned long long), c->stream)))
        return bail(e, "cudaMemset");
    if ((e = cudaMallocHost(&c->info_host, sizeof(Info))) != cudaSuccess) return bail(e, "cudaMallocHost");
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return bail(e, "cudaStreamSynchronize");
    *out = c;
    return MQR_OK;
}

mqr_status mqr_create(mqr_rect bounds, uint32_t leaf_cap, uint32_t max_objects, mqr_ctx **out) {
    mqr_config cfg;
    mqr_config_default(&cfg);
    cfg.leaf_cap = leaf_cap;
    cfg.max_objects = max_objects;
    return mqr_create_ex(bounds, &cfg, nullptr, out);
}

mqr_status mqr_apply_updates(mqr_ctx *c, const uint32_t *ids_dev, const float *xy_dev, uint32_t n) {
    if (!c) return fail(MQR_ERR_INVALID_ARG, "ctx is NULL");
    if (n == 0) return MQR_OK;
    if (!ids_dev || !xy_dev) return fail(MQR_ERR_INVALID_ARG, "ids_dev / xy_dev is NULL");
    if ((reinterpret_cast<uintptr_t>(xy_dev) & 7u) || (reinterpret_cast<uintptr_t>(ids_dev) & 3u))
        return fail(MQR_ERR_INVALID_ARG, "xy_dev must be 8-byte and ids_dev 4-byte aligned");
    MQR_CUDA(cudaSetDevice(c->device));
    ++c->epoch;
    const bool timed = c->timing && (c->timing_mask & (1u << MQR_PHASE_UPDATES)) &&
                       c->up_pending < mqr_ctx::kMaxPendingUpdates;
    if (timed) cudaEventRecord(c->up_ev[c->up_pending][0], c->stream);
    launch_apply_updates(c->stream, ids_dev, reinterpret_cast<const float2 *>(xy_dev), n, c->nmax,
                         c->epoch, c->stamp.p, c->pos.p, c->upd_err.p);
    if (timed) {
        cudaEventRecord(c->up_ev[c->up_pending][1], c->stream);
        ++c->up_pending;
    }
    if (c->timing) c->up_launches += 2;
    return check_launch("apply_updates");
}

mqr_status mqr_apply_updates_host(mqr_ctx *c, const uint32_t *ids_host, const float *xy_host, uint32_t n) {
    if (!c) return fail(MQR_ERR_INVALID_ARG, "ctx is NULL");
    if (n == 0) return MQR_OK;
    if (!ids_host || !xy_host) return fail(MQR_ERR_INVALID_ARG, "ids_host / xy_host is NULL");
    MQR_CUDA(cudaSetDevice(c->device));
    MQR_CUDA(c->up_ids.ensure(n));
    MQR_CUDA(c->up_xy.ensure(n));
    MQR_CUDA(cudaMemcpyAsync(c->up_ids.p, ids_host, (size_t)n * 4, cudaMemcpyHostToDevice, c->stream));
    MQR_CUDA(cudaMemcpyAsync(c->up_xy.p, xy_host, (size_t)n * 8, cudaMemcpyHostToDevice, c->stream));
    mqr_status s = mqr_apply_updates(c, c->up_ids.p, reinterpret_cast<const float *>(c->up_xy.p), n);
    if (s != MQR_OK) return s;
    // the host buffers may be reused as soon as we return
    MQR_CUDA(cudaStreamSynchronize(c->stream));
    return MQR_OK;
}

static bool slots_busy(const mqr_ctx *c) {
    for (const mqr_ctx *sl : c->slots)
        if (sl->slot_busy) return true;
    return false;
}

static mqr_status tick_args(mqr_ctx *c, const void *rects, uint32_t Q, int kind, uint64_t *out_count) {
    if (!c) return fail(MQR_ERR_INVALID_ARG, "ctx is NULL");
    if (c->parent) return fail(MQR_ERR_INVALID_ARG, "a slot answers through mqr_slot_begin / mqr_slot_end");
    if (slots_busy(c)) return fail(MQR_ERR_INVALID_ARG, "a slot of this context has a join pending (mqr_slot_end)");
    if (!out_count) return fail(MQR_ERR_INVALID_ARG, "out_count is NULL");
    if (Q > 0 && !rects) return fail(MQR_ERR_INVALID_ARG, "rects is NULL");
    if (Q >= (1u << 30)) return fail(MQR_ERR_INVALID_ARG, "Q must be < 2^30");
    if (kind < MQR_OUT_PAIRS || kind > MQR_OUT_PAIRS_ATOMIC) return fail(MQR_ERR_INVALID_ARG, "unknown output kind");
    if (c->n_worlds && (!c->world_q_set || Q != c->world_q_total))
        return fail(MQR_ERR_INVALID_ARG, "batched worlds: Q must equal the total of mqr_set_query_worlds");
    return MQR_OK;
}

mqr_status mqr_set_graph(mqr_ctx *c, int enable) {
    if (!c) return fail(MQR_ERR_INVALID_ARG, "ctx is NULL");
    MQR_CUDA(cudaSetDevice(c->device));
    MQR_CUDA(cudaStreamSynchronize(c->stream));
    c->graph_on = enable != 0;
    if (!c->graph_on) free_graphs(c);
    return MQR_OK;
}

mqr_status mqr_set_worlds(mqr_ctx *c, uint32_t n_worlds, const uint32_t *obj_base_host) {
    if (!c) return fail(MQR_ERR_INVALID_ARG, "ctx is NULL");
    if (n_worlds == 0 || n_worlds > kMaxWorlds) return fail(MQR_ERR_INVALID_ARG, "n_worlds must be 1..16384");
    if (n_worlds > 1 && !obj_base_host) return fail(MQR_ERR_INVALID_ARG, "obj_base_host is NULL");
    MQR_CUDA(cudaSetDevice(c->device));
    MQR_CUDA(cudaStreamSynchronize(c->stream));
    c->world_q_set = false;
    if (n_worlds == 1) {                        // one world: the plain index
        c->n_worlds = c->world_bits = 0;
        return MQR_OK;
    }
    if (obj_base_host[0] != 0 || obj_base_host[n_worlds] != c->nmax)
        return fail(MQR_ERR_INVALID_ARG, "obj_base must start at 0 and end at max_objects");
    for (uint32_t w = 0; w < n_worlds; ++w)
        if (obj_base_host[w + 1] < obj_base_host[w]) return fail(MQR_ERR_INVALID_ARG, "obj_base must not decrease");
    uint32_t bits = 0;
    while ((1u << (2 * bits)) < n_worlds) ++bits;
    if (c->cfg.index_kind == MQR_INDEX_UNIFORM_GRID && c->cfg.grid_level < bits)
        return fail(MQR_ERR_INVALID_ARG, "uniform grid: grid_level must be >= log4(n_worlds)");
    MQR_CUDA(c->world_obj.ensure((size_t)n_worlds + 1));
    MQR_CUDA(c->world_q.ensure((size_t)n_worlds + 1));
    MQR_CUDA(cudaMemcpy(c->world_obj.p, obj_base_host, ((size_t)n_worlds + 1) * 4, cudaMemcpyHostToDevice));
    c->n_worlds = n_worlds;
    c->world_bits = bits;
    return MQR_OK;
}

mqr_status mqr_set_query_worlds(mqr_ctx *c, const uint32_t *q_base_host) {
    if (!c) return fail(MQR_ERR_INVALID_ARG, "ctx is NULL");
    if (!c->n_worlds) return fail(MQR_ERR_INVALID_ARG, "no batched worlds (mqr_set_worlds)");
    if (!q_base_host) return fail(MQR_ERR_INVALID_ARG, "q_base_host is NULL");
    if (q_base_host[0] != 0) return fail(MQR_ERR_INVALID_ARG, "q_base must start at 0");
    for (uint32_t w = 0; w < c->n_worlds; ++w)
        if (q_base_host[w + 1] < q_base_host[w]) return fail(MQR_ERR_INVALID_ARG, "q_base must not decrease");
    MQR_CUDA(cudaSetDevice(c->device));
    MQR_CUDA(cudaStreamSynchronize(c->stream));
    MQR_CUDA(cudaMemcpy(c->world_q.p, q_base_host, ((size_t)c->n_worlds + 1) * 4, cudaMemcpyHostToDevice));
    c->world_q_total = q_base_host[c->n_worlds];
    c->world_q_set = true;
    return MQR_OK;
}

mqr_status mqr_tick(mqr_ctx *c, const float *rects_dev, uint32_t Q, int kind, void *out_dev,
                    uint64_t out_capacity_bytes, uint64_t *out_count, uint64_t *offsets_dev) {
    mqr_status s = tick_args(c, rects_dev, Q, kind, out_count);
    if (s != MQR_OK) return s;
    if ((kind == MQR_OUT_CSR || kind == MQR_OUT_CSR_SORTED) && !offsets_dev)
        return fail(MQR_ERR_INVALID_ARG, "CSR output needs offsets_dev");
    *out_count = 0;
    MQR_CUDA(cudaSetDevice(c->device));
    return tick_device(c, rects_dev, Q, kind, out_dev, out_capacity_bytes, out_count, offsets_dev);
}

// Wait for the host copies started by mqr_tick_host_async.
static mqr_status host_copies_wait(mqr_ctx *c) {
    for (int b = 0; b < 2; ++b)
        if (c->copy_pending[b]) {
            MQR_CUDA(cudaEventSynchronize(c->copy_done[b]));
            c->copy_pending[b] = false;
        }
    return MQR_OK;
}

// The host-buffer tick: inputs staged to the device, the tick into a device
// staging buffer, the result copied back -- on the context's stream (sync) or
// on a second stream left running (async, staging buffers alternating).
static mqr_status tick_host_impl(mqr_ctx *c, const float *rects_host, uint32_t Q, int kind, void *out_host,
                                 uint64_t out_capacity_bytes, uint64_t *out_count, uint64_t *offsets_host,
                                 bool async) {
    mqr_status s = tick_args(c, rects_host, Q, kind, out_count);
    if (s != MQR_OK) return s;
    if ((kind == MQR_OUT_CSR || kind == MQR_OUT_CSR_SORTED) && !offsets_host)
        return fail(MQR_ERR_INVALID_ARG, "CSR output needs offsets_host");
    *out_count = 0;
    MQR_CUDA(cudaSetDevice(c->device));
    int b = 0;
    if (async) {
        if (!c->copy_stream) {
            MQR_CUDA(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
            for (int k = 0; k < 2; ++k) MQR_CUDA(cudaEventCreateWithFlags(&c->copy_done[k], cudaEventDisableTiming));
        }
        b = c->next_stage;
        if (c->copy_pending[b]) {                          // the copy that last read this staging buffer
            MQR_CUDA(cudaEventSynchronize(c->copy_done[b]));
            c->copy_pending[b] = false;
        }
    } else {
        s = host_copies_wait(c);
        if (s != MQR_OK) return s;
    }
    DevBuf<unsigned char> &stage = b ? c->out_stage2 : c->out_stage;
    DevBuf<unsigned long long> &ostage = b ? c->off_stage2 : c->off_stage;
    MQR_CUDA(c->q_rects.ensure(std::max<size_t>(Q, 1)));
    if (Q) MQR_CUDA(cudaMemcpyAsync(c->q_rects.p, rects_host, (size_t)Q * 16, cudaMemcpyHostToDevice, c->stream));
    uint64_t *offs_dev = nullptr;
    if (offsets_host) {
        MQR_CUDA(ostage.ensure((size_t)Q + 1));
        offs_dev = reinterpret_cast<uint64_t *>(ostage.p);
    }
    const float *rd = reinterpret_cast<const float *>(c->q_rects.p);
    // Device staging buffer: as large as the caller's buffer allows, grown on
    // demand to the size needed plus a quarter (at most the caller's buffer),
    // so that ticks of slowly growing output do not grow it every time; the
    // tick is then answered again.
    size_t want = out_capacity_bytes;
    if (kind == MQR_OUT_BITMAP) want = std::min<uint64_t>(want, (uint64_t)Q * bitmap_words_per_row(c->nmax) * 4);
    if (kind == MQR_OUT_COUNT) want = 0;
    size_t have = std::min(stage.n, want);
    s = tick_device(c, rd, Q, kind, have ? stage.p : nullptr, have, out_count, offs_dev);
    if (s == MQR_ERR_CAPACITY && kind != MQR_OUT_COUNT) {
        uint64_t need = kind == MQR_OUT_BITMAP ? *out_count * 4 : *out_count * out_elem_bytes(kind);
        if (need > out_capacity_bytes) return s;
        const size_t grow = std::min<uint64_t>(need + need / 4, want);
        MQR_CUDA(stage.ensure(std::max<size_t>(std::max<size_t>(grow, need), 1)));
        s = tick_device(c, rd, Q, kind, stage.p, std::min<size_t>(stage.n, want), out_count, offs_dev);
    }
    if (s != MQR_OK) return s;
    uint64_t bytes = kind == MQR_OUT_BITMAP ? *out_count * 4
                     : (kind == MQR_OUT_COUNT ? 0 : *out_count * out_elem_bytes(kind));
    if (bytes && !out_host) return fail(MQR_ERR_INVALID_ARG, "out_host is NULL");
    cudaStream_t cs = async ? c->copy_stream : c->stream;   // the tick's kernels have completed
    if (bytes) MQR_CUDA(cudaMemcpyAsync(out_host, stage.p, bytes, cudaMemcpyDeviceToHost, cs));
    if (offsets_host)
        MQR_CUDA(cudaMemcpyAsync(offsets_host, offs_dev, ((size_t)Q + 1) * 8, cudaMemcpyDeviceToHost, cs));
    if (async) {
        MQR_CUDA(cudaEventRecord(c->copy_done[b], cs));
        c->copy_pending[b] = true;
        c->next_stage = b ^ 1;
    } else {
        MQR_CUDA(cudaStreamSynchronize(c->stream));
    }
    return MQR_OK;
}

mqr_status mqr_tick_host(mqr_ctx *c, const float *rects_host, uint32_t Q, int kind, void *out_host,
                         uint64_t out_capacity_bytes, uint64_t *out_count, uint64_t *offsets_host) {
    return tick_host_impl(c, rects_host, Q, kind, out_host, out_capacity_bytes, out_count, offsets_host, false);
}

mqr_status mqr_tick_host_async(mqr_ctx *c, const float *rects_host, uint32_t Q, int kind, void *out_host,
                               uint64_t out_capacity_bytes, uint64_t *out_count, uint64_t *offsets_host) {
    return tick_host_impl(c, rects_host, Q, kind, out_host, out_capacity_bytes, out_count, offsets_host, true);
}

mqr_status mqr_host_wait(mqr_ctx *c) {
    if (!c) return fail(MQR_ERR_INVALID_ARG, "ctx is NULL");
    MQR_CUDA(cudaSetDevice(c->device));
    return host_copies_wait(c);
}

mqr_status mqr_tick_admit(mqr_ctx *c, const float *rects_dev, uint32_t Q, int kind, void *out_dev,
                          uint64_t out_capacity_bytes, uint32_t *admitted, uint64_t *out_count,
                          uint64_t *offsets_dev) {
    mqr_status s = tick_args(c, rects_dev, Q, kind, out_count);
    if (s != MQR_OK) return s;
    if (!admitted) return fail(MQR_ERR_INVALID_ARG, "admitted is NULL");
    if (kind != MQR_OUT_PAIRS && kind != MQR_OUT_CSR && kind != MQR_OUT_RUNS)
        return fail(MQR_ERR_INVALID_ARG, "admission supports the PAIRS, CSR and RUNS kinds");
    if (out_dev && (reinterpret_cast<uintptr_t>(out_dev) & 15u))
        return fail(MQR_ERR_INVALID_ARG, "out_dev must be 16-byte aligned");
    *out_count = 0;
    *admitted = 0;
    MQR_CUDA(cudaSetDevice(c->device));
    const float4 *rects = reinterpret_cast<const float4 *>(rects_dev);
    unsigned long long *offs = reinterpret_cast<unsigned long long *>(offsets_dev);
    if (!offs) {
        MQR_CUDA(c->off_stage.ensure((size_t)Q + 1));
        offs = c->off_stage.p;
    }
    const int ek = kind == MQR_OUT_PAIRS ? kEmitPairs : (kind == MQR_OUT_CSR ? kEmitIds : kEmitRuns);
    // one pass: exact counts and per-query offsets, the longest prefix of
    // queries whose output fits (on the device), the emit of that prefix
    const unsigned long long cap_elems = out_dev ? out_capacity_bytes / out_elem_bytes(kind) : 0;
    s = run_tick(c, rects, Q, ek, out_dev, cap_elems, offs, true);
    if (s != MQR_OK) return s;
    admission_counts(c->last, Q, admitted, out_count);
    return MQR_OK;
}

mqr_status mqr_snapshot(mqr_ctx *c) {
    if (!c) return fail(MQR_ERR_INVALID_ARG, "ctx is NULL");
    if (c->parent) return fail(MQR_ERR_INVALID_ARG, "a slot has no index of its own");
    if (c->slots.empty()) return fail(MQR_ERR_INVALID_ARG, "no slot of this context (mqr_slot_create)");
    if (slots_busy(c)) return fail(MQR_ERR_INVALID_ARG, "a slot of this context has a join pending (mqr_slot_end)");
    MQR_CUDA(cudaSetDevice(c->device));
    Arena a = arena_layout(c->nmax, 0, c->sub_q.n, c->cand_tiles);
    MQR_CUDA(c->arena.ensure(a.total));
    mqr_status s = enqueue_index(c, a);
    if (s != MQR_OK) return s;
    c->have_snapshot = true;
    c->snap_pending = true;
    return MQR_OK;
}

mqr_status mqr_slot_create(mqr_ctx *c, void *cuda_stream, mqr_slot **out) {
    if (!c || !out) return fail(MQR_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (c->parent) return fail(MQR_ERR_INVALID_ARG, "a slot cannot have slots");
    MQR_CUDA(cudaSetDevice(c->device));
    MQR_CUDA(cudaStreamSynchronize(c->stream));
    if (!c->snap_ready) {
        MQR_CUDA(cudaEventCreateWithFlags(&c->snap_ready, cudaEventDisableTiming));
        MQR_CUDA(c->snap_info.ensure(4));
    }
    mqr_ctx *sl = new (std::nothrow) mqr_ctx();
    if (!sl) return fail(MQR_ERR_OOM, "host allocation failed");
    sl->parent = c;
    sl->device = c->device;
    sl->num_sms = c->num_sms;
    sl->cfg = c->cfg;
    sl->bounds = c->bounds;
    sl->sx = c->sx;
    sl->sy = c->sy;
    sl->nmax = c->nmax;
    c->slots.push_back(sl);                       // from here on mqr_destroy(sl) cleans up
    auto bail = [&](cudaError_t e, const char *what) {
        mqr_status st = cuda_fail(e, what);
        mqr_destroy(sl);
        return st;
    };
    cudaError_t e;
    if (cuda_stream) {
        sl->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    } else {
        if ((e = cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking)) != cudaSuccess)
            return bail(e, "cudaStreamCreate");
        sl->own_stream = true;
    }
    if ((e = cudaEventCreateWithFlags(&sl->slot_done, cudaEventDisableTiming)) != cudaSuccess)
        return bail(e, "cudaEventCreate");
    const size_t n = std::max<size_t>(c->nmax, 1);
    if ((e = sl->leaf_nsub.ensure(n)) || (e = sl->leaf_sub_off.ensure(n + 1)) || (e = sl->leaf_word_off.ensure(n + 1)) ||
        (e = sl->leaf_item_off.ensure(n + 1)))
        return bail(e, "cudaMalloc (slot leaf lists)");
    if ((e = cudaMallocHost(&sl->info_host, sizeof(Info))) != cudaSuccess) return bail(e, "cudaMallocHost");
    *out = reinterpret_cast<mqr_slot *>(sl);
    return MQR_OK;
}

void mqr_slot_destroy(mqr_slot *slot) { mqr_destroy(reinterpret_cast<mqr_ctx *>(slot)); }

mqr_status mqr_slot_begin(mqr_slot *slot, const float *rects_dev, uint32_t Q, int kind, void *out_dev,
                          uint64_t out_capacity_bytes, uint64_t *offsets_dev) {
    mqr_ctx *sl = reinterpret_cast<mqr_ctx *>(slot);
    if (!sl) return fail(MQR_ERR_INVALID_ARG, "slot is NULL");
    mqr_ctx *c = sl->parent;
    if (!c) return fail(MQR_ERR_INVALID_ARG, "the slot's context was destroyed");
    if (sl->slot_busy) return fail(MQR_ERR_INVALID_ARG, "the slot has a join pending (mqr_slot_end)");
    if (!c->have_snapshot) return fail(MQR_ERR_INVALID_ARG, "no snapshot of the context yet (mqr_snapshot)");
    if (Q > 0 && !rects_dev) return fail(MQR_ERR_INVALID_ARG, "rects_dev is NULL");
    if (Q >= (1u << 30)) return fail(MQR_ERR_INVALID_ARG, "Q must be < 2^30");
    if (kind != MQR_OUT_PAIRS && kind != MQR_OUT_CSR && kind != MQR_OUT_RUNS)
        return fail(MQR_ERR_INVALID_ARG, "slots support the PAIRS, CSR and RUNS kinds");
    if (c->n_worlds) return fail(MQR_ERR_INVALID_ARG, "slots are not available with batched worlds");
    if (out_dev && (reinterpret_cast<uintptr_t>(out_dev) & 15u))
        return fail(MQR_ERR_INVALID_ARG, "out_dev must be 16-byte aligned");
    if (offsets_dev && (reinterpret_cast<uintptr_t>(offsets_dev) & 7u))
        return fail(MQR_ERR_INVALID_ARG, "offsets_dev must be 8-byte aligned");
    MQR_CUDA(cudaSetDevice(sl->device));
    // the join follows its context's current configuration
    sl->cfg = c->cfg;
    sl->bps_cand = c->bps_cand;
    sl->bps_compact = c->bps_compact;
    sl->bps_filter = c->bps_filter;
    sl->bps_emit = c->bps_emit;
    unsigned long long *offs = reinterpret_cast<unsigned long long *>(offsets_dev);
    if (!offs) {
        MQR_CUDA(sl->off_stage.ensure((size_t)Q + 1));
        offs = sl->off_stage.p;
    }
    mqr_status s = ensure_tick_buffers(sl, Q);
    if (s != MQR_OK) return s;
    const int ek = kind == MQR_OUT_PAIRS ? kEmitPairs : (kind == MQR_OUT_CSR ? kEmitIds : kEmitRuns);
    const unsigned long long cap_elems = out_dev ? out_capacity_bytes / out_elem_bytes(kind) : 0;
    const float4 *rects = reinterpret_cast<const float4 *>(rects_dev);
    sl->retries = 0;
    Caps caps{};
    s = attempt_enqueue(sl, rects, Q, ek, out_dev, cap_elems, offs, true, caps);
    if (s != MQR_OK) return s;
    MQR_CUDA(cudaEventRecord(sl->slot_done, sl->stream));
    sl->job = mqr_ctx::SlotJob{rects, Q, ek, kind, out_dev, cap_elems, offs, caps};
    sl->slot_busy = true;
    return MQR_OK;
}

mqr_status mqr_slot_end(mqr_slot *slot, uint32_t *admitted, uint64_t *out_count) {
    mqr_ctx *sl = reinterpret_cast<mqr_ctx *>(slot);
    if (!sl || !admitted || !out_count) return fail(MQR_ERR_INVALID_ARG, "NULL argument");
    if (!sl->slot_busy) return fail(MQR_ERR_INVALID_ARG, "no join pending on the slot (mqr_slot_begin)");
    *admitted = 0;
    *out_count = 0;
    MQR_CUDA(cudaSetDevice(sl->device));
    mqr_ctx::SlotJob &j = sl->job;
    mqr_status s = MQR_OK;
    bool done = false;
    for (int attempt = 0; attempt < 8 && s == MQR_OK && !done; ++attempt) {
        if (attempt > 0) {                       // an internal buffer grew: answer again
            s = attempt_enqueue(sl, j.rects, j.Q, j.emit_kind, j.out, j.cap, j.offsets, true, j.caps);
            if (s != MQR_OK) break;
            ++sl->retries;
        }
        cudaError_t e = cudaStreamSynchronize(sl->stream);
        if (e != cudaSuccess) { s = cuda_fail(e, "cudaStreamSynchronize"); break; }
        bool again = false;
        s = attempt_check(sl, j.Q, j.emit_kind, j.caps, &again);
        done = !again;
    }
    if (s == MQR_OK && !done) s = fail(MQR_ERR_INTERNAL, "buffer growth did not converge");
    if (s == MQR_OK && (cudaEventRecord(sl->slot_done, sl->stream) != cudaSuccess))
        s = fail(MQR_ERR_CUDA, "cudaEventRecord");
    sl->slot_busy = false;
    if (s != MQR_OK) return s;
    admission_counts(sl->last, j.Q, admitted, out_count);
    if (sl->bad_id) {
        sl->bad_id = false;
        return fail(MQR_ERR_INVALID_ARG, "an update id was >= max_objects (ignored); the join was answered without it");
    }
    return MQR_OK;
}

mqr_status mqr_slot_get_stats(const mqr_slot *slot, mqr_stats *out) {
    if (!slot) return fail(MQR_ERR_INVALID_ARG, "slot is NULL");
    return mqr_get_stats(reinterpret_cast<const mqr_ctx *>(slot), out);
}

mqr_status mqr_get_stats(const mqr_ctx *c, mqr_stats *o) {
    if (!c || !o) return fail(MQR_ERR_INVALID_ARG, "NULL argument");
    const Info &in = c->last;
    std::memset(o, 0, sizeof(*o));
    o->n_objects = in.n_present;
    o->n_queries = c->last_q;
    o->n_leaves = in.n_leaves;
    o->max_level = in.max_level;
    o->n_sub_intersecting = in.n_sub_i;
    o->n_sub_covering = in.n_sub_c;
    o->n_covering_runs = in.n_sub - in.n_sub_i;
    o->n_tests = in.n_tests;
    o->n_filter_items = in.n_items;
    o->n_bitmap_words = in.n_words;
    o->n_results = in.n_results;
    o->n_results_covering = in.n_results_cov;
    o->n_retries = c->retries;
    o->n_filter_loads = in.n_item_objs;
    o->n_pairs = in.n_pairs;
    o->n_candidates = in.n_cand;
    return MQR_OK;
}

mqr_status mqr_region_counts(mqr_ctx *c, uint32_t region_bits, uint32_t *counts_host) {
    if (!c || !counts_host) return fail(MQR_ERR_INVALID_ARG, "NULL argument");
    if (region_bits < 1 || region_bits > kMaxRegionBits) return fail(MQR_ERR_INVALID_ARG, "region_bits must be 1..4");
    {
        mqr_status si = index_ready(c);
        if (si != MQR_OK) return si;
    }
    const size_t R = (size_t)1 << (2 * region_bits);
    MQR_CUDA(cudaSetDevice(c->device));
    MQR_CUDA(c->region_cnt.ensure(R));
    MQR_CUDA(launch_region_counts(c->stream, c->skey.p, (uint32_t)c->last.n_present, region_bits,
                                  c->region_cnt.p));
    MQR_CUDA(cudaMemcpyAsync(counts_host, c->region_cnt.p, R * 4, cudaMemcpyDeviceToHost, c->stream));
    MQR_CUDA(cudaStreamSynchronize(c->stream));
    return MQR_OK;
}

mqr_status mqr_region_work(mqr_ctx *c, const float *rects_dev, uint32_t Q, uint32_t region_bits, double *out_host) {
    if (!c || !out_host) return fail(MQR_ERR_INVALID_ARG, "NULL argument");
    if (region_bits < 1 || region_bits > kMaxRegionBits) return fail(MQR_ERR_INVALID_ARG, "region_bits must be 1..4");
    if (c->snap_pending) (void)index_ready(c);   // a newer snapshot invalidates the join records
    if (!c->have_tick) return fail(MQR_ERR_INVALID_ARG, "no tick has completed yet");
    if (c->last_emit_kind == kEmitAtomic)
        return fail(MQR_ERR_INVALID_ARG, "the last tick used the atomic baseline (no per-subquery counts)");
    if (c->n_worlds) return fail(MQR_ERR_INVALID_ARG, "not available with batched worlds");
    if (Q != c->last_q) return fail(MQR_ERR_INVALID_ARG, "Q must be the last tick's query count");
    if (Q && !rects_dev) return fail(MQR_ERR_INVALID_ARG, "rects_dev is NULL");
    const size_t R = (size_t)1 << (2 * region_bits);
    MQR_CUDA(cudaSetDevice(c->device));
    MQR_CUDA(c->region_stats.ensure(kRegionStats * R));
    MQR_CUDA(launch_region_work(c->stream, c->num_sms, c->leaf_lo.p, c->leaf_beg.p, (uint32_t)c->last.n_leaves,
                                c->sub_leaf.p, c->sub_len.p, c->sub_res.p, c->last.n_sub,
                                reinterpret_cast<const float4 *>(rects_dev), Q, c->bounds.xmin, c->bounds.ymin,
                                c->sx, c->sy, region_bits, c->region_stats.p));
    MQR_CUDA(cudaMemcpyAsync(out_host, c->region_stats.p, kRegionStats * R * sizeof(double),
                             cudaMemcpyDeviceToHost, c->stream));
    MQR_CUDA(cudaStreamSynchronize(c->stream));
    return MQR_OK;
}

mqr_status mqr_result_footprint(mqr_ctx *c, uint64_t *out_host) {
    if (!c || !out_host) return fail(MQR_ERR_INVALID_ARG, "NULL argument");
    if (c->snap_pending) (void)index_ready(c);   // a newer snapshot invalidates the join records
    if (!c->have_tick) return fail(MQR_ERR_INVALID_ARG, "no tick has completed yet");
    if (c->last_emit_kind == kEmitAtomic)
        return fail(MQR_ERR_INVALID_ARG, "the last tick used the atomic baseline (no per-subquery counts)");
    MQR_CUDA(cudaSetDevice(c->device));
    const uint32_t L = (uint32_t)c->last.n_leaves;
    MQR_CUDA(c->fp_mark.ensure(std::max<size_t>(((size_t)L + 3) & ~(size_t)3, 4)));
    MQR_CUDA(c->fp_sum.ensure(4));
    MQR_CUDA(launch_footprint(c->stream, c->num_sms, c->sub_leaf.p, c->sub_len.p, c->sub_res.p, c->last.n_sub,
                              c->leaf_beg.p, L, c->fp_mark.p, c->fp_sum.p));
    unsigned long long h[4] = {0, 0, 0, 0};
    MQR_CUDA(cudaMemcpyAsync(h, c->fp_sum.p, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    MQR_CUDA(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < 4; ++i) out_host[i] = h[i];
    return MQR_OK;
}

mqr_status mqr_debug_stall_scan(int enable) {
    g_stall_scan.store(enable != 0);
    return MQR_OK;
}

mqr_status mqr_export_state(mqr_ctx *c, float *xy_host, uint8_t *present_host, uint32_t cap) {
    if (!c || !xy_host || !present_host) return fail(MQR_ERR_INVALID_ARG, "NULL argument");
    if (cap < c->nmax) return fail(MQR_ERR_CAPACITY, "buffers must hold max_objects entries");
    MQR_CUDA(cudaSetDevice(c->device));
    if (!c->nmax) return MQR_OK;
    MQR_CUDA(c->state_flags.ensure(c->nmax));
    launch_state_flags(c->stream, c->stamp.p, c->nmax, c->state_flags.p);
    MQR_CUDA(cudaGetLastError());
    MQR_CUDA(cudaMemcpyAsync(xy_host, c->pos.p, (size_t)c->nmax * sizeof(float2), cudaMemcpyDeviceToHost,
                             c->stream));
    MQR_CUDA(cudaMemcpyAsync(present_host, c->state_flags.p, c->nmax, cudaMemcpyDeviceToHost, c->stream));
    MQR_CUDA(cudaStreamSynchronize(c->stream));
    return MQR_OK;
}

mqr_status mqr_import_state(mqr_ctx *c, const float *xy_host, const uint8_t *present_host, uint32_t n) {
    if (!c || !xy_host || !present_host) return fail(MQR_ERR_INVALID_ARG, "NULL argument");
    if (n != c->nmax) return fail(MQR_ERR_INVALID_ARG, "n must equal max_objects");
    MQR_CUDA(cudaSetDevice(c->device));
    if (!c->nmax) return MQR_OK;
    MQR_CUDA(c->state_flags.ensure(c->nmax));
    MQR_CUDA(cudaStreamSynchronize(c->stream));
    ++c->epoch;                                    // restored objects: updated by this call
    MQR_CUDA(cudaMemcpyAsync(c->pos.p, xy_host, (size_t)c->nmax * sizeof(float2), cudaMemcpyHostToDevice,
                             c->stream));
    MQR_CUDA(cudaMemcpyAsync(c->state_flags.p, present_host, c->nmax, cudaMemcpyHostToDevice, c->stream));
    launch_state_stamps(c->stream, c->state_flags.p, c->nmax, c->epoch, c->stamp.p);
    MQR_CUDA(cudaGetLastError());
    MQR_CUDA(cudaStreamSynchronize(c->stream));    // the host buffers may be reused at once
    return MQR_OK;
}

mqr_status mqr_debug_fail_allocation(int after) {
    g_fail_alloc_after.store(after < 0 ? -1 : after);
    return MQR_OK;
}

mqr_status mqr_get_leaves(mqr_ctx *c, uint32_t *leaves_host, uint64_t cap, uint64_t *n) {
    if (!c || !n) return fail(MQR_ERR_INVALID_ARG, "NULL argument");
    {
        mqr_status si = index_ready(c);
        if (si != MQR_OK) return si;
    }
    const uint64_t L = c->last.n_leaves;
    *n = L;
    if (L == 0) return MQR_OK;
    if (cap < L || !leaves_host) return fail(MQR_ERR_CAPACITY, "leaves_host too small");
    MQR_CUDA(cudaSetDevice(c->device));
    uint32_t *lo = new (std::nothrow) uint32_t[3 * L + 1];
    if (!lo) return fail(MQR_ERR_OOM, "host allocation failed");
    uint32_t *hi = lo + L, *beg = lo + 2 * L;
    cudaError_t e = cudaMemcpyAsync(lo, c->leaf_lo.p, L * 4, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaMemcpyAsync(hi, c->leaf_hi.p, L * 4, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaMemcpyAsync(beg, c->leaf_beg.p, (L + 1) * 4, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) {
        delete[] lo;
        return cuda_fail(e, "mqr_get_leaves copy");
    }
    for (uint64_t k = 0; k < L; ++k) {
        uint32_t span = hi[k] - lo[k] + 1u;
        uint32_t s = 0;
        while ((1ull << (2 * (s + 1))) <= span) ++s;
        leaves_host[4 * k + 0] = 15u - s;
        leaves_host[4 * k + 1] = s >= 15 ? 0u : lo[k] >> (2 * s);
        leaves_host[4 * k + 2] = beg[k];
        leaves_host[4 * k + 3] = beg[k + 1];
    }
    delete[] lo;
    return MQR_OK;
}

mqr_status mqr_get_sorted(mqr_ctx *c, uint32_t *keys_host, uint32_t *ids_host, uint64_t cap, uint64_t *n) {
    if (!c || !n) return fail(MQR_ERR_INVALID_ARG, "NULL argument");
    {
        mqr_status si = index_ready(c);
        if (si != MQR_OK) return si;
    }
    const uint64_t N = c->last.n_present;
    *n = N;
    if (N == 0) return MQR_OK;
    if (cap < N) return fail(MQR_ERR_CAPACITY, "buffers too small");
    MQR_CUDA(cudaSetDevice(c->device));
    if (keys_host) MQR_CUDA(cudaMemcpyAsync(keys_host, c->skey.p, N * 4, cudaMemcpyDeviceToHost, c->stream));
    if (ids_host) MQR_CUDA(cudaMemcpyAsync(ids_host, c->sid.p, N * 4, cudaMemcpyDeviceToHost, c->stream));
    MQR_CUDA(cudaStreamSynchronize(c->stream));
    return MQR_OK;
}

mqr_status mqr_get_sorted_async(mqr_ctx *c, uint32_t *ids_host, uint64_t cap, uint64_t *n) {
    if (!c || !n || !ids_host) return fail(MQR_ERR_INVALID_ARG, "NULL argument");
    {
        mqr_status si = index_ready(c);
        if (si != MQR_OK) return si;
    }
    if (!c->copy_stream) return fail(MQR_ERR_INVALID_ARG, "no mqr_tick_host_async before");
    const uint64_t N = c->last.n_present;
    *n = N;
    if (N == 0) return MQR_OK;
    if (cap < N) return fail(MQR_ERR_CAPACITY, "buffer too small");
    MQR_CUDA(cudaSetDevice(c->device));
    const int b = c->next_stage ^ 1;                 // the staging set of the last asynchronous tick
    DevBuf<uint32_t> &snap = b ? c->sid_stage2 : c->sid_stage;
    if (!c->snap_done) MQR_CUDA(cudaEventCreateWithFlags(&c->snap_done, cudaEventDisableTiming));
    // the previous copy out of this snapshot buffer is ordered before the last tick's output copy,
    // which the last asynchronous tick already waited for
    MQR_CUDA(snap.ensure(c->nmax));
    MQR_CUDA(cudaMemcpyAsync(snap.p, c->sid.p, N * 4, cudaMemcpyDeviceToDevice, c->stream));
    MQR_CUDA(cudaEventRecord(c->snap_done, c->stream));
    MQR_CUDA(cudaStreamWaitEvent(c->copy_stream, c->snap_done, 0));
    MQR_CUDA(cudaMemcpyAsync(ids_host, snap.p, N * 4, cudaMemcpyDeviceToHost, c->copy_stream));
    MQR_CUDA(cudaEventRecord(c->copy_done[b], c->copy_stream));
    c->copy_pending[b] = true;
    return MQR_OK;
}

mqr_status mqr_set_timing_phases(mqr_ctx *c, uint32_t phase_mask) {
    if (!c) return fail(MQR_ERR_INVALID_ARG, "ctx is NULL");
    MQR_CUDA(cudaSetDevice(c->device));
    if (phase_mask && !c->ev[0][0]) {
        for (int p = 0; p < MQR_NUM_PHASES; ++p)
            for (int k = 0; k < 2; ++k) MQR_CUDA(cudaEventCreate(&c->ev[p][k]));
        for (int p = 0; p < mqr_ctx::kMaxPendingUpdates; ++p)
            for (int k = 0; k < 2; ++k) MQR_CUDA(cudaEventCreate(&c->up_ev[p][k]));
    }
    c->timing = phase_mask != 0;
    c->timing_mask = phase_mask & ((1u << MQR_NUM_PHASES) - 1u);
    std::memset(&c->acc, 0, sizeof(c->acc));
    std::memset(c->ev_used, 0, sizeof(c->ev_used));
    c->up_pending = 0;
    c->up_launches = 0;
    return MQR_OK;
}

mqr_status mqr_set_timing(mqr_ctx *c, int enable) {
    return mqr_set_timing_phases(c, enable ? (1u << MQR_NUM_PHASES) - 1u : 0u);
}

mqr_status mqr_get_timing(const mqr_ctx *c, mqr_timing *out) {
    if (!c || !out) return fail(MQR_ERR_INVALID_ARG, "NULL argument");
    *out = c->acc;
    return MQR_OK;
}

}  // extern "C"
