/*
 * mqr.h -- C ABI of libmqr: repeated range queries over moving objects on one
 * GB300 GPU (sm_103a).
 *
 * The library answers, tick after tick, the spatial join between the latest
 * known positions of a population of moving objects and the range queries
 * issued during the tick (Lettich et al., "Manycore processing of repeated
 * range queries over massive moving objects observations", Sec. 2.5 "Problem
 * statement").  It indexes the objects with a point-region quadtree whose
 * leaves hold at most leaf_cap objects (Def. "MBR partitioning into a
 * quadtree-induced regular grid", Alg. 1), splits every query over the leaves
 * it meets (Def. "Mapping functions"), tests intersecting subqueries against
 * the leaf's objects into 32-bit bitmap words (Sec. 5.4, Alg. 2), and decodes
 * the words plus the covering subqueries into the result (Sec. 5.5 Alg. 4,
 * Sec. 5.6).
 *
 * Conventions shared by every entry point:
 *  - Every call returns an mqr_status; nothing aborts the process.  On an
 *    error, mqr_last_error() returns a message (thread-local, valid until the
 *    next call on the same thread).
 *  - Pointers named *_dev are CUDA device pointers (or managed memory) owned
 *    by the caller; pointers named *_host are host pointers owned by the
 *    caller.  The library never frees caller memory and keeps no pointer to
 *    it after the call returns.
 *  - All device work is enqueued on the context's stream (see mqr_create_ex);
 *    device inputs must stay valid until that stream reaches the call's work,
 *    which mqr_tick waits for before returning.
 *  - A context is not thread-safe: one thread at a time per context.
 *  - Coordinates are IEEE float32; a query (xa, ya, xb, yb) is the CLOSED
 *    rectangle xa <= x <= xb, ya <= y <= yb (Def. 1).  A query with a NaN
 *    corner, or with xa > xb or ya > yb, has an empty result.  NaN object
 *    coordinates never match; infinite ones match only infinite edges.
 */
#ifndef MQR_H
#define MQR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mqr_ctx mqr_ctx;

typedef enum {
    MQR_OK = 0,
    MQR_ERR_INVALID_ARG = 1, /* bad pointer, size, kind or id                */
    MQR_ERR_OOM = 2,         /* device or host allocation failed             */
    MQR_ERR_CAPACITY = 3,    /* output buffer too small: *out_count = needed */
    MQR_ERR_CUDA = 4,        /* a CUDA call failed (message has the detail)  */
    MQR_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up           */
    MQR_ERR_INTERNAL = 6
} mqr_status;

/* The indexed space: objects outside it are still answered exactly (their
 * cell index is clamped to the border cells). */
typedef struct {
    float xmin, ymin, xmax, ymax;
} mqr_rect;

/* Result layouts written by mqr_tick.  R = total number of (query, object)
 * results of the tick, Q = number of queries, W = ceil(max_objects / 32).
 *  PAIRS         out_dev: uint32 pairs (qidx, id), R of them (8*R bytes),
 *                grouped by query in ascending qidx; order inside a query
 *                unspecified.
 *  PAIRS_SORTED  as PAIRS, ascending in (qidx, id).
 *  CSR           out_dev: uint32 ids, R of them (4*R bytes), grouped by query
 *                in ascending qidx; offsets_dev (required) gets uint64[Q+1]
 *                with the start of every query's list.  Order inside a query
 *                unspecified.
 *  CSR_SORTED    as CSR, ids ascending inside each query.
 *  BITMAP        out_dev: Q rows of W uint32 words (4*Q*W bytes); bit
 *                (id mod 32) of word id/32 of row qidx is 1 iff object id is
 *                in the result of query qidx.  Padding bits are 0.
 *  COUNT         no id output (out_dev may be NULL); only *out_count and, if
 *                given, offsets_dev.
 *  RUNS          covering-compressed pairs (the paper reports a covering
 *                subquery as (query, cell) and leaves its expansion to the
 *                consumer, Sec. 1 and Sec. 5.6): out_dev holds 8-byte
 *                elements grouped by query in ascending qidx, each either a
 *                result pair (qidx, id) with qidx < 2^31, or a covering run
 *                taking two elements (qidx | 2^31, first) (count, 0): every
 *                object sorted_ids[first .. first + count) of the tick's
 *                Morton-sorted order (mqr_get_sorted) is in the result of
 *                qidx.  *out_count = number of elements (R_I + 2 * runs);
 *                offsets_dev counts elements too.  Every result appears
 *                exactly once, as a pair or inside one run.
 *  PAIRS_ATOMIC  as PAIRS but in no particular order, produced by the
 *                paper's baseline filtering (Alg. 3: results appended through
 *                shared-memory buffers and an atomic global counter, with no
 *                bitmaps and no decoding phase; the ablation of the paper's
 *                study S1).  offsets_dev must be NULL.
 * offsets_dev, when non-NULL, receives the per-query offsets for every kind
 * except PAIRS_ATOMIC.
 * out_dev must be 16-byte aligned (cudaMalloc and torch allocations are).
 * The sorted kinds are limited to R < 2^30. */
typedef enum {
    MQR_OUT_PAIRS = 0,
    MQR_OUT_PAIRS_SORTED = 1,
    MQR_OUT_CSR = 2,
    MQR_OUT_CSR_SORTED = 3,
    MQR_OUT_BITMAP = 4,
    MQR_OUT_COUNT = 5,
    MQR_OUT_RUNS = 6,
    MQR_OUT_PAIRS_ATOMIC = 7
} mqr_out_kind;

typedef enum {
    MQR_INDEX_QUADTREE = 0,     /* PR-quadtree, leaves hold <= leaf_cap objects (Alg. 1) */
    MQR_INDEX_UNIFORM_GRID = 1  /* uniform grid of 2^grid_level cells per axis (Def. uniform grid) */
} mqr_index_kind;

typedef struct {
    uint32_t max_objects;  /* object ids are in [0, max_objects)                      */
    uint32_t leaf_cap;     /* th_quad: a quadrant holding more objects is split        */
    int32_t index_kind;    /* mqr_index_kind                                           */
    uint32_t grid_level;   /* uniform grid only: 1..15                                 */
    int32_t covering;      /* 1 (default): covering subqueries skip containment tests
                              (Sec. 5.6); 0: every subquery is tested                  */
    int32_t reserved[3];   /* must be 0                                                */
} mqr_config;

/* Counters of the last completed tick (Sec. 7 metrics). */
typedef struct {
    uint64_t n_objects;          /* objects present (ever updated)                 */
    uint64_t n_queries;
    uint64_t n_leaves;           /* non-empty index cells                          */
    uint64_t max_level;          /* deepest leaf level (l_deep)                    */
    uint64_t n_sub_intersecting; /* |Q_I|                                          */
    uint64_t n_sub_covering;     /* covering subqueries, counted per leaf          */
    uint64_t n_covering_runs;    /* covering subqueries after merging adjacent leaves */
    uint64_t n_tests;            /* sum over cells of |Q_I^c| * |P^c|              */
    uint64_t n_filter_items;     /* warp work items of the filtering kernel        */
    uint64_t n_bitmap_words;     /* 32-bit words of the filtering bitmaps          */
    uint64_t n_results;          /* R                                              */
    uint64_t n_results_covering; /* results coming from covering subqueries        */
    uint64_t n_retries;          /* internal buffer growths during the tick        */
    uint64_t n_filter_loads;     /* object records loaded by the filtering kernel  */
    uint64_t n_pairs;            /* (query, block) pairs of query splitting        */
    uint64_t n_candidates;       /* (query, leaf) candidates classified            */
} mqr_stats;

/* Pipeline phases timed by mqr_set_timing (CUDA events on the context's
 * stream around each phase's kernels). */
typedef enum {
    MQR_PHASE_UPDATES = 0,     /* position updates (Sec. 2.2)                  */
    MQR_PHASE_KEYS = 1,        /* Morton keys + sort histograms (Alg. 1)       */
    MQR_PHASE_SORT = 2,        /* radix sort of the objects (Alg. 1)           */
    MQR_PHASE_LEAVES = 3,      /* quadtree / grid leaves (Alg. 1)              */
    MQR_PHASE_QUERY_BLOCKS = 4,/* query splitting: lookup table, blocks, scan (Sec. 5.3) */
    MQR_PHASE_GROUP = 5,       /* grouping subqueries by leaf (Sec. 5.3 sorting) */
    MQR_PHASE_CANDIDATES = 6,  /* query splitting: candidates -> subqueries      */
    MQR_PHASE_FILTER = 7,      /* filtering into bitmap words (Sec. 5.4)        */
    MQR_PHASE_RESULT_SCAN = 8, /* result-count scan (Sec. 5.5)                  */
    MQR_PHASE_EMIT = 9,        /* decoding + covering expansion (Sec. 5.5, 5.6) */
    MQR_PHASE_OFFSETS = 10,    /* per-query offsets                             */
    MQR_PHASE_OUTPUT_SORT = 11,/* sorted output kinds                           */
    MQR_NUM_PHASES = 12
} mqr_phase;

typedef struct {
    double ms[MQR_NUM_PHASES];         /* accumulated device time per phase      */
    uint64_t launches[MQR_NUM_PHASES]; /* kernels launched per phase             */
    uint64_t ticks;                    /* ticks accumulated                      */
} mqr_timing;

/* Fill *cfg with defaults: max_objects = 1<<20, leaf_cap = 128, quadtree,
 * grid_level = 8, covering = 1. */
mqr_status mqr_config_default(mqr_config *cfg);

/* Create a context over `bounds` with a PR-quadtree index of leaf capacity
 * `leaf_cap` (th_quad, Def. quadtree grid) for object ids in
 * [0, max_objects).  Uses the CUDA device current on the calling thread and a
 * stream the context creates.  *out receives the context; destroy it with
 * mqr_destroy.  Errors: INVALID_ARG (NULL out, leaf_cap == 0, bounds not
 * finite or empty), OOM, CUDA. */
mqr_status mqr_create(mqr_rect bounds, uint32_t leaf_cap, uint32_t max_objects, mqr_ctx **out);

/* As mqr_create with every knob of mqr_config.  `cuda_stream` is a
 * cudaStream_t the caller owns (NULL: the context creates its own); all work
 * of the context is enqueued on it. */
mqr_status mqr_create_ex(mqr_rect bounds, const mqr_config *cfg, void *cuda_stream, mqr_ctx **out);

/* Apply position updates (Sec. 2.2 "Batch processing"): object ids_dev[i]
 * moves to (xy_dev[2i], xy_dev[2i+1]).  Within one call the LAST occurrence
 * of a repeated id wins; across calls the later call wins.  An object is
 * present from its first update on.  All calls made before an mqr_tick
 * belong to that tick; the tick answers against the state at its start
 * (timeslice semantics, Sec. 2.3), so calls made after mqr_tick returns
 * belong to the next tick.  ids_dev: uint32[n] device; xy_dev: float32[2n]
 * device, interleaved (x, y).  Asynchronous: returns once enqueued.  Ids
 * >= max_objects are ignored and reported as INVALID_ARG by the next
 * mqr_tick.  n == 0 is a no-op. */
mqr_status mqr_apply_updates(mqr_ctx *ctx, const uint32_t *ids_dev, const float *xy_dev, uint32_t n);

/* As mqr_apply_updates with host buffers (copied to the device on the
 * context's stream before the call returns; page-locked buffers copy fastest). */
mqr_status mqr_apply_updates_host(mqr_ctx *ctx, const uint32_t *ids_host, const float *xy_host, uint32_t n);

/* Answer Q queries against the current state (one tick, Sec. 2.5):
 * rects_dev: float32[4Q] device, (xa, ya, xb, yb) per query; the query index
 * qidx is its position in rects_dev.  kind: an mqr_out_kind.  out_dev /
 * out_capacity_bytes: caller's device output buffer (see mqr_out_kind).
 * out_count (host, required): receives the number of results R (pairs or ids),
 * for BITMAP the number of words Q*W, for RUNS the number of 8-byte elements.  offsets_dev: NULL or uint64[Q+1]
 * device.  Blocks until the tick's work on the stream is complete.
 * Errors: INVALID_ARG, CAPACITY (buffer too small; *out_count holds the
 * size needed, nothing usable was written; call again with a larger buffer),
 * TIMEOUT, CUDA, OOM. */
mqr_status mqr_tick(mqr_ctx *ctx, const float *rects_dev, uint32_t Q, int kind,
                    void *out_dev, uint64_t out_capacity_bytes, uint64_t *out_count,
                    uint64_t *offsets_dev);

/* As mqr_tick with host buffers: rects_host is copied in, the result is
 * copied to out_host (and offsets_host if non-NULL) before the call returns. */
mqr_status mqr_tick_host(mqr_ctx *ctx, const float *rects_host, uint32_t Q, int kind,
                         void *out_host, uint64_t out_capacity_bytes, uint64_t *out_count,
                         uint64_t *offsets_host);

/* As mqr_tick_host, but returns as soon as the tick's result is complete in
 * device staging memory and its copy to out_host (and offsets_host) has been
 * started on a second stream, so that the copy of one tick overlaps the
 * updates and kernels of the next (the host link, not the GPU, bounds a
 * pair-list output on this hardware).  *out_count is set on return.  The host
 * buffers must not be read or reused until mqr_host_wait returns; page-locked
 * buffers are needed for the overlap.  Two ticks' copies may be in flight (two
 * staging buffers alternate); a third call first waits for the oldest.
 * mqr_tick_host waits for every pending copy first.  Library design
 * convenience, not a step of the method. */
mqr_status mqr_tick_host_async(mqr_ctx *ctx, const float *rects_host, uint32_t Q, int kind,
                               void *out_host, uint64_t out_capacity_bytes, uint64_t *out_count,
                               uint64_t *offsets_host);

/* Wait until every copy started by mqr_tick_host_async has landed. */
mqr_status mqr_host_wait(mqr_ctx *ctx);

/* After mqr_tick_host_async: start copying that tick's Morton-sorted object
 * ids (what a consumer of the RUNS kind needs to expand covering runs; the
 * same array as mqr_get_sorted's ids) to ids_host on the same second stream,
 * behind the tick's output.  *n receives their number; they land by
 * mqr_host_wait.  A snapshot is taken on the device first, so the next tick
 * may start at once.  cap (in ids) too small: CAPACITY. */
mqr_status mqr_get_sorted_async(mqr_ctx *ctx, uint32_t *ids_host, uint64_t cap, uint64_t *n);

/* A tick with admission by output memory, for served streams (the tick and
 * latency model of Sec. 2.4, Def. 2-3 and Lemma 2: a tick must finish within
 * the latency budget, so its output is bounded).  As mqr_tick, but instead of
 * failing with CAPACITY it answers the longest prefix rects[0 .. *admitted)
 * of the queries whose output fits out_capacity_bytes (the exact counts of
 * the two-pass scheme, Sec. 5.3, decide it before anything is written); the
 * queries from *admitted on are not answered, and the caller submits them
 * again in a later tick.  kind: PAIRS, CSR or RUNS.  *out_count: elements
 * written (results for PAIRS/CSR, 8-byte elements for RUNS).  offsets_dev:
 * NULL or uint64[Q+1] device; entries 0 .. *admitted are the answered
 * queries' offsets (later entries describe the unanswered queries and are to
 * be ignored).  Blocks until the output is written.  Errors as mqr_tick,
 * except that CAPACITY is not returned for the output buffer. */
mqr_status mqr_tick_admit(mqr_ctx *ctx, const float *rects_dev, uint32_t Q, int kind, void *out_dev,
                          uint64_t out_capacity_bytes, uint32_t *admitted, uint64_t *out_count,
                          uint64_t *offsets_dev);

/* Join slots: continuous batching of query batches against one snapshot of
 * the object state (the served-stream model of Sec. 2.4, Def. 2-3 and
 * Lemmas 1-2: batches that arrive while others are on the GPU start at once
 * and their work overlaps on the device; the timeslice semantics of Sec. 2.3
 * hold because every batch of a snapshot sees the same positions).
 *
 * mqr_snapshot builds the index (Morton keys, sort, leaves; Alg. 1) of the
 * context's current state on the context's stream and returns without
 * waiting; the slots of the context then answer batches against it, each on
 * its own stream and with its own per-query buffers, reading the snapshot's
 * index without copying it.  The next mqr_snapshot (or mqr_tick) of the
 * context overwrites the index, so every slot's join must have been ended
 * first (else INVALID_ARG); position updates may be applied while joins run
 * (they belong to the next snapshot).
 *
 * mqr_slot_create: a slot of ctx working on cuda_stream (a cudaStream_t the
 * caller owns, which should be another stream than the context's; NULL: the
 * slot creates its own), with about 16 bytes per object of per-leaf lists
 * and per-query buffers grown on demand.  Errors: INVALID_ARG, OOM, CUDA.  mqr_slot_destroy: waits for the slot's work and
 * frees it; NULL is a no-op.  Destroying a context makes its remaining slots
 * unusable (destroy them too).  Batched worlds are not supported by slots. */
typedef struct mqr_slot mqr_slot;
mqr_status mqr_slot_create(mqr_ctx *ctx, void *cuda_stream, mqr_slot **out);
void mqr_slot_destroy(mqr_slot *slot);
mqr_status mqr_snapshot(mqr_ctx *ctx);

/* Start answering Q queries (rects_dev as for mqr_tick) on the slot against
 * the context's last snapshot, with admission by output memory as in
 * mqr_tick_admit: the longest prefix of the queries whose output fits
 * out_capacity_bytes is answered (decided on the device from the exact
 * counts, before anything is written).  kind: PAIRS, CSR or RUNS (RUNS
 * refers to the snapshot's sorted ids, mqr_get_sorted of the context).
 * offsets_dev: NULL or uint64[Q+1] device (entries 0 .. admitted valid).
 * Returns once the work is enqueued on the slot's stream; rects_dev, out_dev
 * and offsets_dev must stay valid until mqr_slot_end.  One join per slot at a
 * time.  Errors: INVALID_ARG (no snapshot, a join pending, bad kind or
 * alignment), OOM, CUDA. */
mqr_status mqr_slot_begin(mqr_slot *slot, const float *rects_dev, uint32_t Q, int kind, void *out_dev,
                          uint64_t out_capacity_bytes, uint64_t *offsets_dev);

/* Wait for the slot's join (answering it again if an internal buffer had to
 * grow) and report *admitted (queries answered: a prefix) and *out_count
 * (output elements written).  Errors: INVALID_ARG (nothing pending; or an
 * update id >= max_objects was ignored, after the join was answered),
 * TIMEOUT, CUDA, OOM. */
mqr_status mqr_slot_end(mqr_slot *slot, uint32_t *admitted, uint64_t *out_count);

/* Counters of the slot's last join (as mqr_get_stats). */
mqr_status mqr_slot_get_stats(const mqr_slot *slot, mqr_stats *out);

/* Graph mode (enable = 1): the tick's ~20 kernel launches are captured once
 * into a CUDA graph and the graph is replayed by later ticks with the same
 * arguments (rects_dev, Q, kind, out_dev, capacity, offsets_dev) while no
 * internal buffer was reallocated; anything else captures again.  Results
 * are identical to the plain launches.  Phase timing (mqr_set_timing,
 * mqr_set_timing_phases) works under replay: the timed phases' event records
 * are event-record nodes of the captured graph, recorded by every replay (a
 * change of the timed phases captures again).  Ticks with slots on the
 * context, admission (mqr_tick_admit) or the sorted kinds' output sort run as
 * plain launches.  enable = 0 frees the graph.  Library design convenience,
 * not a step of the method. */
mqr_status mqr_set_graph(mqr_ctx *ctx, int enable);

/* Batched independent worlds in one index (many small instances of the
 * problem of Sec. 2.5 answered by one tick; the paper has no batched mode,
 * this keeps each world's result exact and its own).  World w owns the
 * object ids [obj_base_host[w], obj_base_host[w+1]) (obj_base_host: uint32
 * host array of n_worlds+1 entries, 0 first, max_objects last, not
 * decreasing); its objects and queries are in the context's bounds, in its
 * own coordinates.  Internally the quadtree (Alg. 1) gets ceil(log4
 * n_worlds) levels above the worlds' roots, so each world is one node, keys
 * keep their 30 bits (a world's cells are its l_max cells shifted right by
 * those levels) and no leaf spans two worlds; containment tests use the
 * objects' own coordinates, so results are exact.  n_worlds = 1 returns to
 * the plain index.  1 <= n_worlds <= 16384.  Call between ticks; the query
 * ranges must then be set with mqr_set_query_worlds. */
mqr_status mqr_set_worlds(mqr_ctx *ctx, uint32_t n_worlds, const uint32_t *obj_base_host);

/* Query ranges of the batched worlds for the following ticks: the queries
 * [q_base_host[w], q_base_host[w+1]) of a tick's rects belong to world w
 * (uint32 host array of n_worlds+1 entries, 0 first, not decreasing); the
 * ticks must pass Q = q_base_host[n_worlds].  Result pairs carry the global
 * query index and object id. */
mqr_status mqr_set_query_worlds(mqr_ctx *ctx, const uint32_t *q_base_host);

/* Change the index between ticks (leaves are rebuilt every tick, Alg. 1):
 * index_kind MQR_INDEX_QUADTREE with leaf_cap >= 1 (th_quad), or
 * MQR_INDEX_UNIFORM_GRID with 1 <= grid_level <= 15 (and >= the batched
 * worlds' levels).  Results never depend on the choice; time does.  Errors:
 * INVALID_ARG. */
mqr_status mqr_set_index(mqr_ctx *ctx, int index_kind, uint32_t leaf_cap, uint32_t grid_level);

/* Launch shapes of the work-item kernels: blocks per SM of the candidate
 * pass (which also places the subquery records), the pass that files the
 * intersecting subqueries into their leaves' lists (compact_blocks_per_sm),
 * the filter (Alg. 2) and the decoding / emit (Alg. 4); 0 keeps the default
 * (8).  Their blocks draw work items from
 * counters or stride over them, so the shapes change time, never results;
 * block sizes are fixed per kernel by its register budget.  An autotuner
 * (autotune.tune_launch_config) picks them by timing.  1 <= value <= 64.
 * Call between ticks.  Errors: INVALID_ARG. */
typedef struct {
    uint32_t candidate_blocks_per_sm;
    uint32_t compact_blocks_per_sm;
    uint32_t filter_blocks_per_sm;
    uint32_t emit_blocks_per_sm;
} mqr_launch_config;
mqr_status mqr_set_launch_config(mqr_ctx *ctx, const mqr_launch_config *cfg);

/* Per-region split thresholds of the quadtree (Alg. 1's th_quad chosen per
 * region instead of once): the quadrants of level region_bits (1..4) are the
 * regions, numbered in Morton order (region r holds the keys whose top
 * 2*region_bits bits are r); a quadrant at or below that level splits iff it
 * holds more objects than caps_host[r] of its region (and is above l_max);
 * non-empty quadrants above that level always split.  caps_host: uint32 host
 * array of 4^region_bits thresholds, each in 1..16384 (copied).  leaf_cap is
 * then unused; region_bits = 0 returns to the single leaf_cap (caps_host may
 * be NULL).  Applies to MQR_INDEX_QUADTREE ticks (a uniform grid ignores it);
 * combines with batched worlds (no leaf above either level).  Results never
 * depend on the thresholds; time does.  Call between ticks.  Errors:
 * INVALID_ARG. */
mqr_status mqr_set_region_caps(mqr_ctx *ctx, uint32_t region_bits, const uint32_t *caps_host);

/* Objects per region in the last completed tick: counts_host[r] = the number
 * of present objects whose key has the Morton prefix r of length
 * 2*region_bits (uint32 host array of 4^region_bits entries; regions as in
 * mqr_set_region_caps, in the batched worlds' key space when worlds are
 * set).  Computed on the device from the tick's sorted keys (Alg. 1), so a
 * caller can choose the next tick's per-region thresholds from the local
 * density.  1 <= region_bits <= 4.  Blocks.  Errors: INVALID_ARG (also
 * before the first tick). */
mqr_status mqr_region_counts(mqr_ctx *ctx, uint32_t region_bits, uint32_t *counts_host);

/* Per-region work of the last completed tick, the node-level data a cost
 * model of the split thresholds learns from: out_host (double host array of
 * 9 x 4^region_bits, statistic-major: out_host[s * 4^region_bits + r]) gets
 * for every region r (as in mqr_region_counts)
 *   s = 0 objects, 1 leaves (Alg. 1), 2 queries whose centre lies in r
 *   (inverted, NaN or infinite rectangles skipped), 3 the sum of log2 of
 *   those queries' longer sides, 4 intersecting subqueries on leaves of r,
 *   5 covering subqueries on leaves of r (Def. mapping functions), 6 the
 *   containment tests of the filter (Alg. 2: the leaf's objects for every
 *   intersecting subquery), 7 results of intersecting subqueries, 8 results
 *   of covering subqueries.
 * rects_dev / Q: the last tick's queries (device, as passed to it).  Computed
 * on the device from the tick's leaf table and subquery records; valid until
 * the next tick.  1 <= region_bits <= 4.  Blocks.  Errors: INVALID_ARG (no
 * tick yet, a different Q, the atomic-baseline kind, batched worlds). */
mqr_status mqr_region_work(mqr_ctx *ctx, const float *rects_dev, uint32_t Q, uint32_t region_bits,
                           double *out_host);

/* Learned tick-cost model: a multilayer perceptron 5 -> 64 -> 64 -> 1 with
 * ReLU hidden layers, trained on the device (hand-written forward, backward
 * and Adam kernels, one block) to map tick features to the logarithm of the
 * tick's time, so that a caller can pick the index configuration of the next
 * tick (mqr_set_index).  The paper models its phases' costs analytically
 * (the filtering complexity of Sec. 5.4); this learns the cost from
 * measurements instead.  Parameters (mqr_cost_param_count() floats):
 * W1[64][5], b1[64], W2[64][64], b2[64], W3[64], b3, row-major, host
 * arrays.  The model lives on the current device with its own stream. */
typedef struct mqr_cost mqr_cost;
uint32_t mqr_cost_param_count(void);
/* Parameters start at zero: set an initialisation with mqr_cost_set_params. */
mqr_status mqr_cost_create(mqr_cost **out);
/* Replace the parameters (host array) and reset the optimiser state. */
mqr_status mqr_cost_set_params(mqr_cost *m, const float *params_host, uint32_t n_params);
mqr_status mqr_cost_get_params(mqr_cost *m, float *params_host, uint32_t n_params);
/* `epochs` full-batch Adam steps (beta 0.9 / 0.999, eps 1e-8, bias-corrected)
 * of the mean squared error over the n samples X_host[n][5] -> y_host[n];
 * *loss_out (may be NULL) = the loss before the last step.  Blocks. */
mqr_status mqr_cost_train(mqr_cost *m, const float *X_host, const float *y_host, uint32_t n, uint32_t epochs,
                          float lr, float *loss_out);
/* The gradient of the mean squared error over the n samples with respect to
 * the parameters (grad_host: mqr_cost_param_count() floats), computed by the
 * training kernel's backward pass without updating anything; *loss_out (may
 * be NULL) = the loss.  n >= 1.  Blocks. */
mqr_status mqr_cost_gradient(mqr_cost *m, const float *X_host, const float *y_host, uint32_t n, float *grad_host,
                             float *loss_out);
/* out_host[i] = model(X_host[i]) for n samples.  Blocks. */
mqr_status mqr_cost_predict(mqr_cost *m, const float *X_host, uint32_t n, float *out_host);
void mqr_cost_destroy(mqr_cost *m);

/* Counters of the last completed tick. */
mqr_status mqr_get_stats(const mqr_ctx *ctx, mqr_stats *out);

/* Copy the last tick's non-empty quadtree leaves (Alg. 1 output, Morton
 * order) to the host: 4 uint32 per leaf {level, z, begin, end}, where z is
 * the leaf's Morton code at its level and [begin, end) its run of objects in
 * the tick's Morton-sorted object order.  *n receives the number of leaves;
 * if cap (in leaves) is too small, CAPACITY is returned and nothing copied. */
mqr_status mqr_get_leaves(mqr_ctx *ctx, uint32_t *leaves_host, uint64_t cap, uint64_t *n);

/* Copy the last tick's Morton-sorted objects (Alg. 1 GPUradixSort output) to
 * the host: keys_host[k] = 30-bit Morton code at l_max = 15, ids_host[k] =
 * object id, for the *n present objects.  Either pointer may be NULL. */
mqr_status mqr_get_sorted(mqr_ctx *ctx, uint32_t *keys_host, uint32_t *ids_host, uint64_t cap, uint64_t *n);

/* The join's leaf footprint in the last completed tick: out_host[0] = the
 * leaves that produced at least one result (every leaf of a covering run,
 * Sec. 5.6, and the leaf of every intersecting subquery with a non-zero
 * result count, Sec. 5.4), out_host[1] = the objects in those leaves,
 * out_host[2] = the leaves with at least one intersecting subquery (the
 * cells the filtering of Alg. 2 tests), out_host[3] = the objects in those.
 * Decoding (Alg. 4) must read the ids of the first kind of leaf at least
 * once, filtering the positions of the second: 4 * out_host[1] and
 * 8 * out_host[3] bytes of the join's algorithmic traffic.
 * out_host: uint64 host array of 4.  Computed on the device from the tick's
 * subquery records and leaf table (valid until the next tick); a measurement,
 * not a step of the method.  Blocks.  Errors: INVALID_ARG (NULL, no tick yet,
 * the atomic-baseline kind), OOM, CUDA. */
mqr_status mqr_result_footprint(mqr_ctx *ctx, uint64_t *out_host);

/* Checkpoint of the object state (Sec. 2.2: the latest position of every
 * object; the index is rebuilt from it every tick, Alg. 1): xy_host (float
 * host array of 2 x max_objects, (x, y) per id) and present_host (uint8 host
 * array of max_objects: 1 if the object was ever updated) receive the state
 * as of the calls enqueued so far.  cap = the arrays' length in objects, at
 * least max_objects.  Blocks.  Errors: INVALID_ARG, CAPACITY. */
mqr_status mqr_export_state(mqr_ctx *ctx, float *xy_host, uint8_t *present_host, uint32_t cap);

/* Restart from a checkpoint: the state of every object becomes xy_host /
 * present_host (as mqr_export_state writes them; n = max_objects), as if one
 * update call had set the present ones, so later updates win over it.  A
 * context with the same bounds and configuration then answers every tick
 * exactly as the one that exported.  Blocks.  Errors: INVALID_ARG. */
mqr_status mqr_import_state(mqr_ctx *ctx, const float *xy_host, const uint8_t *present_host, uint32_t n);

/* Test hook for failure handling: the next `after` device buffer allocations
 * of any context succeed and the one after them fails as if the device were
 * out of memory (the call that needed it returns OOM, its context stays
 * usable); the hook then disarms itself.  after < 0 disarms it. */
mqr_status mqr_debug_fail_allocation(int after);

/* Test hook for the bounded device-side waits: enable != 0 arms it, and the
 * next tick that runs the result-count scan (Sec. 5.5; any context) runs it
 * with the status of its first tile withheld and a 1 ms wait limit, so that
 * every later tile's look-back wait runs out: that tick returns
 * MQR_ERR_TIMEOUT, writes no output, and leaves its context usable (the next
 * tick is answered normally).  The hook then disarms itself; enable = 0
 * disarms it.  The wait gives up on its own: nothing faults or hangs.  The
 * tick needs more than one scan tile (over 2,048 subquery records) for a
 * wait to happen. */
mqr_status mqr_debug_stall_scan(int enable);

/* Enable (1) or disable (0) per-phase timing; enabling resets the
 * accumulators.  Timing adds two event records per phase to the stream. */
mqr_status mqr_set_timing(mqr_ctx *ctx, int enable);

/* Per-phase timing of only the phases whose bit (1 << mqr_phase) is set in
 * phase_mask: their device time is measured with two event records each,
 * while kernel launches are counted for every phase (no events); 0 turns
 * timing off.  Resets the accumulators.  Fewer event records perturb the
 * tick less (each costs a few microseconds of stream time). */
mqr_status mqr_set_timing_phases(mqr_ctx *ctx, uint32_t phase_mask);

/* Per-phase device time and kernel-launch counts accumulated over the ticks
 * completed since timing was enabled. */
mqr_status mqr_get_timing(const mqr_ctx *ctx, mqr_timing *out);

/* Largest n accepted by mqr_sort_objects_noalloc. */
#define MQR_NOALLOC_MAX_OBJECTS 262144u

/* Allocation-free Morton sort of n objects, for callers that cannot allocate
 * device memory: embedders that own all device memory (a fixed budget or their
 * own pool) and latency-critical loops that cannot afford the device-wide
 * synchronisation cudaMalloc / cudaFree may cause.  The paper has no
 * counterpart: this is a library convenience, not a step of the method.
 * Objects 0..n-1 are at (xy_dev[2i], xy_dev[2i+1]) (float32, device, all
 * present); on return keys_out_dev[k] (uint32, device) holds the k-th
 * smallest Morton key at l_max = 15 over `bounds` and ids_out_dev[k] its
 * object id (ties in id order) -- the same order mqr_get_sorted reports for a
 * context holding those objects.  Scratch memory is a fixed array of about
 * 4.3 MB held by every GPU that loads the library until the process exits;
 * n > MQR_NOALLOC_MAX_OBJECTS is rejected with INVALID_ARG.  The first call
 * on a device looks the array's address up (cudaGetSymbolAddress), so make it
 * before any stream capture.  All calls share the array: calls that overlap
 * on the GPU (e.g. on different streams) race.  Blocks until done.  Errors:
 * INVALID_ARG, CUDA, TIMEOUT, INTERNAL.  cuda_stream: a cudaStream_t or NULL. */
mqr_status mqr_sort_objects_noalloc(mqr_rect bounds, const float *xy_dev, uint32_t n,
                                    uint32_t *keys_out_dev, uint32_t *ids_out_dev, void *cuda_stream);

/* Message of the last failed call on this thread ("" if none). */
const char *mqr_last_error(void);

/* Release the context and everything it allocated.  NULL is a no-op. */
void mqr_destroy(mqr_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* MQR_H */
