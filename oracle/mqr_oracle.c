/*
 * mqr_oracle.c -- plain, slow, single-threaded CPU oracle for the per-tick
 * repeated-range-query join of Lettich et al., "Manycore processing of
 * repeated range queries over massive moving objects observations".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  The CUDA product path
 * never calls it and shares no code, header, table or constant with it.
 *
 * What it computes, each function citing the passage it follows:
 *   - orc_apply_updates : batch processing, last update of an object in a tick
 *                         wins (Sec. 2.2 "Batch processing").
 *   - orc_join_grid     : Def. 1 (result set of a range query, closed
 *                         rectangle, FP32 comparisons) evaluated through a
 *                         uniform grid (Def. "MBR partitioning into a uniform
 *                         grid"), the method's answer written as its plain
 *                         definition.  Grid cell indices are computed in
 *                         double precision on purpose: any monotone cell
 *                         function gives the exact Def. 1 answer.
 *   - orc_join_brute    : Def. 1 by testing every (query, object) pair.
 *   - orc_count_grid    : Def. 1 result counts per query, and optionally an
 *                         order-independent checksum of each result set.
 *   - orc_cell / orc_morton / orc_keys : the Morton code z(i,j) of the
 *                         2^15 x 2^15 grid at l_max = 15 (Sec. 5.3 index
 *                         creation, Alg. 1 GPUcalculateMortonHash), with the
 *                         FP32 cell function read as
 *                         i = min(floor((x - x0) * scale), 2^15 - 1),
 *                         scale = 2^15 / (x1 - x0) rounded to FP32, NaN and
 *                         negative values mapped to cell 0.
 *   - orc_quadtree      : Alg. 1 (GPU-based PR-quadtree construction) executed
 *                         level by level on the Morton-sorted keys: detect the
 *                         child quadrant intervals of every quadrant to split,
 *                         keep a quadrant as a leaf when it holds at most
 *                         th_quad objects or sits at l_max.
 *   - orc_quadtree_regions : the same with a split threshold per region (the
 *                         quadrants of one chosen level): quadrants above that
 *                         level split when non-empty, the others compare their
 *                         count with their region's threshold.
 *   - orc_subqueries    : Def. "Mapping functions" (function g, query
 *                         splitting, intersecting vs covering subqueries),
 *                         by testing the query against every leaf.
 *
 * Every function is a direct transcription of its definition: no blocking,
 * fusion or reordering.  Build with -O2 -ffp-contract=off (no fast-math) so
 * that FP32 expressions are evaluated exactly as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Def. 1: membership of a point in a closed query rectangle.                 */
/* rect = (xa, ya, xb, yb); point (x, y) belongs iff xa<=x<=xb and ya<=y<=yb. */
/* ------------------------------------------------------------------------ */
static int orc_in_rect(float x, float y, const float *r)
{
    return (r[0] <= x) && (x <= r[2]) && (r[1] <= y) && (y <= r[3]);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2 batch processing: the updates of a tick are applied in arrival   */
/* order, so the most recent update of an object is the one that survives.   */
/* Returns 0, or -1 if an id is outside [0, nmax) (nothing is written then). */
/* ------------------------------------------------------------------------ */
int orc_apply_updates(float *pos, uint8_t *present, uint32_t nmax,
                      const uint32_t *ids, const float *xy, uint32_t n)
{
    for (uint32_t i = 0; i < n; ++i)
        if (ids[i] >= nmax) return -1;
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t id = ids[i];
        pos[2 * (size_t)id + 0] = xy[2 * (size_t)i + 0];
        pos[2 * (size_t)id + 1] = xy[2 * (size_t)i + 1];
        present[id] = 1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Dynamic result buffer (plain growable arrays).                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint32_t *ids;
    uint64_t n, cap;
} orc_vec;

static int orc_vec_push(orc_vec *v, uint32_t x)
{
    if (v->n == v->cap) {
        uint64_t nc = v->cap ? v->cap * 2 : 1024;
        uint32_t *p = (uint32_t *)realloc(v->ids, nc * sizeof(uint32_t));
        if (!p) return -1;
        v->ids = p;
        v->cap = nc;
    }
    v->ids[v->n++] = x;
    return 0;
}

static int orc_cmp_u32(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}

void orc_free(void *p) { free(p); }

/* A query is empty when a corner is NaN or the rectangle is inverted: Def. 1
 * then admits no point (every comparison with NaN is false). */
static int orc_query_is_empty(const float *r)
{
    if (isnan(r[0]) || isnan(r[1]) || isnan(r[2]) || isnan(r[3])) return 1;
    return (r[0] > r[2]) || (r[1] > r[3]);
}

/* ------------------------------------------------------------------------ */
/* Def. 1 by brute force: every query against every present object.          */
/* Output: offsets[Q+1] (caller-allocated) and a malloc'ed array of ids,     */
/* ascending per query, returned through *ids_out (free with orc_free).      */
/* Returns the total number of results, or -1 on allocation failure.        */
/* ------------------------------------------------------------------------ */
int64_t orc_join_brute(const float *pos, const uint8_t *present, uint32_t nmax,
                       const float *rects, uint32_t Q,
                       uint64_t *offsets, uint32_t **ids_out)
{
    orc_vec v = {0, 0, 0};
    for (uint32_t q = 0; q < Q; ++q) {
        const float *r = rects + 4 * (size_t)q;
        offsets[q] = v.n;
        for (uint32_t id = 0; id < nmax; ++id) {
            if (!present[id]) continue;
            if (orc_in_rect(pos[2 * (size_t)id], pos[2 * (size_t)id + 1], r))
                if (orc_vec_push(&v, id)) { free(v.ids); return -1; }
        }
    }
    offsets[Q] = v.n;
    *ids_out = v.ids;
    return (int64_t)v.n;
}

/* ------------------------------------------------------------------------ */
/* Def. 1 through a uniform grid over the bounds (Def. "MBR partitioning     */
/* into a uniform grid", cells of side cell_side, G x G cells with           */
/* G = clamp(floor((x1 - x0) / cell_side), 1, 4096)).  Cell indices in       */
/* double precision, clamped to [0, G-1], NaN to cell 0: a monotone map      */
/* applied to objects and to query corners alike, so every object that       */
/* satisfies the FP32 test of Def. 1 lies in the cell range of the query.    */
/* ------------------------------------------------------------------------ */
static uint32_t orc_grid_cell(double v, double lo, double cw, uint32_t G)
{
    if (isnan(v)) return 0;
    double t = floor((v - lo) / cw);
    if (!(t >= 0.0)) return 0;
    if (t >= (double)(G - 1)) return G - 1;
    return (uint32_t)t;
}

int64_t orc_join_grid(const float *pos, const uint8_t *present, uint32_t nmax,
                      const float *rects, uint32_t Q,
                      double x0, double y0, double x1, double y1,
                      double cell_side,
                      uint64_t *offsets, uint32_t **ids_out)
{
    if (!(cell_side > 0.0)) cell_side = 1e-12;
    double gx = floor((x1 - x0) / cell_side), gy = floor((y1 - y0) / cell_side);
    uint32_t GX = gx < 1.0 ? 1u : (gx > 4096.0 ? 4096u : (uint32_t)gx);
    uint32_t GY = gy < 1.0 ? 1u : (gy > 4096.0 ? 4096u : (uint32_t)gy);
    double cwx = (x1 - x0) / GX, cwy = (y1 - y0) / GY;
    size_t ncell = (size_t)GX * GY;

    /* Counting sort of present ids by cell: ids ascend within each cell. */
    uint64_t *cstart = (uint64_t *)calloc(ncell + 1, sizeof(uint64_t));
    uint32_t *cell_of = (uint32_t *)malloc((size_t)(nmax ? nmax : 1) * sizeof(uint32_t));
    if (!cstart || !cell_of) { free(cstart); free(cell_of); return -1; }
    uint64_t npres = 0;
    for (uint32_t id = 0; id < nmax; ++id) {
        if (!present[id]) continue;
        uint32_t ci = orc_grid_cell(pos[2 * (size_t)id], x0, cwx, GX);
        uint32_t cj = orc_grid_cell(pos[2 * (size_t)id + 1], y0, cwy, GY);
        cell_of[id] = cj * GX + ci;
        cstart[cell_of[id] + 1]++;
        npres++;
    }
    for (size_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
    uint32_t *cell_ids = (uint32_t *)malloc((size_t)(npres ? npres : 1) * sizeof(uint32_t));
    uint64_t *fill = (uint64_t *)malloc(ncell * sizeof(uint64_t));
    if (!cell_ids || !fill) { free(cstart); free(cell_of); free(cell_ids); free(fill); return -1; }
    memcpy(fill, cstart, ncell * sizeof(uint64_t));
    for (uint32_t id = 0; id < nmax; ++id)
        if (present[id]) cell_ids[fill[cell_of[id]]++] = id;

    orc_vec v = {0, 0, 0};
    for (uint32_t q = 0; q < Q; ++q) {
        const float *r = rects + 4 * (size_t)q;
        offsets[q] = v.n;
        if (orc_query_is_empty(r)) continue;
        uint32_t i0 = orc_grid_cell(r[0], x0, cwx, GX), i1 = orc_grid_cell(r[2], x0, cwx, GX);
        uint32_t j0 = orc_grid_cell(r[1], y0, cwy, GY), j1 = orc_grid_cell(r[3], y0, cwy, GY);
        uint64_t first = v.n;
        for (uint32_t cj = j0; cj <= j1; ++cj)
            for (uint32_t ci = i0; ci <= i1; ++ci) {
                size_t c = (size_t)cj * GX + ci;
                for (uint64_t k = cstart[c]; k < cstart[c + 1]; ++k) {
                    uint32_t id = cell_ids[k];
                    if (orc_in_rect(pos[2 * (size_t)id], pos[2 * (size_t)id + 1], r))
                        if (orc_vec_push(&v, id)) {
                            free(v.ids); free(cstart); free(cell_of); free(cell_ids); free(fill);
                            return -1;
                        }
                }
            }
        qsort(v.ids + first, (size_t)(v.n - first), sizeof(uint32_t), orc_cmp_u32);
    }
    offsets[Q] = v.n;
    free(cstart); free(cell_of); free(cell_ids); free(fill);
    *ids_out = v.ids;
    return (int64_t)v.n;
}

/* Order-independent checksum of one result (query q, object id): the
 * splitmix64 output function (Steele, Lea & Flood 2014; Vigna's constants)
 * applied to (q << 32 | id).  A query's checksum is the sum of its results'
 * values modulo 2^64, so any permutation of a result list gives the same
 * checksum while a missing, extra or changed id changes it. */
static uint64_t orc_result_hash(uint32_t q, uint32_t id)
{
    uint64_t z = ((uint64_t)q << 32) | id;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

/* Per-query result counts (Def. 1 through the same uniform grid, no id
 * list) and, if hashes is not NULL, each query's checksum of its results
 * (orc_result_hash summed over the Def. 1 result set): used to check large
 * workloads on every query without storing their id lists. */
int64_t orc_count_grid(const float *pos, const uint8_t *present, uint32_t nmax,
                       const float *rects, uint32_t Q,
                       double x0, double y0, double x1, double y1,
                       double cell_side, uint64_t *counts, uint64_t *hashes)
{
    if (!(cell_side > 0.0)) cell_side = 1e-12;
    double gx = floor((x1 - x0) / cell_side), gy = floor((y1 - y0) / cell_side);
    uint32_t GX = gx < 1.0 ? 1u : (gx > 4096.0 ? 4096u : (uint32_t)gx);
    uint32_t GY = gy < 1.0 ? 1u : (gy > 4096.0 ? 4096u : (uint32_t)gy);
    double cwx = (x1 - x0) / GX, cwy = (y1 - y0) / GY;
    size_t ncell = (size_t)GX * GY;
    uint64_t *cstart = (uint64_t *)calloc(ncell + 1, sizeof(uint64_t));
    uint32_t *cell_of = (uint32_t *)malloc((size_t)(nmax ? nmax : 1) * sizeof(uint32_t));
    if (!cstart || !cell_of) { free(cstart); free(cell_of); return -1; }
    uint64_t npres = 0;
    for (uint32_t id = 0; id < nmax; ++id) {
        if (!present[id]) continue;
        uint32_t ci = orc_grid_cell(pos[2 * (size_t)id], x0, cwx, GX);
        uint32_t cj = orc_grid_cell(pos[2 * (size_t)id + 1], y0, cwy, GY);
        cell_of[id] = cj * GX + ci;
        cstart[cell_of[id] + 1]++;
        npres++;
    }
    for (size_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
    uint32_t *cell_ids = (uint32_t *)malloc((size_t)(npres ? npres : 1) * sizeof(uint32_t));
    uint64_t *fill = (uint64_t *)malloc(ncell * sizeof(uint64_t));
    if (!cell_ids || !fill) { free(cstart); free(cell_of); free(cell_ids); free(fill); return -1; }
    memcpy(fill, cstart, ncell * sizeof(uint64_t));
    for (uint32_t id = 0; id < nmax; ++id)
        if (present[id]) cell_ids[fill[cell_of[id]]++] = id;
    uint64_t total = 0;
    for (uint32_t q = 0; q < Q; ++q) {
        const float *r = rects + 4 * (size_t)q;
        uint64_t cnt = 0, h = 0;
        if (!orc_query_is_empty(r)) {
            uint32_t i0 = orc_grid_cell(r[0], x0, cwx, GX), i1 = orc_grid_cell(r[2], x0, cwx, GX);
            uint32_t j0 = orc_grid_cell(r[1], y0, cwy, GY), j1 = orc_grid_cell(r[3], y0, cwy, GY);
            for (uint32_t cj = j0; cj <= j1; ++cj)
                for (uint32_t ci = i0; ci <= i1; ++ci) {
                    size_t c = (size_t)cj * GX + ci;
                    for (uint64_t k = cstart[c]; k < cstart[c + 1]; ++k) {
                        uint32_t id = cell_ids[k];
                        if (orc_in_rect(pos[2 * (size_t)id], pos[2 * (size_t)id + 1], r)) {
                            cnt += 1;
                            if (hashes) h += orc_result_hash(q, id);
                        }
                    }
                }
        }
        counts[q] = cnt;
        if (hashes) hashes[q] = h;
        total += cnt;
    }
    free(cstart); free(cell_of); free(cell_ids); free(fill);
    return (int64_t)total;
}

/* Query-major bitmap of a CSR result (reading of the bitmap layout of the
 * filtering phase, extended to the whole Q x N result): word
 * q * ceil(nmax/32) + id/32, bit id mod 32, least significant bit first. */
void orc_bitmap(const uint64_t *offsets, const uint32_t *ids, uint32_t Q,
                uint32_t nmax, uint32_t *words)
{
    size_t W = ((size_t)nmax + 31) / 32;
    memset(words, 0, (size_t)Q * W * sizeof(uint32_t));
    for (uint32_t q = 0; q < Q; ++q)
        for (uint64_t k = offsets[q]; k < offsets[q + 1]; ++k)
            words[(size_t)q * W + ids[k] / 32] |= 1u << (ids[k] % 32);
}

/* ------------------------------------------------------------------------ */
/* Morton code of the 2^15 x 2^15 grid at l_max = 15 (Sec. 5.3, Alg. 1).     */
/* ------------------------------------------------------------------------ */

/* FP32 cell function: t = (v - lo) * scale in FP32 round-to-nearest;
 * NaN or t < 0 -> 0; t >= 2^15 - 1 -> 2^15 - 1; otherwise floor(t). */
uint32_t orc_cell(float v, float lo, float scale)
{
    volatile float d = v - lo;   /* volatile: keep the two roundings apart */
    volatile float t = d * scale;
    if (!(t >= 0.0f)) return 0;  /* NaN and negatives */
    if (t >= 32767.0f) return 32767;
    return (uint32_t)t;          /* truncation == floor for t >= 0 */
}

/* scale = 2^15 / (x1 - x0), each operation rounded to FP32. */
float orc_scale(float lo, float hi)
{
    volatile float w = hi - lo;
    volatile float s = 32768.0f / w;
    return s;
}

/* z(i, j): bit b of i goes to bit 2b, bit b of j to bit 2b + 1. */
uint32_t orc_morton(uint32_t i, uint32_t j)
{
    uint32_t z = 0;
    for (uint32_t b = 0; b < 15; ++b) {
        z |= ((i >> b) & 1u) << (2 * b);
        z |= ((j >> b) & 1u) << (2 * b + 1);
    }
    return z;
}

/* Keys of all slots: z for present objects, 0xFFFFFFFF for absent ones. */
void orc_keys(const float *pos, const uint8_t *present, uint32_t nmax,
              float x0, float y0, float x1, float y1, uint32_t *keys)
{
    float sx = orc_scale(x0, x1), sy = orc_scale(y0, y1);
    for (uint32_t id = 0; id < nmax; ++id) {
        if (!present[id]) { keys[id] = 0xFFFFFFFFu; continue; }
        uint32_t i = orc_cell(pos[2 * (size_t)id], x0, sx);
        uint32_t j = orc_cell(pos[2 * (size_t)id + 1], y0, sy);
        keys[id] = orc_morton(i, j);
    }
}

/* ------------------------------------------------------------------------ */
/* Alg. 1: PR-quadtree leaves over Morton-sorted keys (l_max levels, the     */
/* key of a point at level l is its l_max key divided by 4^(l_max - l)).     */
/* A quadrant is split iff it holds more than th_quad objects and l < l_max; */
/* quadrants reached at l_max are leaves whatever their size.  The root      */
/* (level 0) is split iff n > th_quad.  Leaves are returned sorted by their  */
/* first l_max key (Morton order), empty leaves included.                    */
/* leaf record: {level, z at that level, begin, end} into the sorted keys.   */
/* Returns the number of leaves, or -1 if out_cap is too small / no memory.  */
/* ------------------------------------------------------------------------ */
typedef struct { uint32_t level, z, begin, end; } orc_leaf;

static int orc_leaf_cmp(const void *a, const void *b)
{
    const orc_leaf *x = (const orc_leaf *)a, *y = (const orc_leaf *)b;
    uint64_t kx = (uint64_t)x->z << (2 * (15 - x->level));
    uint64_t ky = (uint64_t)y->z << (2 * (15 - y->level));
    return (kx > ky) - (kx < ky);
}

/* Split threshold of the quadrant z at level l.  With one global th_quad  */
/* (region_bits = 0, caps = {th_quad}) this is Alg. 1's test.  With          */
/* per-region thresholds the quadrants of level region_bits are regions:     */
/* a quadrant at or below that level takes the threshold of the region that  */
/* contains it, caps[z / 4^(l - region_bits)]; every non-empty quadrant      */
/* above that level is split.                                                */
static uint32_t orc_threshold(uint32_t l, uint32_t z, uint32_t region_bits, const uint32_t *caps)
{
    if (l < region_bits) return 0;
    return caps[z >> (2 * (l - region_bits))];
}

int64_t orc_quadtree_regions(const uint32_t *keys, uint32_t n, uint32_t region_bits, const uint32_t *caps,
                             uint32_t lmax, orc_leaf *out, uint64_t out_cap)
{
    uint64_t nleaf = 0;
    if (lmax > 15 || region_bits > lmax) return -1;
    if (n <= orc_threshold(0, 0, region_bits, caps) || lmax == 0) {
        if (out_cap < 1) return -1;
        out[0].level = 0; out[0].z = 0; out[0].begin = 0; out[0].end = n;
        return 1;
    }
    /* I_A: intervals (z, begin, end) of the quadrants to split at level l-1. */
    uint64_t na = 1, acap = 1024;
    orc_leaf *IA = (orc_leaf *)malloc(acap * sizeof(orc_leaf));
    if (!IA) return -1;
    IA[0].level = 0; IA[0].z = 0; IA[0].begin = 0; IA[0].end = n;
    for (uint32_t l = 1; l <= lmax && na > 0; ++l) {
        uint64_t nn = 0, ncap = 4 * na;
        orc_leaf *next = (orc_leaf *)malloc(ncap * sizeof(orc_leaf));
        if (!next) { free(IA); return -1; }
        uint32_t shift = 2 * (lmax - l);
        for (uint64_t a = 0; a < na; ++a) {
            /* GPUdetectQuadrants: the four child intervals of quadrant a,
             * found by scanning its (sorted) objects. */
            uint32_t pos = IA[a].begin;
            for (uint32_t c = 0; c < 4; ++c) {
                uint32_t zc = IA[a].z * 4 + c;
                uint32_t b = pos;
                while (pos < IA[a].end && (keys[pos] >> shift) == zc) ++pos;
                uint32_t cnt = pos - b;
                /* CPUcheckQuadrants: split or keep as leaf. */
                if (cnt > orc_threshold(l, zc, region_bits, caps) && l < lmax) {
                    next[nn].level = l; next[nn].z = zc; next[nn].begin = b; next[nn].end = pos;
                    ++nn;
                } else {
                    if (nleaf >= out_cap) { free(next); free(IA); return -1; }
                    out[nleaf].level = l; out[nleaf].z = zc; out[nleaf].begin = b; out[nleaf].end = pos;
                    ++nleaf;
                }
            }
        }
        free(IA);
        IA = next;
        na = nn;
        (void)acap;
    }
    free(IA);
    qsort(out, (size_t)nleaf, sizeof(orc_leaf), orc_leaf_cmp);
    return (int64_t)nleaf;
}

int64_t orc_quadtree(const uint32_t *keys, uint32_t n, uint32_t th_quad,
                     uint32_t lmax, orc_leaf *out, uint64_t out_cap)
{
    return orc_quadtree_regions(keys, n, 0, &th_quad, lmax, out, out_cap);
}

/* ------------------------------------------------------------------------ */
/* Def. "Mapping functions": g(q) = the leaves whose cell range meets the    */
/* query's cell range (corners mapped with the same FP32 cell function as    */
/* the objects).  A subquery is covering iff the leaf's cell range lies      */
/* strictly inside the query's cell range on both axes (then every object   */
/* of the leaf passes the FP32 test); otherwise it is intersecting.          */
/* A query with a NaN corner or inverted sides has no subquery.             */
/* Writes leaf indices and covering flags (1/0) in leaf order; returns the  */
/* number of subqueries, or -1 if out_cap is too small.                     */
/* ------------------------------------------------------------------------ */
static uint32_t orc_deinterleave(uint32_t z, uint32_t off)
{
    uint32_t v = 0;
    for (uint32_t b = 0; b < 15; ++b) v |= ((z >> (2 * b + off)) & 1u) << b;
    return v;
}

int64_t orc_subqueries(const orc_leaf *leaves, uint64_t nleaves, int skip_empty,
                       const float *rect, float x0, float y0, float x1, float y1,
                       uint32_t *out_leaf, uint8_t *out_cov, uint64_t out_cap)
{
    if (orc_query_is_empty(rect)) return 0;
    float sx = orc_scale(x0, x1), sy = orc_scale(y0, y1);
    uint32_t i0 = orc_cell(rect[0], x0, sx), i1 = orc_cell(rect[2], x0, sx);
    uint32_t j0 = orc_cell(rect[1], y0, sy), j1 = orc_cell(rect[3], y0, sy);
    uint64_t k = 0;
    for (uint64_t c = 0; c < nleaves; ++c) {
        const orc_leaf *L = leaves + c;
        if (skip_empty && L->begin == L->end) continue;
        uint32_t s = 15 - L->level;
        uint32_t z0 = L->z << (2 * s);
        uint32_t bi0 = orc_deinterleave(z0, 0), bj0 = orc_deinterleave(z0, 1);
        uint32_t bi1 = bi0 + (1u << s) - 1, bj1 = bj0 + (1u << s) - 1;
        if (bi1 < i0 || bi0 > i1 || bj1 < j0 || bj0 > j1) continue;
        if (k >= out_cap) return -1;
        out_leaf[k] = (uint32_t)c;
        out_cov[k] = (bi0 > i0 && bi1 < i1 && bj0 > j0 && bj1 < j1) ? 1 : 0;
        ++k;
    }
    return (int64_t)k;
}
